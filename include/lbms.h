/*
 * lbms.h -- C ABI of a GB300 (sm_103a) lattice Boltzmann solver for
 * multicomponent diffusion after the Maxwell-Stefan multiple-relaxation-time
 * model of Chai, Guo, Wang and Shi (arXiv:1808.06787).
 *
 * The model (Sec. 3.1): n species, of which the first S = n - 1 carry
 * distribution functions f_k^i on a DdQq lattice; the last species follows from
 * the closure sum_i xi_i = 1 (Eq. 2-3b).  One time step is the collision of
 * Eq. 3-13a with the cross-species relaxation matrices Lambda^{ij} followed by
 * the propagation of Eq. 3-13b.  At every node the library evaluates
 *   xi_i = sum_k f_k^i                                       (Eq. 3-15)
 *   B(xi, D_ij)                                              (Eq. 2-10)
 *   Lambda_1 with D~ = B^{-1} = c_s^2 (Lambda_1^{-1} - I/2)   (Eqs. 2-11, 3-26)
 *   Lambda_2 from Lambda_1                                   (Eq. 3-16)
 *   f_eq = w_k xi_i                                          (Eq. 3-3)
 * in lattice units (dx = dt = c = 1, c_t = 1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Fields are species-major and x-fastest: a mole-fraction field is
 *   x[sigma][z][y][x] with sigma = 0..n-1; a flux field is
 *   J[sigma][a][z][y][x] with a = 0..dim-1.  2D lattices use nz = 1.
 * - Element type of every field is the handle's dtype (float or double).
 * - Buffers may be device memory or host memory; the library asks the CUDA
 *   runtime which one a pointer is.  Pinned (page-locked) host buffers are read
 *   or written by the kernels in place, through the device's mapping of pinned
 *   memory (no staging copies); pageable host buffers are copied through a
 *   bounded staging area of the workspace.  A host input is read, and a host
 *   output written, before the call returns.
 * - Everything is ordered on the handle's CUDA stream.  Calls that return data
 *   to host memory (lbms_mass, host outputs of lbms_moments) or read host
 *   inputs (lbms_set_state) synchronise that stream; all other calls are
 *   asynchronous.
 * - The library allocates no device memory.  The caller owns the workspace and
 *   every field buffer.  The handle itself is a small host allocation.
 * - Errors are reported by return code; lbms_last_error() gives a message.
 *   Nothing aborts, exits or traps on the device.  Kernels raise status flags
 *   that lbms_status() reads.
 * - Not thread-safe per handle: one host thread drives a handle at a time.
 */
#ifndef LBMS_H
#define LBMS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbms_s lbms_t;

/* Lattices of Sec. 3.1: D2Q5 (Eq. 3-7), D2Q9 (Eq. 3-8), D3Q7 (Eq. 3-10),
 * D3Q15 (Eq. 3-11), D1Q3 (Eq. 3-5), and the two without a rest velocity, D2Q4
 * (Eq. 3-6) and D3Q6 (Eq. 3-9).  Batched solves and the adjoint entry points
 * take all seven. */
enum {
    LBMS_D2Q5 = 0,
    LBMS_D2Q9 = 1,
    LBMS_D3Q7 = 2,
    LBMS_D3Q15 = 3,
    LBMS_D1Q3 = 4,
    LBMS_D2Q4 = 5,
    LBMS_D3Q6 = 6
};

/* Storage and arithmetic type of the populations and of all fields. */
enum { LBMS_F32 = 0, LBMS_F64 = 1 };

/* Face kinds.  PERIODIC wraps (used in all experiments of Sec. 4); NOFLUX is the
 * half-way bounce-back of Sec. 4, f_k(x_f, t+1) = f+_kbar(x_f, t); DIRICHLET
 * holds a fixed composition xi_b on the face by the half-way anti-bounce-back
 * of Sec. 4, f_k(x_f, t+1) = -f+_kbar(x_f, t) + 2 w_kbar xi_{i,b} (set with
 * lbms_set_boundary).  A D2Q9 diagonal link leaving through two wall faces at
 * a corner takes the kind (and composition) of the first of them in axis
 * order x, y, z.  HALO marks a cut of a slab decomposition (see "Slab
 * decomposition" below): only on the faces of the split axis. */
enum { LBMS_PERIODIC = 0, LBMS_NOFLUX = 1, LBMS_DIRICHLET = 2, LBMS_HALO = 3 };

/* Relaxation of the even moments.  MAGIC: Lambda_2 by Eq. 3-16 (off-diagonal
 * entries equal Lambda_1, diagonal 8 (l - 2) / (l - 8)).  SRT: Lambda_2 =
 * Lambda_1, the single-relaxation-time reduction of Sec. 3.1 used for the
 * comparison of Sec. 4.1.  FROZEN: as MAGIC, but Lambda_1 and Lambda_2 (and D~
 * of the flux) are evaluated at a fixed reference composition set with
 * lbms_set_reference instead of each node's own: the scheme becomes linear,
 * which test suites use to compare against exact Fourier amplification; it is
 * not a model of the paper. */
enum { LBMS_RELAX_MAGIC = 0, LBMS_RELAX_SRT = 1, LBMS_RELAX_FROZEN = 2 };

/* Return codes. */
enum {
    LBMS_OK = 0,
    LBMS_EINVAL = 1,    /* bad argument, size or combination */
    LBMS_ENOMEM = 2,    /* workspace too small */
    LBMS_ECUDA = 3,     /* a CUDA runtime call or kernel launch failed */
    LBMS_ENONFINITE = 4,
    LBMS_ERANGE = 5,
    LBMS_ETIMEOUT = 6
};

/* Status flags raised by kernels (lbms_status). */
#define LBMS_FLAG_NONFINITE 0x1u /* a mole fraction became NaN or infinite */
#define LBMS_FLAG_RANGE 0x2u     /* a mole fraction left [-0.05, 1.05] */
#define LBMS_FLAG_INIT 0x4u      /* lbms_set_state input not finite or not summing to 1 */

/* Largest number of species and largest grid. */
#define LBMS_MAX_SPECIES 8
#define LBMS_MAX_CELLS 2147483647L

/*
 * Bytes of device workspace that lbms_create needs for this problem: two
 * population buffers of S * Q * cells elements (ping-pong), per-block partial
 * sums for the mass diagnostic, a status word, the compositions of Dirichlet
 * faces, the halo buffers of the two faces of the split axis (slab
 * decomposition; a few layers of nodes) and a staging area (at most 16 MiB)
 * for host input/output.  Returns 0 for an invalid combination.
 */
size_t lbms_workspace_size(int lattice, int n_species, const int grid[3], int dtype);

/*
 * Create a solver handle.
 *   out        receives the handle (set to NULL on failure).
 *   lattice    LBMS_D2Q5 | LBMS_D2Q9 | LBMS_D3Q7 | LBMS_D3Q15 | LBMS_D1Q3 |
 *              LBMS_D2Q4 | LBMS_D3Q6 (Sec. 3.1).
 *   n_species  n, 2..8.  S = n - 1 species are evolved (Eq. 3-2, i <= n-1).
 *   grid       {nx, ny, nz}, each >= 1; nz must be 1 for 2D lattices and
 *              ny = nz = 1 for D1Q3; nx * ny * nz <= LBMS_MAX_CELLS.
 *   D          host array of n * n binary Maxwell-Stefan diffusivities D_ij in
 *              lattice units (Eq. 2-7), row-major.  Off-diagonal entries must be
 *              finite, > 0 and symmetric (D_ij = D_ji); the diagonal is ignored.
 *   relax      LBMS_RELAX_MAGIC | LBMS_RELAX_SRT | LBMS_RELAX_FROZEN (the last
 *              needs lbms_set_reference before the first step; the adjoint
 *              entry points reject it).
 *   bc         host array of 6 face kinds {x-low, x-high, y-low, y-high, z-low,
 *              z-high}, each LBMS_PERIODIC, LBMS_NOFLUX or LBMS_DIRICHLET, or
 *              LBMS_HALO on a face of the split axis (slab decomposition); a
 *              periodic face must be paired with a periodic face on the same
 *              axis.  Unused z faces of a 2D lattice are ignored.  Every
 *              Dirichlet face needs lbms_set_boundary before the first step.
 *   dtype      LBMS_F32 | LBMS_F64.
 *   workspace  device memory of at least lbms_workspace_size() bytes, aligned
 *              to 256 bytes, owned by the caller and kept alive until
 *              lbms_destroy.
 *   cuda_stream  cudaStream_t on which all work is ordered (NULL = legacy
 *              default stream).
 * The state is undefined until lbms_set_state.  Returns LBMS_EINVAL or
 * LBMS_ENOMEM for bad arguments, LBMS_ECUDA if the runtime fails.
 */
int lbms_create(lbms_t** out, int lattice, int n_species, const int grid[3], const double* D,
                int relax, const int bc[6], int dtype, void* workspace, size_t workspace_bytes,
                void* cuda_stream);

/*
 * Initialise from mole fractions: f_k^i = w_k xi_i(t = 0) (Sec. 4,
 * initialisation), i.e. the post-collision state at t = 0.  x0 holds all n
 * species, [n][nz][ny][nx] of the handle's dtype, host or device.  Each node
 * must be finite and sum to 1 within 1e-5; otherwise LBMS_FLAG_INIT is raised
 * (read it with lbms_status) and the state is still written.  Resets the step
 * counter to 0.  A host x0 synchronises the stream (it may be reused on return).
 */
int lbms_set_state(lbms_t* h, const void* x0);

/*
 * Set the composition xi_b held on Dirichlet face `face` (0..5 in the order of
 * bc; the face must have been created LBMS_DIRICHLET): xi_b is a host array of
 * all n mole fractions, each in [0, 1] and summing to 1 within 1e-6 (the
 * evolved species' values enter the anti-bounce-back rule of Sec. 4).  The
 * values are copied to the workspace in stream order, so steps already queued
 * keep the old composition and later steps see the new one (time-dependent
 * boundaries).  Synchronises the stream; not callable during stream capture.
 * Returns LBMS_EINVAL for a bad face or composition, LBMS_ECUDA if the copy
 * fails.
 */
int lbms_set_boundary(lbms_t* h, int face, const double* xi_b);

/*
 * Reference composition of a LBMS_RELAX_FROZEN handle: xi_ref is a host array
 * of all n mole fractions, each in [0, 1], summing to 1 within 1e-6.  Applies
 * to the steps and moments issued after the call.  Returns LBMS_EINVAL for
 * another relaxation mode or a bad composition.
 */
int lbms_set_reference(lbms_t* h, const double* xi_ref);

/*
 * Advance n_steps >= 0 time steps of Eqs. 3-13a/3-13b (pull form: each node
 * gathers f+_k(x - c_k), collides, and stores its post-collision populations).
 * The last step of each call also writes per-block partial sums of every
 * species' mole fraction, which lbms_mass reduces when it is called, so
 * lbms_mass after lbms_step reads no populations.  Asynchronous: launch errors are returned at once, numerical
 * trouble is raised in the status flags.  Returns LBMS_EINVAL if a Dirichlet
 * face has no composition yet.  With Dirichlet faces the species' masses are
 * not conserved (the faces exchange mass with the outside).
 */
int lbms_step(lbms_t* h, long n_steps);

/*
 * Mole fractions and diffusion fluxes at the current time t (Sec. 3.2):
 *   x_sigma  [n][nz][ny][nx]: xi_i = sum_k f_k^i for i < n-1, and
 *            xi_n = 1 - sum_i xi_i (Eq. 2-3b).  Required.
 *   J_sigma  [n][dim][nz][ny][nx] or NULL: J_i = -sum_j D~_ij grad xi_j with the
 *            local gradient of Eq. xix, evaluated as J = (I - Lambda_1/2) m_1 of
 *            the pre-collision populations at time t (identical by Eq. 3-26),
 *            and J_n = -sum_i J_i (Eq. 2-3a).  J is zero at t = 0.
 * Host or device buffers; host outputs synchronise the stream.
 */
int lbms_moments(lbms_t* h, void* x_sigma, void* J_sigma);

/*
 * Local mole-fraction gradients at the current time t (Sec. 3.2, Eq. xix):
 *   grad_sigma  [n][dim][nz][ny][nx]: grad xi_i = -(1/c_s^2) sum_j
 *               lambda_1^{ij} sum_k c_k f_k^j of the pre-collision populations
 *               at t (i < n-1; lattice units), and grad xi_n = -sum_i grad xi_i.
 *               Zero at t = 0.  The scheme needs no finite differences: this is
 *               the gradient the collision itself carries (Figs. 6-9 plot
 *               -d(xi)/dx next to J).
 * Host or device buffer; a host buffer synchronises the stream.
 */
int lbms_gradient(lbms_t* h, void* grad_sigma);

/*
 * Total amount of each species, mass_out[i] = sum over nodes of xi_i, for all n
 * species (xi of Eq. 3-15, xi_n by Eq. 2-3b).  FP32 solvers add every node's
 * value as a 64-bit fixed-point number with 2^-k resolution, k = 59 - ceil(log2
 * cells) clamped to [8, 40] (k = 35 for 256^3 nodes), which makes the sum exact
 * and independent of order; FP64 solvers use two-sum compensated FP64
 * accumulation in a fixed order.  Repeated calls on the same state agree bit
 * for bit.  mass_out is a host array of n doubles.  Synchronises the stream.
 */
int lbms_mass(lbms_t* h, double* mass_out);

/*
 * Species totals of a population field without a handle, a workspace or any
 * device allocation.  The paper has no counterpart: this is a service entry
 * point for callers that cannot call cudaMalloc -- real-time loops whose device
 * memory is fixed at start-up (an allocation may block or fail at a bad time),
 * plug-ins whose device memory belongs to a host framework's pool, and
 * monitoring code that reads a population buffer it does not own.
 *   lattice, n_species, grid, dtype  as for lbms_create.
 *   populations  device buffer of S * Q * cells elements of dtype, laid out
 *                [s][k][z][y][x] (the layout of a solver's population buffers:
 *                lbms_populations gives the current one).  Read only.  A
 *                pointer the CUDA runtime does not report as device memory is
 *                rejected with LBMS_EINVAL before any work is queued; the
 *                extent of the buffer cannot be checked and is the caller's
 *                responsibility.
 *   mass_out     n doubles, host or device: sum over nodes of xi_i = sum_k f_k^i
 *                for the n - 1 evolved species and of the closure species, with
 *                the reduction lbms_mass uses (bit-identical to lbms_mass right
 *                after lbms_set_state).
 *   cuda_stream  stream the work is ordered on; a host mass_out synchronises it.
 * The per-block partial sums go to a file-scope device array of 4 MiB that
 * every GPU which loads the library keeps until the process exits; grids whose
 * partials do not fit (one record per block and species of the solver's mass
 * kernel -- blocks of 256 nodes, or of 64 nodes on grids too small to give
 * every SM two blocks of 256 -- 8 bytes for F32 and 16 for F64, above
 * 4 MiB - 256 B: about 134 M node-species in F32 and 67 M in F64) are
 * rejected with LBMS_EINVAL and a message in lbms_last_error(NULL).  The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current and keeps it for the life of the process; make that
 * first call before any stream capture, and do not reset the device
 * (cudaDeviceReset) while the library is loaded.  All calls share the one array
 * and every call overwrites the slots it uses, so calls that overlap on the GPU
 * (other streams, other host threads) race.  Calls no cudaMalloc, cudaFree or
 * allocating library routine.
 */
int lbms_mass_noalloc(int lattice, int n_species, const int grid[3], int dtype,
                      const void* populations, double* mass_out, void* cuda_stream);

/* OR of the status flags raised since lbms_set_state.  The step kernels test
 * the mole fractions on the last step of every lbms_step call (an unstable or
 * corrupted state stays out of range or non-finite, so the test at the end of
 * a call sees it); lbms_set_state tests its input.  Synchronises the stream. */
int lbms_status(lbms_t* h, uint32_t* flags);

/*
 * Checkpoints.  lbms_get_state copies the current post-collision populations,
 * S * Q * cells elements laid out [s][k][z][y][x] (k in the library's velocity
 * order: rest, then opposite pairs), to f_out (host or device).
 * lbms_set_state_raw loads such a buffer and sets the step count to `step`, so
 * that the following steps reproduce a run that had reached step `step` from
 * that state bit for bit (the stochastic rounding of FP32 solvers is keyed by
 * the step count).  Host buffers synchronise the stream.
 */
int lbms_get_state(lbms_t* h, void* f_out);
int lbms_set_state_raw(lbms_t* h, const void* f_in, long step);

/*
 * Recompute `count` forward steps between caller buffers, for checkpointed
 * adjoints: from f_in (post-collision populations at step `step`, layout as
 * lbms_get_state) the state after step + j + 1 is written to
 * f_out + j * S * Q * cells elements, j = 0 .. count-1, bit for bit as
 * lbms_step would produce it (the stochastic rounding is keyed by `step`).
 * Device buffers only; f_out must not overlap f_in.  The handle's own state
 * and step count are left as they were.  Stream-ordered, no mass diagnostic.
 */
int lbms_recompute(lbms_t* h, const void* f_in, long step, int count, void* f_out);

/*
 * Adjoint (reverse-mode derivative) of the step, for gradients of a loss L of
 * the final mole fractions with respect to the binary diffusivities D_ij and
 * the initial field.  It differentiates the model's map f+(t-1) -> f+(t)
 * (propagation Eq. 3-13b, collision Eq. 3-13a with Lambda_1 from Eq. 3-26 and
 * Lambda_2 from Eq. 3-16, f_eq of Eq. 3-3) in exact arithmetic.  Up to 5
 * species.  All buffers are device memory.  The adjoint state lambda has the
 * population layout, S * Q * cells elements of 8 bytes each: an FP64 value for
 * FP64 solvers and, for FP32 solvers, a pair of floats (hi, lo) whose sum is
 * the value (about 48 significant bits).  Plain FP32 storage would lose the
 * small per-step changes of lambda coherently over a long backward sweep.
 * f_prev, grad_x and grad_x0 have the handle's dtype.  The per-node Jacobian
 * runs in the handle's dtype on the deviation of lambda from its weighted mean
 * over the directions, which the step maps to itself.
 *   lbms_adjoint_scratch_size  bytes of the gradient accumulator gacc (8
 *                              bytes per warp of 32 nodes and species pair: an
 *                              FP64 value, or a float pair for FP32 solvers);
 *                              zero it before the first step of a backward
 *                              pass.
 *   lbms_adjoint_seed     lambda(T) from dL/dxi(T) ([n][cells], all species,
 *                         the closure species' entry included).
 *   lbms_adjoint_step     lambda(t-1) from lambda(t) (lam_in != lam_out), given
 *                         the forward populations f+(t-1) of that step;
 *                         accumulates dL/d(1/D) into gacc.
 *   lbms_adjoint_steps    `count` adjoint steps in one call (a segment of a
 *                         checkpointed backward sweep): with f_first = f+(t0)
 *                         and f_rest + j S Q cells = f+(t0 + 1 + j), j = 0 ..
 *                         count - 2 (unused for count <= 1), the steps run from
 *                         t0 + count down to t0 + 1; lambda(t0 + count) is read
 *                         from lam_a and the buffers alternate, so lambda(t0)
 *                         ends in lam_a for even count and in lam_b for odd.
 *                         Same result as `count` calls of lbms_adjoint_step.
 *   lbms_adjoint_initial  dL/dx0 ([n][cells]) from lambda(0) (f+(0) = w_k x0);
 *                         the closure species does not enter the model and
 *                         gets zero.
 *   lbms_adjoint_reduce   dL/dD_pq for the pairs p < q in the order (0,1),
 *                         (0,2), .., (0,n-1), (1,2), .. into dL_dD (host or
 *                         device, n (n-1) / 2 doubles); synchronises the stream.
 */
size_t lbms_adjoint_scratch_size(const lbms_t* h);
int lbms_adjoint_seed(lbms_t* h, const void* grad_x, void* lam);
int lbms_adjoint_step(lbms_t* h, const void* f_prev, const void* lam_in, void* lam_out, void* gacc);
int lbms_adjoint_steps(lbms_t* h, const void* f_first, const void* f_rest, int count, void* lam_a, void* lam_b,
                       void* gacc);
int lbms_adjoint_initial(lbms_t* h, const void* lam0, void* grad_x0);
int lbms_adjoint_reduce(lbms_t* h, const void* gacc, double* dL_dD);

/* Number of steps taken since lbms_set_state, or -1 for a NULL handle. */
long lbms_steps_done(const lbms_t* h);

/* Device address, inside the caller's workspace, of the buffer that holds the
 * current post-collision populations (layout as lbms_get_state).  It changes
 * with every step (the two buffers alternate) and after lbms_set_state_raw;
 * NULL for a NULL handle. */
const void* lbms_populations(const lbms_t* h);

/* Message of the last failed call on this handle ("" if none).  With h == NULL,
 * the message of the last failed lbms_create on this thread. */
const char* lbms_last_error(const lbms_t* h);

/* Release the handle.  Does not free the caller's workspace. */
void lbms_destroy(lbms_t* h);

/* ========================================================================= */
/* Slab decomposition: one grid split into slabs along its split axis -- the  */
/* lattice's last axis (z for D3Q7, D3Q15, D3Q6; y for D2Q5, D2Q9, D2Q4; x    */
/* for D1Q3), so that a layer of nodes is contiguous -- each slab a handle of */
/* its own (on one GPU, or one per GPU), with one exchange per time step.     */
/* ========================================================================= */
/*
 * The propagation of Eq. 3-13b is nearest-neighbour: a step of a slab needs,
 * beyond its own populations, only the populations of the neighbouring slabs'
 * boundary layers that cross the cut towards it (1 per species and node for
 * D2Q5, D3Q7, D2Q4, D3Q6 and D1Q3, 3 for D2Q9, 5 for D3Q15).  A slab is a handle
 * created with LBMS_HALO on the faces of the split axis that are cuts (the
 * slab's grid is its own share of the layers; the other axes and their faces
 * are those of the whole grid; a wrapping split axis makes both ends cuts).
 * Every step also writes the slab's own crossing populations into a send
 * buffer per cut face; before each step the caller copies each neighbour's
 * send buffer into this slab's receive buffer of the same face, and the step
 * reads it as the populations beyond the cut.  Fields, masses (lbms_mass) and
 * fluxes of a slab are those of its own nodes.
 *
 * lbms_set_subdomain    sets the index, in the undivided grid, of the slab's
 *                       first layer along the split axis.  FP32 solvers key
 *                       their stochastic rounding by the node index, so with
 *                       it the slabs of a decomposed run evolve bit for bit as
 *                       the undivided grid does.  Call before the first step.
 * lbms_halo_buffers     device addresses (inside the workspace) of the send
 *                       buffer of cut face `face` (0..5, as bc) and of the
 *                       receive buffer the next step reads, and their size in
 *                       bytes; the layout of both is [populations crossing the
 *                       face][S][layer nodes].  The receive buffer alternates
 *                       with the population buffers, so ask again before every
 *                       exchange.  lbms_set_state fills the send buffers too.
 * lbms_slab_step        n_steps steps of `count` slabs of one grid on one GPU,
 *                       given in split-axis order, all on one stream and at the
 *                       same step: each step copies the send buffers into the
 *                       neighbours' receive buffers (device-to-device) and then
 *                       steps every slab.  Errors go to lbms_last_error(subs[0])
 *                       (or lbms_last_error(NULL) for NULL arguments).
 * lbms_step on a slab with LBMS_HALO faces takes n_steps <= 1 (the exchange
 * belongs between steps).  lbms_set_state_raw, lbms_recompute and the adjoint
 * entry points reject slabs; batched solves do not take LBMS_HALO.
 */
int lbms_set_subdomain(lbms_t* h, long first_layer);
int lbms_halo_buffers(lbms_t* h, int face, void** send, void** recv, size_t* bytes);
int lbms_slab_step(lbms_t* const* subs, int count, long n_steps);

/* ========================================================================= */
/* Batched solves: many independent problems of one lattice, species count   */
/* and dtype, each with its own grid, diffusivities and faces, stepped        */
/* together (the model of Sec. 3.1 applied to every instance).                */
/* ========================================================================= */

typedef struct lbms_batch_s lbms_batch_t;

/* Number of step candidates lbms_batch_tune chooses from: 7 schedules x 2
 * kernel shapes. */
#define LBMS_BATCH_CANDIDATES 14

/*
 * Workspace bytes for `count` instances with grids[3 * i + {0,1,2}] = {nx, ny,
 * nz} of instance i (0 for an invalid combination).  Instance i owns
 * ceil(cells_i / 256) * 256 node slots of one shared node space; the
 * workspace holds two population buffers over that space, per-block mass
 * partials, the instance tables and a staging area for host I/O (at least the
 * largest instance's fields, at least 16 MiB).
 */
size_t lbms_batch_workspace_size(int lattice, int n_species, int count, const int* grids, int dtype);

/*
 * Create a batch.  lattice, n_species, relax, dtype, workspace and cuda_stream
 * as for lbms_create; the total node slots must stay below LBMS_MAX_CELLS.
 *   grids  host array of count * 3 extents.
 *   D      host array of count * n * n diffusivities (instance-major), each
 *          block symmetric with positive off-diagonal entries.
 *   bc     host array of count * 6 face kinds as for lbms_create (periodic,
 *          no-flux or Dirichlet; Dirichlet faces need
 *          lbms_batch_set_boundary before the first step), or NULL for all
 *          periodic.
 * Errors as for lbms_create (messages via lbms_batch_last_error(NULL)).
 */
int lbms_batch_create(lbms_batch_t** out, int lattice, int n_species, int count, const int* grids,
                      const double* D, int relax, const int* bc, int dtype, void* workspace,
                      size_t workspace_bytes, void* cuda_stream);

/*
 * Initialise every instance from mole fractions (Sec. 4 initialisation, as
 * lbms_set_state).  Instance i's field is [n][nz][ny][nx] at element offset
 * offsets[i] of x0; offsets == NULL means packed (instance after instance).
 * x0 may be host or device memory; a host x0 synchronises the stream (it may
 * be reused on return).
 */
int lbms_batch_set_state(lbms_batch_t* b, const void* x0, const int64_t* offsets);

/*
 * Advance every instance by n_steps (Eqs. 3-13a/3-13b), with the candidate
 * (schedule and kernel shape) chosen by lbms_batch_tune or
 * lbms_batch_set_schedule (default: all instances per launch, see below).
 * Each instance evolves exactly as lbms_step would
 * evolve it alone, bit for bit.  The last step writes the mass partials.
 */
int lbms_batch_step(lbms_batch_t* b, long n_steps);

/*
 * Mole fractions (and fluxes if J_sigma != NULL) of every instance, as
 * lbms_moments: instance i's x block at element offsets[i] of x_sigma and its
 * J block ([n][dim][cells]) at element dim * offsets[i] of J_sigma; offsets ==
 * NULL means packed.  Host or device buffers; synchronises the stream.
 */
int lbms_batch_moments(lbms_batch_t* b, void* x_sigma, void* J_sigma, const int64_t* offsets);

/*
 * Composition xi_b (host array of all n mole fractions) held on Dirichlet face
 * `face` (0..5) of instance `instance`, as lbms_set_boundary for a single
 * solve: stream-ordered, synchronises the stream; LBMS_EINVAL for a face that
 * is not Dirichlet or a bad composition.
 */
int lbms_batch_set_boundary(lbms_batch_t* b, int instance, int face, const double* xi_b);

/* Per-instance species totals, mass_out[i * n + s], as lbms_mass.  Host array;
 * synchronises the stream. */
int lbms_batch_mass(lbms_batch_t* b, double* mass_out);

/* OR of the status flags of all instances.  Synchronises the stream. */
int lbms_batch_status(lbms_batch_t* b, uint32_t* flags);

/*
 * Step candidates c = schedule + 7 * shape.  Schedules (c % 7): 0 streams all
 * instances through HBM every step (CUDA graph of 32 steps); 1..6 run groups
 * of consecutive instances whose two population buffers fit in 24, 24, 48,
 * 48, 96, 96 MB for 8 or 32 steps each (chunk 8, 32, 8, 32, 8, 32), so that a
 * group stays in L2 between its steps.  Kernel shapes (c / 7): 0 takes one
 * node per thread (blocks of 256 threads), 1 two nodes per thread (blocks of
 * 128 threads over the same 256-node blocks; paired loads of the rest
 * populations and paired stores), available for D2Q5, D1Q3 and D2Q4 with
 * n <= 3 in F32 only
 * (LBMS_EINVAL otherwise).  The default is candidate 7 where shape 1 exists,
 * else 0.  Results do not depend on the candidate.  lbms_batch_get_schedule
 * returns the current candidate.
 */
int lbms_batch_set_schedule(lbms_batch_t* b, int candidate);
int lbms_batch_get_schedule(const lbms_batch_t* b);

/* Kernel launches one step takes under the current schedule (1 for the
 * streamed schedule, the number of instance groups otherwise); a call of
 * lbms_batch_step(n) launches n times this many step kernels and one mass
 * reduction.  -1 for a NULL handle. */
int lbms_batch_launches_per_step(const lbms_batch_t* b);

/*
 * Candidate tuner: times every candidate over trial_steps steps (after one
 * untimed warm-up of the same length), keeps the fastest and returns it in
 * *chosen; ms_per_step, if not NULL, receives LBMS_BATCH_CANDIDATES timings
 * (-1 for the candidates this batch cannot run).
 * It advances the instances by up to 2 * LBMS_BATCH_CANDIDATES * trial_steps
 * steps: call it before lbms_batch_set_state.
 */
int lbms_batch_tune(lbms_batch_t* b, int trial_steps, double* ms_per_step, int* chosen);

long lbms_batch_steps_done(const lbms_batch_t* b);
const char* lbms_batch_last_error(const lbms_batch_t* b);
void lbms_batch_destroy(lbms_batch_t* b);

#ifdef __cplusplus
}
#endif

#endif /* LBMS_H */
