// Host runtime behind the C ABI of include/lbms.h: argument checks, workspace
// layout, ping-pong buffers, CUDA-graph replay of step runs, host staging and
// the deterministic mass reduction.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <new>

#include "adjoint.cuh"
#include "lbms_internal.h"
#include "node.cuh"

using namespace lbms;

namespace {

constexpr size_t kAlign = 256;
constexpr size_t kStagingMax = size_t(16) << 20;  // host I/O chunk area
constexpr int kGraphSteps = 32;                   // steps per captured graph (even)
// captured run lengths: full runs of kGraphSteps, then the even remainder in
// binary pieces (all even, so a run leaves the buffer parity unchanged)
constexpr int kGraphLens[5] = {kGraphSteps, 16, 8, 4, 2};
// calls of at most kCallGraphMax steps are replayed whole: the plain steps and
// the mass-writing last one in one graph, kept for the kCallGraphs most
// recently used (length, parity) pairs
constexpr long kCallGraphMax = 64;
constexpr int kCallGraphs = 4;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

int lattice_q(int lat)
{
    switch (lat) {
        case LBMS_D2Q5: return 5;
        case LBMS_D2Q9: return 9;
        case LBMS_D3Q7: return 7;
        case LBMS_D3Q15: return 15;
        case LBMS_D1Q3: return 3;
        case LBMS_D2Q4: return 4;
        case LBMS_D3Q6: return 6;
        default: return 0;
    }
}
int lattice_dim(int lat)
{
    return lat == LBMS_D3Q7 || lat == LBMS_D3Q15 || lat == LBMS_D3Q6 ? 3 : (lat == LBMS_D1Q3 ? 1 : 2);
}

struct Layout {
    size_t f_bytes, off_f0, off_f1, off_partials, off_mass, off_status, off_bound, off_halo,
        halo_bytes, off_staging, staging_bytes, total;
};

// Populations crossing a cut of the split axis in one direction.
int lattice_halo_width(int lat)
{
    switch (lat) {
        case LBMS_D2Q5: return halo_width<LBMS_D2Q5>();
        case LBMS_D2Q9: return halo_width<LBMS_D2Q9>();
        case LBMS_D3Q7: return halo_width<LBMS_D3Q7>();
        case LBMS_D3Q15: return halo_width<LBMS_D3Q15>();
        case LBMS_D1Q3: return halo_width<LBMS_D1Q3>();
        case LBMS_D2Q4: return halo_width<LBMS_D2Q4>();
        case LBMS_D3Q6: return halo_width<LBMS_D3Q6>();
        default: return 0;
    }
}

// Nodes per layer of the split axis (the slowest axis of the lattice's dimension).
size_t split_plane(int lat, const int grid[3])
{
    const int dim = lattice_dim(lat);
    return dim == 3 ? (size_t)grid[0] * grid[1] : (dim == 2 ? (size_t)grid[0] : 1);
}

bool make_layout(int lat, int n, const int grid[3], int dtype, Layout* L)
{
    const int Q = lattice_q(lat);
    if (!Q || n < 2 || n > LBMS_MAX_SPECIES || !grid) return false;
    if (dtype != LBMS_F32 && dtype != LBMS_F64) return false;
    if (grid[0] < 1 || grid[1] < 1 || grid[2] < 1) return false;
    if (lattice_dim(lat) < 3 && grid[2] != 1) return false;
    if (lattice_dim(lat) == 1 && grid[1] != 1) return false;
    const double cells_d = (double)grid[0] * grid[1] * grid[2];
    if (cells_d > (double)LBMS_MAX_CELLS) return false;
    const size_t cells = (size_t)grid[0] * grid[1] * grid[2];
    const size_t es = dtype == LBMS_F64 ? 8 : 4;
    const int dim = lattice_dim(lat);
    L->f_bytes = align_up((size_t)(n - 1) * Q * cells * es);
    L->off_f0 = 0;
    L->off_f1 = L->f_bytes;
    L->off_partials = 2 * L->f_bytes;
    const size_t blocks = partial_slots((uint32_t)cells);
    L->off_mass = L->off_partials + align_up(blocks * n * sizeof(double2));
    L->off_status = L->off_mass + align_up(LBMS_MAX_SPECIES * sizeof(double));
    L->off_bound = L->off_status + kAlign;
    L->off_halo = L->off_bound + align_up(6 * LBMS_MAX_SPECIES * sizeof(double));
    // slab cuts: per face of the split axis a send buffer and one receive buffer
    // per population-buffer parity, [halo_width][S][plane] each
    L->halo_bytes = align_up((size_t)lattice_halo_width(lat) * (n - 1) * split_plane(lat, grid) * es);
    L->off_staging = L->off_halo + 6 * L->halo_bytes;
    size_t want = (size_t)n * (1 + dim) * cells * es;
    L->staging_bytes = align_up(want < kStagingMax ? want : kStagingMax);
    L->total = L->off_staging + L->staging_bytes;
    return true;
}

thread_local char g_create_error[256] = "";

// Final fixed-order reduction of the per-block mass partials, one block of
// kFinalize threads per species (many loads in flight: the partials of a large
// grid number tens of thousands).  FP32 solvers: exact int64 fixed-point sums
// scaled by 2^-shift.
constexpr int kFinalize = 1024;

__global__ void __launch_bounds__(kFinalize) k_mass_finalize_fixed(const long long* __restrict__ partials,
                                                                   uint32_t blocks, int n, int shift,
                                                                   double* __restrict__ out)
{
    __shared__ long long red[kFinalize / 32];
    const int s = blockIdx.x;
    long long acc = 0;
#pragma unroll 8
    for (uint32_t b = threadIdx.x; b < blocks; b += blockDim.x) acc += partials[(size_t)b * n + s];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (warp == 0) {
        acc = lane < (int)(blockDim.x >> 5) ? red[lane] : 0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
        if (lane == 0) out[s] = ldexp((double)acc, -shift);
    }
}

// FP64 solvers: two-sum pairs merged in a fixed order.
__global__ void __launch_bounds__(kFinalize) k_mass_finalize_pairs(const double2* __restrict__ partials,
                                                                   uint32_t blocks, int n,
                                                                   double* __restrict__ out)
{
    __shared__ double2 red[kFinalize / 32];
    const int s = blockIdx.x;
    double sum = 0.0, comp = 0.0;
#pragma unroll 4
    for (uint32_t b = threadIdx.x; b < blocks; b += blockDim.x) {
        const double2 v = partials[(size_t)b * n + s];
        two_sum_merge(sum, comp, v.x, v.y);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double s2 = __shfl_down_sync(0xffffffffu, sum, off);
        const double c2 = __shfl_down_sync(0xffffffffu, comp, off);
        two_sum_merge(sum, comp, s2, c2);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = make_double2(sum, comp);
    __syncthreads();
    if (warp == 0) {
        sum = lane < (int)(blockDim.x >> 5) ? red[lane].x : 0.0;
        comp = lane < (int)(blockDim.x >> 5) ? red[lane].y : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const double s2 = __shfl_down_sync(0xffffffffu, sum, off);
            const double c2 = __shfl_down_sync(0xffffffffu, comp, off);
            two_sum_merge(sum, comp, s2, c2);
        }
        if (lane == 0) out[s] = sum + comp;
    }
}

__global__ void k_set_word(uint32_t* w, uint32_t v) { *w = v; }

struct GradScale {
    double v[16];  // 1 / D_pq^2 per pair
};

// dL/dD_pq = -(1/D_pq^2) sum over the warps' slots of the accumulated dL/dc_pq
// (c = 1/D), one block per pair, fixed order.
__global__ void k_adjoint_reduce(const double* __restrict__ gacc, uint32_t slots, int np, int pairs_f32,
                                 GradScale gs, double* __restrict__ out)
{
    __shared__ double2 red[kBlock / 32];
    const int q = blockIdx.x;
    double sum = 0.0, comp = 0.0;
    for (uint32_t b = threadIdx.x; b < slots; b += blockDim.x) {
        if (pairs_f32) {  // FP32 solvers: (hi, lo) float pairs
            const float2 v = reinterpret_cast<const float2*>(gacc)[(size_t)b * np + q];
            two_sum_add(sum, comp, (double)v.x);
            two_sum_add(sum, comp, (double)v.y);
        } else {
            two_sum_add(sum, comp, gacc[(size_t)b * np + q]);
        }
    }
    block_reduce_pair(sum, comp, red);
    if (threadIdx.x == 0) out[q] = -(sum + comp) * gs.v[q];
}

// Fraction bits of the fixed-point mass partials: the sum of |xi| <= 4 over all
// nodes must stay below 2^62.
int fixed_shift_for(uint32_t cells)
{
    int l = 0;
    while ((1ull << l) < cells) ++l;
    int k = 62 - l - 3;
    return k > 40 ? 40 : (k < 8 ? 8 : k);
}

}  // namespace

struct lbms_s {
    int lattice = 0, n = 0, S = 0, Q = 0, dim = 0, dtype = 0, relax = 0;
    int nx = 1, ny = 1, nz = 1;
    uint32_t cells = 0, blocks = 0;  // blocks: of the step and mass kernels (mass partial slots)
    uint32_t step_block = 256;        // their threads per block
    uint32_t noflux = 0;
    uint32_t dirichlet = 0;  // Dirichlet faces
    uint32_t halo = 0;       // slab cut faces (LBMS_HALO)
    uint32_t plane = 1;      // nodes per layer of the split axis
    uint32_t origin = 0;     // global index of node 0 (lbms_set_subdomain)
    void* halo_send[2] = {nullptr, nullptr};                // [face: low, high]
    void* halo_recv[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [parity][face]
    uint32_t xb_set = 0;     // Dirichlet faces whose composition has been set
    void* xb = nullptr;      // device [6][S] compositions of the Dirichlet faces, solver dtype
    size_t es = 4;
    double invD[LBMS_MAX_SPECIES][LBMS_MAX_SPECIES] = {};
    double xref[LBMS_MAX_SPECIES] = {};  // reference composition (frozen mode)
    bool xref_set = false;
    char* ws = nullptr;
    Layout lay{};
    void* f[2] = {nullptr, nullptr};
    int cur = 0;  // f[cur] holds the post-collision populations at time t
    void* partials = nullptr;
    int fixed_shift = 32;
    double* mass_dev = nullptr;
    bool partials_valid = false;  // the mass partials are those of the current state
    bool mass_valid = false;      // mass_dev holds their reduction
    uint32_t* status = nullptr;
    uint32_t* clock = nullptr;  // two step-counter words after the status word
    char* staging = nullptr;
    cudaStream_t stream = nullptr;
    cudaStream_t capture = nullptr;
    // captured runs of kGraphLens[j] plain steps starting from buffer parity p
    cudaGraphExec_t graph[2][5] = {};
    struct CallGraph {
        long n = 0;      // steps of the call
        int parity = 0;  // buffer parity it starts from
        unsigned long long used = 0;
        cudaGraphExec_t exec = nullptr;
    } call_graph[kCallGraphs];
    unsigned long long call_tick = 0;
    bool graphs_ok = true;
    long steps = 0;
    char err[512] = "";
};

namespace {

int fail(lbms_t* h, int code, const char* fmt, ...)
{
    char* buf = h ? h->err : g_create_error;
    size_t cap = h ? sizeof(h->err) : sizeof(g_create_error);
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, cap, fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(lbms_t* h, cudaError_t e, const char* what)
{
    return fail(h, LBMS_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

cudaError_t dispatch(const lbms_t* h, Op op, const KArgs& a)
{
    switch (h->lattice) {
        case LBMS_D2Q5: return dispatch_d2q5(op, h->dtype, a);
        case LBMS_D2Q9: return dispatch_d2q9(op, h->dtype, a);
        case LBMS_D3Q7: return dispatch_d3q7(op, h->dtype, a);
        case LBMS_D3Q15: return dispatch_d3q15(op, h->dtype, a);
        case LBMS_D1Q3: return dispatch_d1q3(op, h->dtype, a);
        case LBMS_D2Q4: return dispatch_d2q4(op, h->dtype, a);
        default: return dispatch_d3q6(op, h->dtype, a);
    }
}

cudaError_t adj_dispatch(const lbms_t* h, AdjOp op, const AArgs& a)
{
    switch (h->lattice) {
        case LBMS_D2Q5: return adj_dispatch_d2q5(op, h->dtype, a);
        case LBMS_D2Q9: return adj_dispatch_d2q9(op, h->dtype, a);
        case LBMS_D3Q7: return adj_dispatch_d3q7(op, h->dtype, a);
        case LBMS_D3Q15: return adj_dispatch_d3q15(op, h->dtype, a);
        case LBMS_D1Q3: return adj_dispatch_d1q3(op, h->dtype, a);
        case LBMS_D2Q4: return adj_dispatch_d2q4(op, h->dtype, a);
        default: return adj_dispatch_d3q6(op, h->dtype, a);
    }
}

KArgs base_args(const lbms_t* h, cudaStream_t st)
{
    KArgs a;
    a.nx = h->nx; a.ny = h->ny; a.nz = h->nz;
    a.cells = h->cells;
    a.step_block = h->step_block;
    a.noflux = h->noflux;
    a.dirichlet = h->dirichlet;
    a.xb = h->xb;
    a.halo = h->halo;
    a.plane = h->plane;
    a.origin = h->origin;
    a.halo_send[0] = h->halo_send[0];
    a.halo_send[1] = h->halo_send[1];
    a.relax = h->relax;
    a.n_species = h->n;
    memcpy(a.invD, h->invD, sizeof(a.invD));
    memcpy(a.xref, h->xref, sizeof(a.xref));
    a.status = h->status;
    a.fixed_shift = h->fixed_shift;
    a.stream = st;
    return a;
}

// One step from f[src] into f[1 - src], optionally with mass partials.
cudaError_t launch_step(const lbms_t* h, int src, bool mass, cudaStream_t st)
{
    KArgs a = base_args(h, st);
    a.fin = h->f[src];
    a.fout = h->f[1 - src];
    a.halo_recv[0] = h->halo_recv[src][0];
    a.halo_recv[1] = h->halo_recv[src][1];
    a.partials = h->partials;
    a.clock_in = h->clock + src;
    a.clock_out = h->clock + (1 - src);
    // steps alternate their direction through the grid: each starts where the
    // one before ended, whose last writes are still in L2
    a.reverse = src;
    return dispatch(h, mass ? OP_STEP_MASS : OP_STEP, a);
}

cudaError_t launch_finalize(const lbms_t* h, cudaStream_t st)
{
    if (h->dtype == LBMS_F32)
        k_mass_finalize_fixed<<<h->n, kFinalize, 0, st>>>(static_cast<const long long*>(h->partials),
                                                         h->blocks, h->n, h->fixed_shift, h->mass_dev);
    else
        k_mass_finalize_pairs<<<h->n, kFinalize, 0, st>>>(static_cast<const double2*>(h->partials),
                                                         h->blocks, h->n, h->mass_dev);
    return cudaGetLastError();
}

// Capture kGraphSteps plain steps starting from buffer `parity`.
// The captured graphs hold the kernel arguments: dropped whenever those change.
void drop_graphs(lbms_t* h)
{
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 5; ++j)
            if (h->graph[i][j]) {
                cudaGraphExecDestroy(h->graph[i][j]);
                h->graph[i][j] = nullptr;
            }
    for (auto& c : h->call_graph) {
        if (c.exec) cudaGraphExecDestroy(c.exec);
        c = lbms_t::CallGraph{};
    }
}

// One whole call: n - 1 plain steps and the mass-writing one from parity p.
cudaError_t build_call_graph(lbms_t* h, long n, int parity, cudaGraphExec_t* out)
{
    cudaError_t e = cudaStreamBeginCapture(h->capture, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t le = cudaSuccess;
    int src = parity;
    for (long i = 0; i < n && le == cudaSuccess; ++i) {
        le = launch_step(h, src, i == n - 1, h->capture);
        src = 1 - src;
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(h->capture, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return le;
    }
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    return e;
}

// The graph of a call of n steps from the current parity (built on first use,
// replacing the least recently used one), or null when it cannot be captured.
cudaGraphExec_t call_graph_for(lbms_t* h, long n)
{
    lbms_t::CallGraph* slot = &h->call_graph[0];
    for (auto& c : h->call_graph) {
        if (c.exec && c.n == n && c.parity == h->cur) {
            c.used = ++h->call_tick;
            return c.exec;
        }
        if (c.used < slot->used) slot = &c;
    }
    if (slot->exec) cudaGraphExecDestroy(slot->exec);
    *slot = lbms_t::CallGraph{};
    cudaGraphExec_t g = nullptr;
    if (build_call_graph(h, n, h->cur, &g) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    slot->n = n;
    slot->parity = h->cur;
    slot->used = ++h->call_tick;
    slot->exec = g;
    return g;
}

cudaError_t build_graph(lbms_t* h, int parity, int j)
{
    cudaError_t e = cudaStreamBeginCapture(h->capture, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t le = cudaSuccess;
    int src = parity;
    for (int i = 0; i < kGraphLens[j] && le == cudaSuccess; ++i) {
        le = launch_step(h, src, false, h->capture);
        src = 1 - src;
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(h->capture, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return le;
    }
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(&h->graph[parity][j], g, 0);
    cudaGraphDestroy(g);
    return e;
}

}  // namespace

namespace lbms {

int mass_fixed_shift(uint32_t cells) { return fixed_shift_for(cells); }

bool is_device_ptr(const void* p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

void* pinned_alias(const void* p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

cudaError_t device_sm_count(int* sms)
{
    static std::mutex mu;
    static int cached[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0 || dev >= 64 || !cached[dev]) {
        int v = 0;
        e = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        v = v < 1 ? 1 : (v > kMaxSms ? kMaxSms : v);
        if (dev < 0 || dev >= 64) {
            *sms = v;
            return cudaSuccess;
        }
        cached[dev] = v;
    }
    *sms = cached[dev];
    return cudaSuccess;
}

cudaError_t launch_mass_reduce(int dtype, const void* partials, uint32_t blocks, int n, int shift,
                               double* out, cudaStream_t stream)
{
    if (dtype == LBMS_F32)
        k_mass_finalize_fixed<<<n, kFinalize, 0, stream>>>(static_cast<const long long*>(partials), blocks,
                                                          n, shift, out);
    else
        k_mass_finalize_pairs<<<n, kFinalize, 0, stream>>>(static_cast<const double2*>(partials), blocks, n,
                                                          out);
    return cudaGetLastError();
}

int set_call_error(int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_create_error, sizeof(g_create_error), fmt, ap);
    va_end(ap);
    return code;
}

}  // namespace lbms

extern "C" {

size_t lbms_workspace_size(int lattice, int n_species, const int grid[3], int dtype)
{
    Layout L;
    return make_layout(lattice, n_species, grid, dtype, &L) ? L.total : 0;
}

int lbms_create(lbms_t** out, int lattice, int n_species, const int grid[3], const double* D,
                int relax, const int bc[6], int dtype, void* workspace, size_t workspace_bytes,
                void* cuda_stream)
{
    g_create_error[0] = '\0';
    if (!out) return fail(nullptr, LBMS_EINVAL, "out is NULL");
    *out = nullptr;
    Layout L;
    if (!make_layout(lattice, n_species, grid, dtype, &L))
        return fail(nullptr, LBMS_EINVAL, "invalid lattice/species/grid/dtype combination");
    if (relax != LBMS_RELAX_MAGIC && relax != LBMS_RELAX_SRT && relax != LBMS_RELAX_FROZEN)
        return fail(nullptr, LBMS_EINVAL, "invalid relaxation mode %d", relax);
    if (!D || !bc) return fail(nullptr, LBMS_EINVAL, "D and bc must not be NULL");
    if (!workspace) return fail(nullptr, LBMS_EINVAL, "workspace is NULL");
    if ((uintptr_t)workspace % kAlign)
        return fail(nullptr, LBMS_EINVAL, "workspace must be 256-byte aligned");
    if (workspace_bytes < L.total)
        return fail(nullptr, LBMS_ENOMEM, "workspace holds %zu bytes, %zu needed", workspace_bytes,
                    L.total);
    const int n = n_species;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            if (i == j) continue;
            const double d = D[i * n + j];
            if (!(isfinite(d) && d > 0.0))
                return fail(nullptr, LBMS_EINVAL, "D[%d][%d] = %g is not finite and positive", i, j, d);
            if (d != D[j * n + i])
                return fail(nullptr, LBMS_EINVAL, "D is not symmetric at (%d, %d)", i, j);
        }
    const int dim = lattice_dim(lattice);
    uint32_t noflux = 0, dirichlet = 0, halo = 0;
    for (int a = 0; a < dim; ++a) {
        const int lo = bc[2 * a], hi = bc[2 * a + 1];
        if (lo < LBMS_PERIODIC || lo > LBMS_HALO || hi < LBMS_PERIODIC || hi > LBMS_HALO)
            return fail(nullptr, LBMS_EINVAL, "invalid face kind on axis %d", a);
        if ((lo == LBMS_HALO || hi == LBMS_HALO) && a != dim - 1)
            return fail(nullptr, LBMS_EINVAL,
                        "LBMS_HALO faces belong to the split axis (the lattice's last axis), not axis %d", a);
        if ((lo == LBMS_PERIODIC) != (hi == LBMS_PERIODIC))
            return fail(nullptr, LBMS_EINVAL, "a periodic face must be paired on axis %d", a);
        if (lo == LBMS_NOFLUX) noflux |= 1u << (2 * a);
        if (hi == LBMS_NOFLUX) noflux |= 1u << (2 * a + 1);
        if (lo == LBMS_DIRICHLET) dirichlet |= 1u << (2 * a);
        if (hi == LBMS_DIRICHLET) dirichlet |= 1u << (2 * a + 1);
        if (lo == LBMS_HALO) halo |= 1u << (2 * a);
        if (hi == LBMS_HALO) halo |= 1u << (2 * a + 1);
    }
    int sms = 0;
    cudaError_t se = device_sm_count(&sms);
    if (se != cudaSuccess) return fail(nullptr, LBMS_ECUDA, "device query: %s", cudaGetErrorString(se));
    lbms_t* h = new (std::nothrow) lbms_t;
    if (!h) return fail(nullptr, LBMS_ENOMEM, "host allocation failed");
    h->lattice = lattice;
    h->n = n;
    h->S = n - 1;
    h->Q = lattice_q(lattice);
    h->dim = dim;
    h->dtype = dtype;
    h->relax = relax;
    h->nx = grid[0]; h->ny = grid[1]; h->nz = grid[2];
    h->cells = (uint32_t)((size_t)grid[0] * grid[1] * grid[2]);
    h->blocks = step_blocks(h->cells, sms);
    h->step_block = step_block_for(h->cells, sms);
    h->noflux = noflux;
    h->dirichlet = dirichlet;
    h->halo = halo;
    h->plane = (uint32_t)split_plane(lattice, grid);
    h->es = dtype == LBMS_F64 ? 8 : 4;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) h->invD[i][j] = i == j ? 0.0 : 1.0 / D[i * n + j];
    h->ws = static_cast<char*>(workspace);
    h->lay = L;
    h->f[0] = h->ws + L.off_f0;
    h->f[1] = h->ws + L.off_f1;
    h->partials = h->ws + L.off_partials;
    h->fixed_shift = fixed_shift_for(h->cells);
    h->mass_dev = reinterpret_cast<double*>(h->ws + L.off_mass);
    h->status = reinterpret_cast<uint32_t*>(h->ws + L.off_status);
    h->clock = h->status + 16;
    h->staging = h->ws + L.off_staging;
    h->xb = h->ws + L.off_bound;
    for (int f = 0; f < 2; ++f) {
        h->halo_send[f] = h->ws + L.off_halo + (size_t)(3 * f) * L.halo_bytes;
        h->halo_recv[0][f] = h->ws + L.off_halo + (size_t)(3 * f + 1) * L.halo_bytes;
        h->halo_recv[1][f] = h->ws + L.off_halo + (size_t)(3 * f + 2) * L.halo_bytes;
    }
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaStreamCreateWithFlags(&h->capture, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete h;
        return fail(nullptr, LBMS_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
    }
    e = cudaMemsetAsync(h->status, 0, sizeof(uint32_t), h->stream);
    if (e != cudaSuccess) {
        cudaStreamDestroy(h->capture);
        delete h;
        return fail(nullptr, LBMS_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    }
    *out = h;
    return LBMS_OK;
}

int lbms_set_state(lbms_t* h, const void* x0)
{
    if (!h) return LBMS_EINVAL;
    if (!x0) return fail(h, LBMS_EINVAL, "x0 is NULL");
    h->err[0] = '\0';
    cudaError_t e = cudaMemsetAsync(h->status, 0, sizeof(uint32_t), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->clock, 0, 2 * sizeof(uint32_t), h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemsetAsync");
    h->cur = 0;
    h->steps = 0;
    h->partials_valid = false;
    h->mass_valid = false;
    KArgs a = base_args(h, h->stream);
    a.fout = h->f[0];
    const void* alias = pinned_alias(x0);
    if (alias || is_device_ptr(x0)) {
        // device memory, or pinned host memory read by the kernel in place
        a.field_in = alias ? alias : x0;
        a.c0 = 0; a.c1 = h->cells; a.stride = h->cells;
        e = dispatch(h, OP_INIT, a);
        if (e == cudaSuccess && alias) e = cudaStreamSynchronize(h->stream);  // x0 is free on return
        return e == cudaSuccess ? LBMS_OK : cuda_fail(h, e, "init kernel");
    }
    const uint32_t chunk = (uint32_t)(h->lay.staging_bytes / (h->n * h->es));
    const char* src = static_cast<const char*>(x0);
    for (uint32_t c0 = 0; c0 < h->cells; c0 += chunk) {
        const uint32_t c1 = c0 + chunk < h->cells ? c0 + chunk : h->cells;
        for (int s = 0; s < h->n; ++s) {
            e = cudaMemcpyAsync(h->staging + (size_t)s * chunk * h->es,
                                src + ((size_t)s * h->cells + c0) * h->es, (size_t)(c1 - c0) * h->es,
                                cudaMemcpyHostToDevice, h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpyAsync (host to device)");
        }
        a.field_in = h->staging;
        a.c0 = c0; a.c1 = c1; a.stride = chunk;
        e = dispatch(h, OP_INIT, a);
        if (e != cudaSuccess) return cuda_fail(h, e, "init kernel");
    }
    e = cudaStreamSynchronize(h->stream);  // x0 is free on return
    return e == cudaSuccess ? LBMS_OK : cuda_fail(h, e, "cudaStreamSynchronize");
}

int lbms_set_boundary(lbms_t* h, int face, const double* xi_b)
{
    if (!h) return LBMS_EINVAL;
    if (face < 0 || face > 5 || !((h->dirichlet >> face) & 1u))
        return fail(h, LBMS_EINVAL, "face %d is not a Dirichlet face", face);
    if (!xi_b) return fail(h, LBMS_EINVAL, "xi_b is NULL");
    double sum = 0.0;
    for (int s = 0; s < h->n; ++s) {
        if (!isfinite(xi_b[s]) || xi_b[s] < -1e-6 || xi_b[s] > 1.0 + 1e-6)
            return fail(h, LBMS_EINVAL, "xi_b[%d] = %g is not a mole fraction", s, xi_b[s]);
        sum += xi_b[s];
    }
    if (fabs(sum - 1.0) > 1e-6)
        return fail(h, LBMS_EINVAL, "the composition sums to %.9g, not 1", sum);
    h->err[0] = '\0';
    // stream-ordered: steps launched before this call see the old composition
    double v64[LBMS_MAX_SPECIES];
    float v32[LBMS_MAX_SPECIES];
    for (int s = 0; s < h->S; ++s) {
        v64[s] = xi_b[s];
        v32[s] = (float)xi_b[s];
    }
    const void* src = h->dtype == LBMS_F64 ? static_cast<const void*>(v64) : static_cast<const void*>(v32);
    cudaError_t e = cudaMemcpyAsync(static_cast<char*>(h->xb) + (size_t)face * h->S * h->es, src,
                                    (size_t)h->S * h->es, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpyAsync (boundary composition)");
    // the copy reads pageable memory: wait for it before the locals go away
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
    h->xb_set |= 1u << face;
    return LBMS_OK;
}

int lbms_set_reference(lbms_t* h, const double* xi_ref)
{
    if (!h) return LBMS_EINVAL;
    if (h->relax != LBMS_RELAX_FROZEN)
        return fail(h, LBMS_EINVAL, "the handle's relaxation mode is not LBMS_RELAX_FROZEN");
    if (!xi_ref) return fail(h, LBMS_EINVAL, "xi_ref is NULL");
    double sum = 0.0;
    for (int s = 0; s < h->n; ++s) {
        if (!isfinite(xi_ref[s]) || xi_ref[s] < 0.0 || xi_ref[s] > 1.0)
            return fail(h, LBMS_EINVAL, "xi_ref[%d] = %g is not a mole fraction", s, xi_ref[s]);
        sum += xi_ref[s];
    }
    if (fabs(sum - 1.0) > 1e-6) return fail(h, LBMS_EINVAL, "xi_ref sums to %.9g, not 1", sum);
    h->err[0] = '\0';
    for (int s = 0; s < h->n; ++s) h->xref[s] = xi_ref[s];
    h->xref_set = true;
    drop_graphs(h);
    return LBMS_OK;
}

int lbms_step(lbms_t* h, long n_steps)
{
    if (!h) return LBMS_EINVAL;
    if (n_steps < 0) return fail(h, LBMS_EINVAL, "n_steps = %ld is negative", n_steps);
    if (h->dirichlet & ~h->xb_set)
        return fail(h, LBMS_EINVAL, "Dirichlet face mask 0x%x has no composition set",
                    h->dirichlet & ~h->xb_set);
    if (h->relax == LBMS_RELAX_FROZEN && !h->xref_set)
        return fail(h, LBMS_EINVAL, "LBMS_RELAX_FROZEN needs lbms_set_reference first");
    if (h->halo && n_steps > 1)
        return fail(h, LBMS_EINVAL,
                    "a slab with LBMS_HALO faces takes one step per call (its halos are exchanged "
                    "between steps); use lbms_slab_step for several");
    h->err[0] = '\0';
    if (n_steps == 0) return LBMS_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(h->stream, &cs);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamIsCapturing");
    const bool use_graphs = h->graphs_ok && cs == cudaStreamCaptureStatusNone;
    if (use_graphs && n_steps >= 2 && n_steps <= kCallGraphMax) {
        cudaGraphExec_t g = call_graph_for(h, n_steps);
        if (g) {
            e = cudaGraphLaunch(g, h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphLaunch");
            if (n_steps & 1) h->cur = 1 - h->cur;
            h->steps += n_steps;
            h->partials_valid = true;
            h->mass_valid = false;
            return LBMS_OK;
        }
    }
    long left = n_steps;  // the last step also writes the mass partials
    for (int j = 0; use_graphs && j < 5; ++j) {
        while (left - 1 >= kGraphLens[j] && use_graphs) {
            if (!h->graph[h->cur][j]) {
                e = build_graph(h, h->cur, j);
                if (e != cudaSuccess) {
                    // fall back to direct launches for this handle
                    cudaGetLastError();
                    h->graphs_ok = false;
                    break;
                }
            }
            e = cudaGraphLaunch(h->graph[h->cur][j], h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphLaunch");
            left -= kGraphLens[j];
            h->steps += kGraphLens[j];
        }
        if (!h->graphs_ok) break;
    }
    while (left > 1) {
        e = launch_step(h, h->cur, false, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "step kernel");
        h->cur = 1 - h->cur;
        --left;
        ++h->steps;
    }
    e = launch_step(h, h->cur, true, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "step kernel");
    h->cur = 1 - h->cur;
    ++h->steps;
    // the partials are reduced when the masses are asked for (lbms_mass)
    h->partials_valid = true;
    h->mass_valid = false;
    return LBMS_OK;
}

namespace {

// Mole fractions, fluxes and local gradients at the current time, each optional
// (null: not written); device outputs in one launch, host outputs through the
// staging area in chunks.
int moments_impl(lbms_t* h, void* x_sigma, void* J_sigma, void* G_sigma)
{
    h->err[0] = '\0';
    KArgs a = base_args(h, h->stream);
    a.fin = h->steps > 0 ? h->f[1 - h->cur] : nullptr;
    a.fout = h->f[h->cur];
    a.halo_recv[0] = h->halo_recv[1 - h->cur][0];
    a.halo_recv[1] = h->halo_recv[1 - h->cur][1];
    // each output: device memory, pinned host memory written by the kernel in
    // place, or pageable host memory (through the staging area)
    void* outs_in[3] = {x_sigma, J_sigma, G_sigma};
    void* direct[3] = {nullptr, nullptr, nullptr};
    bool all_direct = true, any_pinned = false;
    for (int o = 0; o < 3; ++o) {
        if (!outs_in[o]) continue;
        void* alias = pinned_alias(outs_in[o]);
        if (alias) {
            direct[o] = alias;
            any_pinned = true;
        } else if (is_device_ptr(outs_in[o])) {
            direct[o] = outs_in[o];
        } else {
            all_direct = false;
        }
    }
    cudaError_t e;
    if (all_direct) {
        a.field_x = direct[0];
        a.field_J = direct[1];
        a.field_G = direct[2];
        a.c0 = 0; a.c1 = h->cells; a.stride = h->cells;
        e = dispatch(h, OP_MOMENTS, a);
        if (e == cudaSuccess && any_pinned) e = cudaStreamSynchronize(h->stream);  // host outputs complete
        return e == cudaSuccess ? LBMS_OK : cuda_fail(h, e, "moments kernel");
    }
    // component planes in the staging chunk: x (n), J (n * dim), G (n * dim)
    const int nx = x_sigma ? h->n : 0, nj = J_sigma ? h->n * h->dim : 0, ng = G_sigma ? h->n * h->dim : 0;
    const uint32_t chunk = (uint32_t)(h->lay.staging_bytes / ((nx + nj + ng) * h->es));
    char* outs[3] = {static_cast<char*>(x_sigma), static_cast<char*>(J_sigma), static_cast<char*>(G_sigma)};
    const int planes[3] = {nx, nj, ng};
    for (uint32_t c0 = 0; c0 < h->cells; c0 += chunk) {
        const uint32_t c1 = c0 + chunk < h->cells ? c0 + chunk : h->cells;
        a.field_x = x_sigma ? h->staging : nullptr;
        a.field_J = J_sigma ? h->staging + (size_t)nx * chunk * h->es : nullptr;
        a.field_G = G_sigma ? h->staging + (size_t)(nx + nj) * chunk * h->es : nullptr;
        a.c0 = c0; a.c1 = c1; a.stride = chunk;
        e = dispatch(h, OP_MOMENTS, a);
        if (e != cudaSuccess) return cuda_fail(h, e, "moments kernel");
        const size_t len = (size_t)(c1 - c0) * h->es;
        int base = 0;
        for (int o = 0; o < 3; ++o) {
            for (int q = 0; outs[o] && q < planes[o]; ++q) {
                e = cudaMemcpyAsync(outs[o] + ((size_t)q * h->cells + c0) * h->es,
                                    h->staging + ((size_t)(base + q) * chunk) * h->es, len,
                                    cudaMemcpyDefault, h->stream);
                if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpyAsync (moments)");
            }
            base += planes[o];
        }
    }
    e = cudaStreamSynchronize(h->stream);
    return e == cudaSuccess ? LBMS_OK : cuda_fail(h, e, "cudaStreamSynchronize");
}

}  // namespace

int lbms_moments(lbms_t* h, void* x_sigma, void* J_sigma)
{
    if (!h) return LBMS_EINVAL;
    if (!x_sigma) return fail(h, LBMS_EINVAL, "x_sigma is NULL");
    return moments_impl(h, x_sigma, J_sigma, nullptr);
}

int lbms_gradient(lbms_t* h, void* grad_sigma)
{
    if (!h) return LBMS_EINVAL;
    if (!grad_sigma) return fail(h, LBMS_EINVAL, "grad_sigma is NULL");
    return moments_impl(h, nullptr, nullptr, grad_sigma);
}

int lbms_mass(lbms_t* h, double* mass_out)
{
    if (!h) return LBMS_EINVAL;
    if (!mass_out) return fail(h, LBMS_EINVAL, "mass_out is NULL");
    h->err[0] = '\0';
    cudaError_t e;
    if (!h->partials_valid) {
        KArgs a = base_args(h, h->stream);
        a.fout = h->f[h->cur];
        a.partials = h->partials;
        e = dispatch(h, OP_MASS, a);
        if (e != cudaSuccess) return cuda_fail(h, e, "mass kernel");
        h->partials_valid = true;
        h->mass_valid = false;
    }
    if (!h->mass_valid) {
        e = launch_finalize(h, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "mass finalize kernel");
        h->mass_valid = true;
    }
    e = cudaMemcpyAsync(mass_out, h->mass_dev, sizeof(double) * h->n, cudaMemcpyDeviceToHost,
                        h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpyAsync (mass)");
    e = cudaStreamSynchronize(h->stream);
    return e == cudaSuccess ? LBMS_OK : cuda_fail(h, e, "cudaStreamSynchronize");
}

int lbms_status(lbms_t* h, uint32_t* flags)
{
    if (!h) return LBMS_EINVAL;
    if (!flags) return fail(h, LBMS_EINVAL, "flags is NULL");
    cudaError_t e = cudaMemcpyAsync(flags, h->status, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                    h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpyAsync (status)");
    e = cudaStreamSynchronize(h->stream);
    return e == cudaSuccess ? LBMS_OK : cuda_fail(h, e, "cudaStreamSynchronize");
}

int lbms_get_state(lbms_t* h, void* f_out)
{
    if (!h) return LBMS_EINVAL;
    if (!f_out) return fail(h, LBMS_EINVAL, "f_out is NULL");
    const size_t bytes = (size_t)h->S * h->Q * h->cells * h->es;
    cudaError_t e = cudaMemcpyAsync(f_out, h->f[h->cur], bytes, cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess && !is_device_ptr(f_out)) e = cudaStreamSynchronize(h->stream);
    return e == cudaSuccess ? LBMS_OK : cuda_fail(h, e, "cudaMemcpyAsync (state)");
}

int lbms_set_state_raw(lbms_t* h, const void* f_in, long step)
{
    if (!h) return LBMS_EINVAL;
    if (h->halo) return fail(h, LBMS_EINVAL, "a slab with LBMS_HALO faces is initialised by lbms_set_state only");
    if (!f_in) return fail(h, LBMS_EINVAL, "f_in is NULL");
    if (step < 0) return fail(h, LBMS_EINVAL, "step = %ld is negative", step);
    const size_t bytes = (size_t)h->S * h->Q * h->cells * h->es;
    cudaError_t e = cudaMemcpyAsync(h->f[0], f_in, bytes, cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess) {
        k_set_word<<<1, 1, 0, h->stream>>>(h->clock, (uint32_t)step);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && !is_device_ptr(f_in)) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "raw state upload");
    h->cur = 0;
    h->steps = step;
    h->partials_valid = false;
    h->mass_valid = false;
    return LBMS_OK;
}

int lbms_recompute(lbms_t* h, const void* f_in, long step, int count, void* f_out)
{
    if (!h) return LBMS_EINVAL;
    if (h->halo) return fail(h, LBMS_EINVAL, "lbms_recompute does not take LBMS_HALO faces");
    if (!f_in || !f_out) return fail(h, LBMS_EINVAL, "f_in and f_out must not be NULL");
    if (step < 0 || count < 0) return fail(h, LBMS_EINVAL, "step and count must not be negative");
    if (!is_device_ptr(f_in) || !is_device_ptr(f_out))
        return fail(h, LBMS_EINVAL, "f_in and f_out must be device memory");
    if (h->dirichlet & ~h->xb_set)
        return fail(h, LBMS_EINVAL, "Dirichlet face mask 0x%x has no composition set",
                    h->dirichlet & ~h->xb_set);
    if (h->relax == LBMS_RELAX_FROZEN && !h->xref_set)
        return fail(h, LBMS_EINVAL, "LBMS_RELAX_FROZEN needs lbms_set_reference first");
    h->err[0] = '\0';
    if (count == 0) return LBMS_OK;
    const size_t elems = (size_t)h->S * h->Q * h->cells;
    // the two step-counter words carry step, step + 1, ... through the launches
    k_set_word<<<1, 1, 0, h->stream>>>(h->clock, (uint32_t)step);
    cudaError_t e = cudaGetLastError();
    const char* src = static_cast<const char*>(f_in);
    for (int j = 0; j < count && e == cudaSuccess; ++j) {
        KArgs a = base_args(h, h->stream);
        a.fin = src;
        a.fout = static_cast<char*>(f_out) + (size_t)j * elems * h->es;
        a.partials = h->partials;
        a.clock_in = h->clock + (j & 1);
        a.clock_out = h->clock + 1 - (j & 1);
        e = dispatch(h, OP_STEP, a);
        src = static_cast<const char*>(a.fout);
    }
    // give the handle's own step counter back to its state
    if (e == cudaSuccess) {
        k_set_word<<<1, 1, 0, h->stream>>>(h->clock + h->cur, (uint32_t)h->steps);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? LBMS_OK : cuda_fail(h, e, "recompute");
}

size_t lbms_adjoint_scratch_size(const lbms_t* h)
{
    if (!h || h->halo || h->S > 4 || h->relax == LBMS_RELAX_FROZEN) return 0;
    return (size_t)node_blocks(h->cells) * (kBlock / 32) * (h->n * (h->n - 1) / 2) * sizeof(double);
}

int lbms_adjoint_seed(lbms_t* h, const void* grad_x, void* lam)
{
    if (!h) return LBMS_EINVAL;
    if (h->halo) return fail(h, LBMS_EINVAL, "the adjoint does not take LBMS_HALO faces");
    if (h->S > 4) return fail(h, LBMS_EINVAL, "the adjoint supports up to 5 species");
    if (h->relax == LBMS_RELAX_FROZEN) return fail(h, LBMS_EINVAL, "the adjoint does not take LBMS_RELAX_FROZEN");
    if (!grad_x || !lam) return fail(h, LBMS_EINVAL, "grad_x and lam must not be NULL");
    if (!is_device_ptr(grad_x) || !is_device_ptr(lam))
        return fail(h, LBMS_EINVAL, "grad_x and lam must be device memory");
    AArgs a;
    a.k = base_args(h, h->stream);
    a.grad_x = grad_x;
    a.lam = lam;
    cudaError_t e = adj_dispatch(h, AOP_SEED, a);
    return e == cudaSuccess ? LBMS_OK : cuda_fail(h, e, "adjoint seed kernel");
}

int lbms_adjoint_step(lbms_t* h, const void* f_prev, const void* lam_in, void* lam_out, void* gacc)
{
    if (!h) return LBMS_EINVAL;
    if (h->halo) return fail(h, LBMS_EINVAL, "the adjoint does not take LBMS_HALO faces");
    if (h->S > 4) return fail(h, LBMS_EINVAL, "the adjoint supports up to 5 species");
    if (h->relax == LBMS_RELAX_FROZEN) return fail(h, LBMS_EINVAL, "the adjoint does not take LBMS_RELAX_FROZEN");
    if (!f_prev || !lam_in || !lam_out || !gacc)
        return fail(h, LBMS_EINVAL, "f_prev, lam_in, lam_out and gacc must not be NULL");
    if (lam_in == lam_out) return fail(h, LBMS_EINVAL, "lam_in and lam_out must be different buffers");
    if (!is_device_ptr(f_prev) || !is_device_ptr(lam_in) || !is_device_ptr(lam_out) || !is_device_ptr(gacc))
        return fail(h, LBMS_EINVAL, "f_prev, lam_in, lam_out and gacc must be device memory");
    AArgs a;
    a.k = base_args(h, h->stream);
    a.fprev = f_prev;
    a.lam_in = lam_in;
    a.lam_out = lam_out;
    a.gacc = static_cast<double*>(gacc);
    cudaError_t e = adj_dispatch(h, AOP_STEP, a);
    return e == cudaSuccess ? LBMS_OK : cuda_fail(h, e, "adjoint step kernel");
}

int lbms_adjoint_steps(lbms_t* h, const void* f_first, const void* f_rest, int count, void* lam_a, void* lam_b,
                       void* gacc)
{
    if (!h) return LBMS_EINVAL;
    if (h->halo) return fail(h, LBMS_EINVAL, "the adjoint does not take LBMS_HALO faces");
    if (h->S > 4) return fail(h, LBMS_EINVAL, "the adjoint supports up to 5 species");
    if (h->relax == LBMS_RELAX_FROZEN) return fail(h, LBMS_EINVAL, "the adjoint does not take LBMS_RELAX_FROZEN");
    if (count < 0) return fail(h, LBMS_EINVAL, "count = %d is negative", count);
    if (!f_first || !lam_a || !lam_b || !gacc || (count > 1 && !f_rest))
        return fail(h, LBMS_EINVAL, "f_first, f_rest (count > 1), lam_a, lam_b and gacc must not be NULL");
    if (lam_a == lam_b) return fail(h, LBMS_EINVAL, "lam_a and lam_b must be different buffers");
    if (!is_device_ptr(f_first) || (count > 1 && !is_device_ptr(f_rest)) || !is_device_ptr(lam_a) ||
        !is_device_ptr(lam_b) || !is_device_ptr(gacc))
        return fail(h, LBMS_EINVAL, "f_first, f_rest, lam_a, lam_b and gacc must be device memory");
    h->err[0] = '\0';
    const size_t fbytes = (size_t)h->S * h->Q * h->cells * h->es;
    AArgs a;
    a.k = base_args(h, h->stream);
    a.gacc = static_cast<double*>(gacc);
    // step t0 + count - i (i = 0 .. count - 1) reads f+(t0 + count - i - 1)
    for (int i = 0; i < count; ++i) {
        const int j = count - 1 - i;  // f+(t0 + j)
        a.fprev = j == 0 ? f_first : static_cast<const char*>(f_rest) + (size_t)(j - 1) * fbytes;
        a.lam_in = (i & 1) ? lam_b : lam_a;
        a.lam_out = (i & 1) ? lam_a : lam_b;
        cudaError_t e = adj_dispatch(h, AOP_STEP, a);
        if (e != cudaSuccess) return cuda_fail(h, e, "adjoint step kernel");
    }
    return LBMS_OK;
}

int lbms_adjoint_initial(lbms_t* h, const void* lam0, void* grad_x0)
{
    if (!h) return LBMS_EINVAL;
    if (h->halo) return fail(h, LBMS_EINVAL, "the adjoint does not take LBMS_HALO faces");
    if (h->S > 4) return fail(h, LBMS_EINVAL, "the adjoint supports up to 5 species");
    if (h->relax == LBMS_RELAX_FROZEN) return fail(h, LBMS_EINVAL, "the adjoint does not take LBMS_RELAX_FROZEN");
    if (!lam0 || !grad_x0) return fail(h, LBMS_EINVAL, "lam0 and grad_x0 must not be NULL");
    if (!is_device_ptr(lam0) || !is_device_ptr(grad_x0))
        return fail(h, LBMS_EINVAL, "lam0 and grad_x0 must be device memory");
    AArgs a;
    a.k = base_args(h, h->stream);
    a.lam = const_cast<void*>(lam0);
    a.grad_x0 = grad_x0;
    cudaError_t e = adj_dispatch(h, AOP_INITIAL, a);
    return e == cudaSuccess ? LBMS_OK : cuda_fail(h, e, "adjoint initial kernel");
}

int lbms_adjoint_reduce(lbms_t* h, const void* gacc, double* dL_dD)
{
    if (!h) return LBMS_EINVAL;
    if (h->halo) return fail(h, LBMS_EINVAL, "the adjoint does not take LBMS_HALO faces");
    if (h->S > 4) return fail(h, LBMS_EINVAL, "the adjoint supports up to 5 species");
    if (h->relax == LBMS_RELAX_FROZEN) return fail(h, LBMS_EINVAL, "the adjoint does not take LBMS_RELAX_FROZEN");
    if (!gacc || !dL_dD) return fail(h, LBMS_EINVAL, "gacc and dL_dD must not be NULL");
    if (!is_device_ptr(gacc)) return fail(h, LBMS_EINVAL, "gacc must be device memory");
    const int np = h->n * (h->n - 1) / 2;
    double* slot = reinterpret_cast<double*>(reinterpret_cast<char*>(h->status) + 128);
    double invD2[16];
    int k = 0;
    for (int p = 0; p < h->n; ++p)
        for (int q = p + 1; q < h->n; ++q, ++k) invD2[k] = h->invD[p][q] * h->invD[p][q];
    GradScale gs;
    for (int i = 0; i < np; ++i) gs.v[i] = invD2[i];
    k_adjoint_reduce<<<np, kBlock, 0, h->stream>>>(static_cast<const double*>(gacc), node_blocks(h->cells) * (kBlock / 32),
                                                   np, h->dtype == LBMS_F32 ? 1 : 0, gs, slot);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dL_dD, slot, sizeof(double) * np, cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return e == cudaSuccess ? LBMS_OK : cuda_fail(h, e, "adjoint reduction");
}

long lbms_steps_done(const lbms_t* h) { return h ? h->steps : -1; }

const void* lbms_populations(const lbms_t* h) { return h ? h->f[h->cur] : nullptr; }

int lbms_set_subdomain(lbms_t* h, long first_layer)
{
    if (!h) return LBMS_EINVAL;
    if (first_layer < 0) return fail(h, LBMS_EINVAL, "first_layer = %ld is negative", first_layer);
    h->err[0] = '\0';
    // node indices of the undivided grid (modulo 2^32, as the rounding key takes them)
    h->origin = (uint32_t)((uint64_t)first_layer * h->plane);
    drop_graphs(h);
    return LBMS_OK;
}

int lbms_halo_buffers(lbms_t* h, int face, void** send, void** recv, size_t* bytes)
{
    if (!h) return LBMS_EINVAL;
    if (face < 0 || face > 5 || !((h->halo >> face) & 1u))
        return fail(h, LBMS_EINVAL, "face %d is not an LBMS_HALO face", face);
    h->err[0] = '\0';
    const int side = face & 1;
    if (send) *send = h->halo_send[side];
    if (recv) *recv = h->halo_recv[h->cur][side];
    if (bytes) *bytes = (size_t)lattice_halo_width(h->lattice) * h->S * h->plane * h->es;
    return LBMS_OK;
}

int lbms_slab_step(lbms_t* const* subs, int count, long n_steps)
{
    if (!subs || count < 1) return set_call_error(LBMS_EINVAL, "subs is NULL or count < 1");
    for (int i = 0; i < count; ++i)
        if (!subs[i]) return set_call_error(LBMS_EINVAL, "subs[%d] is NULL", i);
    lbms_t* h0 = subs[0];
    if (n_steps < 0) return fail(h0, LBMS_EINVAL, "n_steps = %ld is negative", n_steps);
    const uint32_t lo_bit = 1u << (2 * (h0->dim - 1)), hi_bit = lo_bit << 1;
    for (int i = 0; i < count; ++i) {
        const lbms_t* h = subs[i];
        // the extents across the split axis (the layer shape) must agree
        if (h->lattice != h0->lattice || h->n != h0->n || h->dtype != h0->dtype || h->plane != h0->plane ||
            (h0->dim >= 2 && h->nx != h0->nx) || (h0->dim == 3 && h->ny != h0->ny))
            return fail(h0, LBMS_EINVAL, "slab %d differs in lattice, species, dtype or layer shape", i);
        if (h->stream != h0->stream) return fail(h0, LBMS_EINVAL, "slab %d is on another stream", i);
        if (h->steps != h0->steps) return fail(h0, LBMS_EINVAL, "slab %d is at another step", i);
        if (h->dirichlet & ~h->xb_set)
            return fail(h0, LBMS_EINVAL, "slab %d: a Dirichlet face has no composition set", i);
        if (h->relax == LBMS_RELAX_FROZEN && !h->xref_set)
            return fail(h0, LBMS_EINVAL, "slab %d: LBMS_RELAX_FROZEN needs lbms_set_reference first", i);
        // a cut is a pair of LBMS_HALO faces: this slab's high face and the next
        // slab's low face (the last slab's high face pairs with the first's low
        // face when the split axis wraps)
        const lbms_t* up = subs[(i + 1) % count];
        if (((h->halo & hi_bit) != 0) != ((up->halo & lo_bit) != 0))
            return fail(h0, LBMS_EINVAL, "the faces between slab %d and slab %d are not a pair of cuts", i,
                        (i + 1) % count);
    }
    h0->err[0] = '\0';
    const size_t hb = (size_t)lattice_halo_width(h0->lattice) * h0->S * h0->plane * h0->es;
    cudaStream_t st = h0->stream;
    for (long t = 0; t < n_steps; ++t) {
        // halo exchange: every slab's receive buffers of its current parity get
        // the neighbours' populations that cross the cuts
        for (int i = 0; i < count; ++i) {
            lbms_t* h = subs[i];
            cudaError_t e = cudaSuccess;
            if (h->halo & hi_bit) {
                lbms_t* up = subs[(i + 1) % count];
                e = cudaMemcpyAsync(up->halo_recv[up->cur][0], h->halo_send[1], hb, cudaMemcpyDeviceToDevice, st);
            }
            if (e == cudaSuccess && (h->halo & lo_bit)) {
                lbms_t* dn = subs[(i + count - 1) % count];
                e = cudaMemcpyAsync(dn->halo_recv[dn->cur][1], h->halo_send[0], hb, cudaMemcpyDeviceToDevice, st);
            }
            if (e != cudaSuccess) return cuda_fail(h0, e, "halo exchange");
        }
        const bool last = t + 1 == n_steps;
        for (int i = 0; i < count; ++i) {
            lbms_t* h = subs[i];
            cudaError_t e = launch_step(h, h->cur, last, st);
            if (e != cudaSuccess) return cuda_fail(h0, e, "step kernel");
            h->cur = 1 - h->cur;
            ++h->steps;
            if (last) {
                h->partials_valid = true;
                h->mass_valid = false;
            }
        }
    }
    return LBMS_OK;
}

const char* lbms_last_error(const lbms_t* h) { return h ? h->err : g_create_error; }

void lbms_destroy(lbms_t* h)
{
    if (!h) return;
    drop_graphs(h);
    if (h->capture) cudaStreamDestroy(h->capture);
    delete h;
}

}  // extern "C"
