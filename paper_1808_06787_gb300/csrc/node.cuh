// Per-node arithmetic of the Maxwell-Stefan MRT model, in registers.
//
// Relaxation matrices.  With D~ = B^{-1} (Eq. 2-11) and the Chapman-Enskog
// relation D~ = c_s^2 (Lambda_1^{-1} - I/2) (Eq. 3-26),
//     Lambda_1 = (B^{-1}/c_s^2 + I/2)^{-1} = K^{-1} B,   K = I/c_s^2 + B/2,
// so one Gauss-Jordan elimination of [K | B] gives Lambda_1 without forming
// B^{-1} (B need not even be invertible); for ternary mixtures the 2 x 2 form
// adj(K) B / det(K) does it with a single reciprocal.  The elimination runs without
// pivoting: B has real non-negative eigenvalues (it is the reduced form of the
// Maxwell-Stefan friction matrix, which is diagonally similar to a symmetric
// positive semi-definite one), and every pivot of K has been found to be at
// least 1/c_s^2 for compositions with vanishing species and diffusivities
// spread over four decades; the test-suite checks that property.
// Lambda_2 follows Eq. 3-16, or equals Lambda_1 for SRT.
//
// Half matrices.  The step kernels carry Lambda_1/2 and Lambda_2/2: they take
// the inverse diffusivities halved, 1/(2 D_ij), so Eq. 2-10 (linear in them)
// yields B/2 directly, K = I/c_s^2 + B/2 needs no scaling, K^{-1} (B/2) is
// Lambda_1/2, and Eq. 3-16 rewritten for l/2 gives Lambda_2/2.  Scaling by a
// power of two is exact, so these are the halves of the unscaled matrices bit
// for bit; the halves of the pair form below fold into them.
//
// Collision.  For moment bases whose rows are the total mass, odd-order rows
// (relaxed by Lambda_1) and even-order rows (relaxed by Lambda_2), the
// moment-space collision of Eq. 3-13a equals the pair form used here: for each
// opposite pair (k, kbar) with g = f - w xi,
//     s = (g_k + g_kbar)/2,  a = (g_k - g_kbar)/2,
//     f+_k = f_k - Lambda_2 s - Lambda_1 a,  f+_kbar = f_k - Lambda_2 s + Lambda_1 a,
// evaluated as (Lambda_2/2)(g_k + g_kbar) and (Lambda_1/2)(g_k - g_kbar),
// and for the rest population f+_0 = f_0 - Lambda_2 g_0.  Sec. 3.1 notes that
// odd/even relaxation groups make the MRT model a two-relaxation-time model.
//
// Conservation in finite precision.  The conserved moment has m - m_eq = 0, so
// in exact arithmetic the collision keeps sum_k f_k of every species at every
// node, which is what makes f+_0 = f_0 - Lambda_2 g_0 equal to
//     f+_0 = f_0 + sum_{k != 0} (f_k - f+_k).
// The kernels use this second form, with the moving populations' increments
// summed first and added to f_0 by an error-free two-sum, so the node's mass is
// carried over exactly up to the single final rounding of f+_0.  In FP32 that
// rounding is stochastic: the two-sum remainder decides whether to round up or
// down, against a uniform number hashed from the node, the species and the
// step count, which makes the residual zero-mean and uncorrelated between
// nodes and between steps.  Round-to-nearest residuals are not: identical
// nodes (a field uniform along an axis) and slowly varying states repeat the
// same residual, and with weights such as 1/9 or 1/36 that do not sum to one in
// FP32 the plain form loses mass at every node every step.  (A hash of the
// state's own bits is not enough either: where the state changes below FP32
// resolution for many steps, the same decision repeats.)  Results stay
// deterministic: the step count is a device counter advanced by every step.
#pragma once

#include "lattice.cuh"

namespace lbms {

// Reciprocal used by the per-node solve: the fast hardware approximation in
// FP32 (well inside the FP32 tolerance), the IEEE division in FP64.
__device__ __forceinline__ float recip(float v) { return __fdividef(1.0f, v); }
__device__ __forceinline__ double recip(double v) { return 1.0 / v; }

// Lambda_1/2 = K^{-1} (B/2) and Lambda_2/2 (Eq. 3-16, or = Lambda_1/2 for SRT) from
// all S+1 mole fractions and the halved inverse diffusivities invDh[i][j] =
// 1/(2 D_ij).
template <int S, typename T, typename InvD>
__device__ __forceinline__ void relaxation_matrices(const T (&xi)[S + 1], const InvD& invDh,
                                                    T cs2inv, int relax, T (&L1)[S][S],
                                                    T (&L2)[S][S])
{
    T K[S][S];
#pragma unroll
    for (int i = 0; i < S; ++i) {
#pragma unroll
        for (int j = 0; j < S; ++j) {
            T b;  // B/2
            if (i != j) {
                b = xi[i] * (invDh[i][S] - invDh[i][j]);  // Eq. 2-10, i != j
            } else {
                b = xi[i] * invDh[i][S];  // Eq. 2-10, i == j
#pragma unroll
                for (int k = 0; k <= S; ++k)
                    if (k != i) b += xi[k] * invDh[i][k];
            }
            L1[i][j] = b;
            K[i][j] = i == j ? b + cs2inv : b;
        }
    }
    if constexpr (S == 2) {
        // ternary mixtures (Remark IV): Lambda_1/2 = adj(K) (B/2) / det(K) = N / d;
        // d = det(K) > 0 because B's eigenvalues are real and non-negative.  With
        // h = N_ii / d, Eq. 3-16 for l = 2h reads lambda_2/2 = 4 (N_ii - d) /
        // (N_ii - 4 d), so one reciprocal of d (N_00 - 4d) (N_11 - 4d) gives 1/d
        // and both diagonal entries of Lambda_2/2 (N_ii - 4d < 0 for l < 8).
        const T d = K[0][0] * K[1][1] - K[0][1] * K[1][0];
        const T b00 = L1[0][0], b01 = L1[0][1], b10 = L1[1][0], b11 = L1[1][1];
        const T n00 = K[1][1] * b00 - K[0][1] * b10;
        const T n01 = K[1][1] * b01 - K[0][1] * b11;
        const T n10 = K[0][0] * b10 - K[1][0] * b00;
        const T n11 = K[0][0] * b11 - K[1][0] * b01;
        T rdet;
        if (relax != LBMS_RELAX_SRT) {  // Eq. 3-16 (the frozen mode uses it too)
            const T p0 = n00 - T(4) * d, p1 = n11 - T(4) * d;
            const T pp = p0 * p1;
            const T inv = recip(d * pp);
            rdet = inv * pp;
            const T q = inv * d;
            L2[0][0] = T(4) * (n00 - d) * (q * p1);
            L2[1][1] = T(4) * (n11 - d) * (q * p0);
        } else {
            rdet = recip(d);
        }
        L1[0][0] = n00 * rdet;
        L1[0][1] = n01 * rdet;
        L1[1][0] = n10 * rdet;
        L1[1][1] = n11 * rdet;
        L2[0][1] = L1[0][1];
        L2[1][0] = L1[1][0];
        if (relax == LBMS_RELAX_SRT) {
            L2[0][0] = L1[0][0];
            L2[1][1] = L1[1][1];
        }
        return;
    } else {
#pragma unroll
        for (int p = 0; p < S; ++p) {
            const T inv = recip(K[p][p]);
#pragma unroll
            for (int j = 0; j < S; ++j) {
                K[p][j] *= inv;
                L1[p][j] *= inv;
            }
#pragma unroll
            for (int r = 0; r < S; ++r) {
                if (r == p) continue;
                const T fac = K[r][p];
#pragma unroll
                for (int j = 0; j < S; ++j) {
                    K[r][j] -= fac * K[p][j];
                    L1[r][j] -= fac * L1[p][j];
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < S; ++i)
#pragma unroll
        for (int j = 0; j < S; ++j) L2[i][j] = L1[i][j];
    if (relax != LBMS_RELAX_SRT) {  // Eq. 3-16 (the frozen mode uses it too)
        // Eq. 3-16 with l = 2 h: lambda_2/2 = 4 (h - 1) / (h - 4)
#pragma unroll
        for (int i = 0; i < S; ++i) {
            const T h = L1[i][i];
            L2[i][i] = T(4) * (h - T(1)) * recip(h - T(4));  // Eq. 3-16, i == j
        }
    }
}

// xi_i = sum_k f_k^i (Eq. 3-15) and xi_n = 1 - sum (Eq. 2-3b).
template <int LAT, int S, typename T>
__device__ __forceinline__ void mole_fractions(const T (&f)[S][Lattice<LAT>::Q], T (&xi)[S + 1])
{
    constexpr int Q = Lattice<LAT>::Q;
    T sum = T(0);
#pragma unroll
    for (int s = 0; s < S; ++s) {
        T x = f[s][0];
#pragma unroll
        for (int k = 1; k < Q; ++k) x += f[s][k];
        xi[s] = x;
        sum += x;
    }
    xi[S] = T(1) - sum;
}

// Final rounding of the rest population from the exact value hi + lo.
__device__ __forceinline__ uint32_t mix32(uint32_t h)
{
    // finaliser of MurmurHash3 (Appleby): avalanche of a 32-bit key
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

// `h` is a uniformly distributed 32-bit number.
__device__ __forceinline__ float round_rest(float hi, float lo, uint32_t h)
{
    // hi = RN(hi + lo) and |lo| <= half the gap to the neighbour on lo's side;
    // moving to that neighbour with probability |lo| / gap is unbiased.
    // (lo != 0 implies hi != 0; the neighbour of a finite non-zero float on the
    // side of lo is one step of its bit pattern away from or toward zero)
    const float u = (float)(h >> 8) * 0x1p-24f;
    const int step = ((lo > 0.0f) == (hi > 0.0f)) ? 1 : -1;
    const float nb = __int_as_float(__float_as_int(hi) + step);
    return (lo != 0.0f && fabsf(lo) > u * fabsf(nb - hi)) ? nb : hi;
}

__device__ __forceinline__ double round_rest(double hi, double, uint32_t) { return hi; }

// Error-free sum a + b = s + e (Knuth's two-sum).
template <typename T>
__device__ __forceinline__ void two_sum(T a, T b, T& s, T& e)
{
    s = a + b;
    const T bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}

// In-place collision in the pair form (see the header comment) with the half
// matrices L1h = Lambda_1/2, L2h = Lambda_2/2; `key` (distinct per node and
// step) seeds the stochastic rounding of the rest population (FP32 only).
template <int LAT, int S, typename T>
__device__ __forceinline__ void collide(T (&f)[S][Lattice<LAT>::Q], const T (&xi)[S + 1],
                                        const T (&L1h)[S][S], const T (&L2h)[S][S], uint32_t key)
{
    using L = Lattice<LAT>;
    // sum of the moving populations' increments f_k - f+_k (each exact: f+_k is
    // within a factor two of f_k); its rounding is far below an ulp of f_0
    T moved[S];
#pragma unroll
    for (int i = 0; i < S; ++i) moved[i] = T(0);
#pragma unroll
    for (int pr = 0; pr < L::NPAIR; ++pr) {
        const int ka = L::K0 + 2 * pr, kb = ka + 1;
        const T wp2 = T(2.0 * L::w(ka));
        T sym[S], asym[S];  // g_k + g_kbar and g_k - g_kbar
#pragma unroll
        for (int j = 0; j < S; ++j) {
            sym[j] = (f[j][ka] + f[j][kb]) - wp2 * xi[j];
            asym[j] = f[j][ka] - f[j][kb];
        }
#pragma unroll
        for (int i = 0; i < S; ++i) {
            T ds = T(0), da = T(0);
#pragma unroll
            for (int j = 0; j < S; ++j) {
                ds += L2h[i][j] * sym[j];
                da += L1h[i][j] * asym[j];
            }
            const T na = f[i][ka] - (ds + da);
            const T nb = f[i][kb] - (ds - da);
            if (ka == 0) {
                // no rest velocity: population 0 is the absorber below
                moved[i] += f[i][kb] - nb;
            } else {
                moved[i] += (f[i][ka] - na) + (f[i][kb] - nb);
                f[i][ka] = na;
            }
            f[i][kb] = nb;
        }
    }
    // population 0 (the rest population; on lattices without one, the first
    // moving population): f+_0 = f_0 + sum_{k != 0} (f_k - f+_k); one hash per
    // node, and per species an odd multiple of it offset by a species constant
    // (a bijection of a uniform 32-bit number, so again uniform)
    const uint32_t hn = mix32(key);
#pragma unroll
    for (int i = 0; i < S; ++i) {
        T hi, lo;
        two_sum(f[i][0], moved[i], hi, lo);
        f[i][0] = round_rest(hi, lo, (hn ^ (0x9e3779b9u * (uint32_t)(i + 1))) * 0x85ebca6bu);
    }
}

// Grid geometry shared by the node kernels.  Coordinates of a linear node
// index come from multiply-shift division by the invariant extents nx and ny
// (Granlund and Montgomery, "Division by invariant integers using
// multiplication", 1994): for n < 2^31 and d < 2^31, with s = 31 + ceil(log2 d)
// and m = ceil(2^s / d), floor(n / d) = (n * m) >> s exactly.
struct FastDiv {
    uint64_t m;
    uint32_t s;
    __device__ __forceinline__ uint32_t div(uint32_t n) const { return (uint32_t)(((uint64_t)n * m) >> s); }
};

struct Geom {
    int nx, ny, nz;
    uint32_t nxy, cells;
    uint32_t noflux;     // bit f set: face f is a wall, no-flux or Dirichlet (x-, x+, y-, y+, z-, z+)
    uint32_t dirichlet;  // bit f set: wall face f holds a fixed composition
    uint32_t halo;       // bit f set: face f is a cut of a slab decomposition (faces of the split axis)
    uint32_t plane;      // nodes per layer of the split axis (nxy in 3D, nx in 2D, 1 in 1D)
    uint32_t origin;     // global index of node 0 (a slab's offset in the undivided grid)
    FastDiv dnx, dny;
};

// Source offsets (in nodes) of the gather along each axis for c = +1 and c = -1,
// with periodic wrap, and whether that source lies across a wall face.
struct Neighbourhood {
    int32_t ox[2], oy[2], oz[2];  // [0]: c = +1 (source at -1), [1]: c = -1 (source at +1)
    bool bx[2], by[2], bz[2];
    uint32_t dir;   // the Dirichlet faces this node lies on (bits as Geom::noflux)
    uint32_t hal;   // the cut faces this node lies on (bits as Geom::noflux)
    uint32_t inpl;  // the node's index within its layer of the split axis
};

// Receive and send buffers of the two cut faces of a slab (faces of the split
// axis): [halo_width][S][plane] each, slot j of halo_slot.  recv_lo holds the
// lower neighbour's populations that cross the cut upward, taken from its top
// layer, recv_hi the upper neighbour's downward ones from its bottom layer;
// send_hi / send_lo are this slab's own, written by every step.
template <typename T>
struct Halo {
    const T* __restrict__ recv_lo;
    const T* __restrict__ recv_hi;
    T* send_lo;
    T* send_hi;
};

// DIM is the lattice's dimension: a 2D grid has nz = 1 and a 1D grid ny = nz = 1,
// so those coordinates need no division.
template <int DIM, bool HALO = true>
__device__ __forceinline__ Neighbourhood neighbourhood(const Geom& g, uint32_t cell)
{
    uint32_t row = 0;
    int x = (int)cell, y = 0, z = 0;
    if (DIM > 1) {
        row = g.dnx.div(cell);
        x = (int)(cell - row * (uint32_t)g.nx);
        y = (int)row;
    }
    if (DIM > 2) {
        z = (int)g.dny.div(row);
        y = (int)(row - (uint32_t)z * (uint32_t)g.ny);
    }
    Neighbourhood h;
    const bool xlo = x == 0, xhi = x == g.nx - 1;
    const bool ylo = y == 0, yhi = y == g.ny - 1;
    const bool zlo = z == 0, zhi = z == g.nz - 1;
    const int32_t sx = 1, sy = g.nx, sz = (int32_t)g.nxy;
    h.ox[0] = xlo ? sx * (g.nx - 1) : -sx;
    h.ox[1] = xhi ? -sx * (g.nx - 1) : sx;
    h.oy[0] = ylo ? sy * (g.ny - 1) : -sy;
    h.oy[1] = yhi ? -sy * (g.ny - 1) : sy;
    h.oz[0] = zlo ? sz * (g.nz - 1) : -sz;
    h.oz[1] = zhi ? -sz * (g.nz - 1) : sz;
    h.bx[0] = xlo && (g.noflux & 1u);
    h.bx[1] = xhi && (g.noflux & 2u);
    h.by[0] = ylo && (g.noflux & 4u);
    h.by[1] = yhi && (g.noflux & 8u);
    h.bz[0] = zlo && (g.noflux & 16u);
    h.bz[1] = zhi && (g.noflux & 32u);
    h.dir = 0u;
    if (g.dirichlet)  // uniform over the grid
        h.dir = g.dirichlet & ((xlo ? 1u : 0u) | (xhi ? 2u : 0u) | (ylo ? 4u : 0u) |
                               (yhi ? 8u : 0u) | (zlo ? 16u : 0u) | (zhi ? 32u : 0u));
    h.hal = 0u;
    h.inpl = 0u;
    if (HALO && g.halo) {  // uniform over the grid: a slab of a decomposed grid
        // faces of the split axis that are cuts: the source across them is in a
        // neighbour's receive buffer; the offsets along that axis are set to stay
        // on the node (the gathered value is replaced)
        if (DIM == 3) {
            h.hal = g.halo & ((zlo ? 16u : 0u) | (zhi ? 32u : 0u));
            if (h.hal & 16u) h.oz[0] = 0;
            if (h.hal & 32u) h.oz[1] = 0;
            h.inpl = cell - (uint32_t)z * g.nxy;
        } else if (DIM == 2) {
            h.hal = g.halo & ((ylo ? 4u : 0u) | (yhi ? 8u : 0u));
            if (h.hal & 4u) h.oy[0] = 0;
            if (h.hal & 8u) h.oy[1] = 0;
            h.inpl = (uint32_t)x;
        } else {
            h.hal = g.halo & ((xlo ? 1u : 0u) | (xhi ? 2u : 0u));
            if (h.hal & 1u) h.ox[0] = 0;
            if (h.hal & 2u) h.ox[1] = 0;
        }
    }
    return h;
}

// Bits of the low and high cut faces of the split axis.
template <int DIM>
__host__ __device__ constexpr uint32_t halo_lo_bit() { return DIM == 3 ? 16u : (DIM == 2 ? 4u : 1u); }
template <int DIM>
__host__ __device__ constexpr uint32_t halo_hi_bit() { return DIM == 3 ? 32u : (DIM == 2 ? 8u : 2u); }

// The wall face the pull source of direction k lies across, or -1.  A D2Q9
// diagonal at a corner can cross two walls: the first in axis order x, y, z
// decides (the paper does not treat corners).
template <int LAT>
__device__ __forceinline__ int link_wall(int k, const Neighbourhood& h)
{
    using L = Lattice<LAT>;
    const int cx = L::cx(k), cy = L::cy(k), cz = L::cz(k);
    if (cx != 0 && h.bx[cx > 0 ? 0 : 1]) return cx > 0 ? 0 : 1;
    if (cy != 0 && h.by[cy > 0 ? 0 : 1]) return cy > 0 ? 2 : 3;
    if (cz != 0 && h.bz[cz > 0 ? 0 : 1]) return cz > 0 ? 4 : 5;
    return -1;
}

// Gather f_k(x, t) = f+_k(x - c_k, t-1) for every species and direction: the
// propagation of Eq. 3-13b read in the pull direction.  A source across a
// periodic face wraps; a source across a no-flux face is replaced by the node's
// own opposite population, f_k(x) = f+_kbar(x) (half-way bounce-back, Sec. 4);
// across a Dirichlet face of composition xi_b by f_k(x) = -f+_kbar(x) +
// 2 w_k xi_{s,b} (half-way anti-bounce-back, Sec. 4).  xb holds the evolved
// species' compositions of the six faces, [6][S]; it is read only on nodes
// next to a Dirichlet face.
// SKIP_REST: the caller has loaded the rest population (k = 0 of a lattice with
// a rest velocity, which never moves) itself.  SKIP_Y: the caller has loaded the
// moving populations that do not move along x (the two-nodes-per-thread kernels
// pair them); their Dirichlet correction below still applies.
template <int LAT, int S, typename T, bool SKIP_REST = false, bool SKIP_Y = false>
__device__ __forceinline__ void pull(const T* __restrict__ fin, const Geom& g, uint32_t cell,
                                     const Neighbourhood& h, T (&f)[S][Lattice<LAT>::Q],
                                     const T* __restrict__ xb, const Halo<T>* halo = nullptr)
{
    using L = Lattice<LAT>;
    constexpr int Q = L::Q;
    constexpr int DIM = L::DIM;
    static_assert(!SKIP_REST || L::K0 == 1, "only a rest population can be skipped");
#pragma unroll
    for (int k = SKIP_REST ? 1 : 0; k < Q; ++k) {
        const int cx = L::cx(k), cy = L::cy(k), cz = L::cz(k);
        if (SKIP_Y && cx == 0 && (cy != 0 || cz != 0)) continue;
        int32_t off = 0;
        bool bounce = false;
        if (cx != 0) { off += h.ox[cx > 0 ? 0 : 1]; bounce |= h.bx[cx > 0 ? 0 : 1]; }
        if (cy != 0) { off += h.oy[cy > 0 ? 0 : 1]; bounce |= h.by[cy > 0 ? 0 : 1]; }
        if (cz != 0) { off += h.oz[cz > 0 ? 0 : 1]; bounce |= h.bz[cz > 0 ? 0 : 1]; }
        const uint32_t src = bounce ? cell : (uint32_t)((int32_t)cell + off);
        const size_t plane = (size_t)(bounce ? opp<LAT>(k) : k) * g.cells;
#pragma unroll
        for (int s = 0; s < S; ++s) f[s][k] = fin[(size_t)s * Q * g.cells + plane + src];
    }
    if (halo && h.hal) {
        // slab cut: a source across a cut face (and across no wall of another
        // axis, which bounces first) is the neighbour's population in the
        // receive buffer, at the source's position within the layer
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const int c = split_c<LAT>(k);
            if (c == 0) continue;
            if (!(h.hal & (c > 0 ? halo_lo_bit<DIM>() : halo_hi_bit<DIM>()))) continue;
            const int cx = L::cx(k), cy = L::cy(k);
            bool bounce = false;
            int32_t inoff = 0;
            if (DIM >= 2 && cx != 0) { inoff += h.ox[cx > 0 ? 0 : 1]; bounce |= h.bx[cx > 0 ? 0 : 1]; }
            if (DIM == 3 && cy != 0) { inoff += h.oy[cy > 0 ? 0 : 1]; bounce |= h.by[cy > 0 ? 0 : 1]; }
            if (bounce) continue;
            const T* rb = c > 0 ? halo->recv_lo : halo->recv_hi;
            const uint32_t at = (uint32_t)((int32_t)h.inpl + inoff);
#pragma unroll
            for (int s = 0; s < S; ++s) f[s][k] = rb[((size_t)halo_slot<LAT>(k) * S + s) * g.plane + at];
        }
    }
    if (h.dir) {
#pragma unroll
        for (int k = L::K0; k < Q; ++k) {
            const int wf = link_wall<LAT>(k, h);
            if (wf >= 0 && ((h.dir >> wf) & 1u)) {
#pragma unroll
                for (int s = 0; s < S; ++s) f[s][k] = T(2.0 * L::w(k)) * xb[wf * S + s] - f[s][k];
            }
        }
    }
}

// Slab cut: a node on a cut face also writes its post-collision populations
// that leave through that face into the face's send buffer.
template <int LAT, int S, typename T>
__device__ __forceinline__ void pack_halo(const T (&f)[S][Lattice<LAT>::Q], const Geom& g,
                                          const Neighbourhood& h, const Halo<T>& halo)
{
    using L = Lattice<LAT>;
    constexpr int DIM = L::DIM;
#pragma unroll
    for (int k = 0; k < L::Q; ++k) {
        const int c = split_c<LAT>(k);
        if (c == 0) continue;
        if (!(h.hal & (c > 0 ? halo_hi_bit<DIM>() : halo_lo_bit<DIM>()))) continue;
        T* sb = c > 0 ? halo.send_hi : halo.send_lo;
#pragma unroll
        for (int s = 0; s < S; ++s) sb[((size_t)halo_slot<LAT>(k) * S + s) * g.plane + h.inpl] = f[s][k];
    }
}

// From the pre-collision populations f at a node and its L1h = Lambda_1/2: the
// fluxes J = (I - Lambda_1/2) m_1 (Eq. 2-12 with Eq. 3-26) and the local
// gradients grad xi = -Lambda_1 m_1 / c_s^2 (Eq. xix), m_1 = sum_k c_k f_k; the
// last species' rows close the sums (Eq. 2-3a).
template <int LAT, int S, typename T>
__device__ __forceinline__ void flux_and_gradient(const T (&f)[S][Lattice<LAT>::Q],
                                                  const T (&L1h)[S][S],
                                                  T (&J)[S + 1][Lattice<LAT>::DIM],
                                                  T (&G)[S + 1][Lattice<LAT>::DIM])
{
    using L = Lattice<LAT>;
    constexpr int Q = L::Q;
    constexpr int DIM = L::DIM;
    T m1[S][DIM];
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            T acc = T(0);
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                const int c = a == 0 ? L::cx(k) : (a == 1 ? L::cy(k) : L::cz(k));
                if (c == 1) acc += f[s][k];
                if (c == -1) acc -= f[s][k];
            }
            m1[s][a] = acc;
        }
#pragma unroll
    for (int a = 0; a < DIM; ++a) J[S][a] = G[S][a] = T(0);
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            T lm = T(0);  // (Lambda_1 m_1)/2
#pragma unroll
            for (int j = 0; j < S; ++j) lm += L1h[s][j] * m1[j][a];
            J[s][a] = m1[s][a] - lm;
            J[S][a] -= J[s][a];
            G[s][a] = -lm * T(2.0 / L::cs2());
            G[S][a] -= G[s][a];
        }
}

// Two-sum accumulation (Knuth): (s, c) += v with the rounding error kept in c.
__device__ __forceinline__ void two_sum_add(double& s, double& c, double v)
{
    const double t = s + v;
    const double bp = t - s;
    c += (s - (t - bp)) + (v - bp);
    s = t;
}

// (s, c) += (s2, c2)
__device__ __forceinline__ void two_sum_merge(double& s, double& c, double s2, double c2)
{
    two_sum_add(s, c, s2);
    c += c2;
}

}  // namespace lbms
