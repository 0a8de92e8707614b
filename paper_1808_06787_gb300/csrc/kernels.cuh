// Node kernels of the solver, templated on lattice, number of evolved species
// S = n - 1 and element type.  One thread owns one node; populations are
// structure-of-arrays, f[(s * Q + k) * cells + cell] with cell = (z * ny + y) *
// nx + x, so that a warp touches 32 consecutive nodes of one population plane.
#pragma once

#include <math.h>

#include "node.cuh"

namespace lbms {

template <typename T>
struct Coeffs {
    T invD[LBMS_MAX_SPECIES][LBMS_MAX_SPECIES];  // 1/D_ij times make_coeffs' scale
    T xref[LBMS_MAX_SPECIES];  // reference composition of LBMS_RELAX_FROZEN
};

// The composition the relaxation matrices are evaluated at: the node's own, or
// the fixed reference of the frozen mode (a test mode that makes the scheme linear).
template <int S, typename T>
__device__ __forceinline__ void lambda_composition(const T (&xi)[S + 1], const Coeffs<T>& co,
                                                   int relax, T (&xl)[S + 1])
{
#pragma unroll
    for (int s = 0; s <= S; ++s) xl[s] = relax == LBMS_RELAX_FROZEN ? co.xref[s] : xi[s];
}

// Mass partials.  FP32 solvers accumulate each node's mole fraction as a signed
// 64-bit fixed-point number xi * 2^shift (exact integer sums, independent of
// order); FP64 solvers use FP64 two-sum pairs.  Both reduce in a fixed order.
struct MassOut {
    void* partials;  // [blocks][S + 1] of int64 (FP32) or double2 (FP64)
    int shift;       // fixed-point fraction bits (FP32)
};

template <typename T>
struct StepParams {
    const T* __restrict__ fin;
    T* __restrict__ fout;
    Geom g;
    int relax;
    MassOut mass;
    uint32_t* status;
    // step counter: read from clock_in, written (+1) to clock_out; the two
    // words alternate with the population buffers, so replays of a captured
    // graph see the true step count
    const uint32_t* clock_in;
    uint32_t* clock_out;
    const T* __restrict__ xb;  // Dirichlet face compositions [6][S]
    Halo<T> halo;              // slab cuts: receive buffers of fin's parity, send buffers
    int reverse;               // blocks take the grid from its end (block b does block n - 1 - b)
    Coeffs<T> co;
};

// Programmatic dependent launch (sm_90 and later).  Time steps are launched
// with programmatic stream serialisation (launch_chained below), so the blocks
// of the next step may be made resident while the current one still runs and
// its launch latency is hidden.  Before touching memory, every thread waits
// here until the grid before it in the stream has completed and its stores are
// visible (a wait the hardware resolves, not a spin on memory), then lets the
// following grid be scheduled.  Arithmetic on the launch parameters alone may
// come first.  In a grid launched without the attribute both return at once.
__device__ __forceinline__ void await_previous_grid()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Launches `kernel` with programmatic stream serialisation: only the
// dependency on the kernel before it in the stream is relaxed, and the kernel
// must call await_previous_grid before touching memory that grid writes or reads.
template <typename... Params, typename... Args>
cudaError_t launch_chained(void (*kernel)(Params...), uint32_t blocks, uint32_t threads,
                           cudaStream_t stream, Args... args)
{
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, args...);
    return cudaGetLastError();
}

// Raise the status flags for mole fractions that are non-finite or far
// outside [0, 1]; the comparison is false for NaN, so one test covers both.
template <int S, typename T>
__device__ __forceinline__ void check_range(const T (&xi)[S + 1], uint32_t* status)
{
    bool bad = false;
#pragma unroll
    for (int s = 0; s <= S; ++s) bad |= !(fabs(xi[s] - T(0.5)) <= T(0.55));
    if (bad) {
        uint32_t fl = 0;
#pragma unroll
        for (int s = 0; s <= S; ++s) fl |= isfinite((double)xi[s]) ? LBMS_FLAG_RANGE : LBMS_FLAG_NONFINITE;
        atomicOr(status, fl);
    }
}

// Block-wide fixed-order reductions; thread 0 receives the block total.  All
// threads of the block must call these.
__device__ __forceinline__ long long block_reduce_fixed(long long v, long long* smem)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) smem[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < (int)(blockDim.x >> 5) ? smem[lane] : 0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    }
    __syncthreads();
    return v;
}

__device__ __forceinline__ void block_reduce_pair(double& s, double& c, double2* smem)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double s2 = __shfl_down_sync(0xffffffffu, s, off);
        const double c2 = __shfl_down_sync(0xffffffffu, c, off);
        two_sum_merge(s, c, s2, c2);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) smem[warp] = make_double2(s, c);
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        s = lane < nw ? smem[lane].x : 0.0;
        c = lane < nw ? smem[lane].y : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const double s2 = __shfl_down_sync(0xffffffffu, s, off);
            const double c2 = __shfl_down_sync(0xffffffffu, c, off);
            two_sum_merge(s, c, s2, c2);
        }
    }
    __syncthreads();
}

// Round-to-nearest-even integer of v for |v| <= 2^42, by float additions: adding
// c = 1.5 * 2^45 rounds v to a multiple of 2^22 whose quotient k is the
// difference of the sum's bit pattern and c's (the sum stays in c's binade);
// the remainder r = v - k 2^22 (|r| <= 2^21) is exact and is rounded the same
// way with 1.5 * 2^23, and since k 2^22 is even, round(v) = k 2^22 + round(r)
// with the same ties.  (It replaces the 64-bit float-to-integer conversion,
// which issues at the FP64 rate, a few per clock per SM.)
__device__ __forceinline__ long long round_to_ll(float v)
{
    const float c = 0x1.8p45f, d = 0x1.8p23f;
    const float sum = __fadd_rn(v, c);
    const int k = __float_as_int(sum) - __float_as_int(c);
    const float r = __fadd_rn(v, -__fadd_rn(sum, -c));
    const int j = __float_as_int(__fadd_rn(r, d)) - __float_as_int(d);
    return (long long)k * (1ll << 22) + j;
}

// The block's sums of N fixed-point values per thread, written to out_row[0..N),
// with one barrier: each warp adds its values by shuffles, lane 0 parks them in
// shared memory, and thread s < N adds slot s of the warps in warp order.
// (Integer sums are exact, so the partials do not depend on the grouping.)
// Called once, at the end of a kernel (the shared slots are not reused).
template <int N>
__device__ __forceinline__ void block_fixed_partials(long long (&q)[N], long long* out_row)
{
    __shared__ long long red[kBlock / 32][N];
#pragma unroll
    for (int s = 0; s < N; ++s)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) q[s] += __shfl_down_sync(0xffffffffu, q[s], off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int s = 0; s < N; ++s) red[warp][s] = q[s];
    __syncthreads();
    if (threadIdx.x < N) {
        long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w][threadIdx.x];
        out_row[threadIdx.x] = t;
    }
}

// Per-block partial sums of the n = S + 1 mole fractions (zero for idle threads).
template <int S>
__device__ __forceinline__ void write_mass_partials(const float (&xi)[S + 1], bool active,
                                                    const MassOut& m, uint32_t row)
{
    const float scale = __int_as_float((127 + m.shift) << 23);  // 2^shift, exact
    long long q[S + 1];
#pragma unroll
    for (int s = 0; s <= S; ++s) {
        // |xi| beyond 4 (already flagged) is clipped so that sums cannot overflow
        const float v = active ? fminf(fmaxf(xi[s], -4.0f), 4.0f) : 0.0f;
        q[s] = round_to_ll(__fmul_rn(v, scale));
    }
    block_fixed_partials<S + 1>(q, static_cast<long long*>(m.partials) + (size_t)row * (S + 1));
}

template <int S>
__device__ __forceinline__ void write_mass_partials(const double (&xi)[S + 1], bool active,
                                                    const MassOut& m, uint32_t row)
{
    __shared__ double2 red[kBlock / 32];
    double2* out = static_cast<double2*>(m.partials);
#pragma unroll
    for (int s = 0; s <= S; ++s) {
        double sum = active ? xi[s] : 0.0, comp = 0.0;
        block_reduce_pair(sum, comp, red);
        if (threadIdx.x == 0) out[(size_t)row * (S + 1) + s] = make_double2(sum, comp);
    }
}

// The block of the grid a step kernel's block takes.  Steps alternate: a
// forward step takes the grid in order; a reverse step takes chunks of
// kRevChunk blocks from the grid's end, each chunk in order, so that it starts
// on the blocks the forward step wrote last, which are still in L2, while its
// accesses still ascend within a chunk.  (A permutation of the blocks: the
// last chunk taken is the remainder at the grid's start.)  Chunks of 32 to
// 256 blocks measured alike and best; 1024 slightly and 4096 or the whole
// grid clearly slower (D3Q7 256^3: 1.045, 1.043, 1.035, 1.033).
constexpr uint32_t kRevChunk = 64;

__device__ __forceinline__ uint32_t grid_block(int reverse)
{
    if (!reverse) return blockIdx.x;
    const uint32_t c = blockIdx.x / kRevChunk, w = blockIdx.x - c * kRevChunk;
    const uint32_t hi = gridDim.x - c * kRevChunk;  // end of the chunk, counted from the grid's end
    return (hi > kRevChunk ? hi - kRevChunk : 0u) + w;
}

// Blocks per SM the FP32 step kernels are compiled for (register budget): one
// node per thread keeps S * Q populations and the S x S matrices in registers,
// and enough resident warps must remain to cover HBM latency.
template <int LAT, int S, typename T>
struct StepOccupancy {
    static constexpr int P = S * Lattice<LAT>::Q;  // populations held per thread
    static constexpr int value =
        sizeof(T) != 4 ? 1
        : Lattice<LAT>::Q <= 9 ? (S <= 2 ? 6 : (S == 3 ? 4 : (S == 4 ? 3 : 2)))
                               : (P <= 15 ? 4 : (P <= 30 ? 3 : 2));
};

// One time step: pull-stream (Eq. 3-13b, bounce-back/periodic faces), mole
// fractions (Eq. 3-15), relaxation matrices (Eqs. 2-10, 3-26, 3-16), collision
// (Eq. 3-13a with f_eq of Eq. 3-3) and store of the post-collision populations.
// HALO: the grid is a slab with cut faces (slab decomposition); kernels of
// undivided grids are compiled without the halo code.
template <int LAT, int S, typename T, bool MASS, bool HALO>
__global__ void __launch_bounds__(kBlock, StepOccupancy<LAT, S, T>::value) k_step(StepParams<T> p)
{
    using L = Lattice<LAT>;
    constexpr int Q = L::Q;
    await_previous_grid();
    const uint32_t lb = grid_block(p.reverse);
    const uint32_t cell = lb * blockDim.x + threadIdx.x;
    const bool active = cell < p.g.cells;
    const uint32_t step = *p.clock_in;
    if (blockIdx.x == 0 && threadIdx.x == 0) *p.clock_out = step + 1;
    T xi[S + 1];
    if (active) {
        const Neighbourhood h = neighbourhood<Lattice<LAT>::DIM, HALO>(p.g, cell);
        T f[S][Q];
        pull<LAT, S, T>(p.fin, p.g, cell, h, f, p.xb, HALO ? &p.halo : nullptr);
        mole_fractions<LAT, S, T>(f, xi);
        if (MASS) check_range<S, T>(xi, p.status);  // once per lbms_step call
        T L1[S][S], L2[S][S];
        T xl[S + 1];
        lambda_composition<S, T>(xi, p.co, p.relax, xl);
        relaxation_matrices<S, T>(xl, p.co.invD, T(1.0 / L::cs2()), p.relax, L1, L2);
        // the rounding key uses the node's index in the undivided grid, so that
        // the slabs of a decomposed grid round as the whole grid does
        collide<LAT, S, T>(f, xi, L1, L2,
                           mix32(step * 0x9e3779b9u) ^ ((HALO ? cell + p.g.origin : cell) * 0x27d4eb2du));
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int k = 0; k < Q; ++k) p.fout[(size_t)(s * Q + k) * p.g.cells + cell] = f[s][k];
        if (HALO && h.hal) pack_halo<LAT, S, T>(f, p.g, h, p.halo);
    }
    if (MASS) write_mass_partials<S>(xi, active, p.mass, lb);
}

// Two nodes per thread (c, c + 1 with c even), for the lattices with Q <= 7 and
// S <= 2 in FP32, whose per-node instruction count rather than HBM bandwidth
// limits the one-node kernel: the pair's rest populations (if the lattice has a
// rest velocity) come in one 8-byte load, with an even nx so do the populations
// that do not move along x (load_pair_y), every post-collision plane goes out in
// one 8-byte store, and the per-thread set-up is shared; the per-node
// arithmetic is that of k_step, so the results are the same bit for bit.
// Blocks of kBlock / 2 threads cover kBlock nodes, the partition of k_step (and
// the same alternation of directions, grid_block).  Needs an even node count (so
// that every population plane starts at an even node); no cut faces.
template <typename T>
struct Pair;
template <>
struct Pair<float> {
    using type = float2;
};
template <>
struct Pair<double> {
    using type = double2;
};

// The moving populations that do not move along x, of the node pair (c0, c0 + 1)
// sharing a row (and a z-plane): one aligned pair load per species and population
// (see k_step_pair).
template <int LAT, int S, typename T>
__device__ __forceinline__ void load_pair_y(const T* __restrict__ fin, uint32_t plane_stride, uint32_t c0,
                                            const Neighbourhood& h, T (&f)[2][S][Lattice<LAT>::Q])
{
    using L = Lattice<LAT>;
    using V = typename Pair<T>::type;
#pragma unroll
    for (int k = 0; k < L::Q; ++k) {
        const int cx = L::cx(k), cy = L::cy(k), cz = L::cz(k);
        if (cx != 0 || (cy == 0 && cz == 0)) continue;
        int32_t off = 0;
        bool bounce = false;
        if (cy != 0) { off += h.oy[cy > 0 ? 0 : 1]; bounce |= h.by[cy > 0 ? 0 : 1]; }
        if (cz != 0) { off += h.oz[cz > 0 ? 0 : 1]; bounce |= h.bz[cz > 0 ? 0 : 1]; }
        const uint32_t src = bounce ? c0 : (uint32_t)((int32_t)c0 + off);
        const size_t plane = (size_t)(bounce ? opp<LAT>(k) : k) * plane_stride;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const V v = *reinterpret_cast<const V*>(fin + (size_t)s * L::Q * plane_stride + plane + src);
            f[0][s][k] = v.x;
            f[1][s][k] = v.y;
        }
    }
}

// Blocks of kBlock / 2 threads per SM asked of the compiler, measured on the
// full-size grids: for D1Q3, D2Q4, D2Q5 and D3Q6 (ternary) the largest count at
// which the plain step compiles without spilling (40, 40, 48 and 56
// registers), each faster than fewer blocks while one more (spilling) is
// slower; for D3Q7, 9 blocks at 56 registers with a 24-byte spill (0.3 %
// faster than 8 blocks without; 10 blocks, 48 registers: 2 % slower).
template <int LAT, int S, typename T>
struct PairOccupancy {
    static constexpr int Q = Lattice<LAT>::Q;
    static constexpr int value = S <= 1 ? 12 : (Q <= 4 ? 12 : (Q == 5 ? 10 : 9));
    // the mass-writing variant holds the pair's mole fractions too: on the 3D
    // lattices it keeps 8 blocks (D3Q7 at 64 registers spills 28 bytes instead
    // of 68; 20-step calls 1.042 -> 1.044 of the copy peak)
    static constexpr int mass = S == 2 && Q >= 6 ? 8 : value;
};

// Mass partials of a pair kernel's block (the block partition of k_step, so the
// partials are the same integers): each thread adds its two nodes' fixed-point
// values before the block reduction.
template <int S>
__device__ __forceinline__ void write_mass_partials_pair(const float (&xi)[2][S + 1], bool active,
                                                         const MassOut& m, uint32_t row)
{
    const float scale = __int_as_float((127 + m.shift) << 23);  // 2^shift, exact
    long long q[S + 1];
#pragma unroll
    for (int s = 0; s <= S; ++s) {
        q[s] = 0;
#pragma unroll
        for (int j = 0; j < 2; ++j)
            q[s] += round_to_ll(__fmul_rn(active ? fminf(fmaxf(xi[j][s], -4.0f), 4.0f) : 0.0f, scale));
    }
    block_fixed_partials<S + 1>(q, static_cast<long long*>(m.partials) + (size_t)row * (S + 1));
}

// MASS: the last step of a call, which also tests the mole fractions' range and
// writes the mass partials (as k_step<..., true, ...>).
template <int LAT, int S, typename T, bool MASS>
__global__ void __launch_bounds__(kBlock / 2, MASS ? PairOccupancy<LAT, S, T>::mass : PairOccupancy<LAT, S, T>::value)
    k_step_pair(StepParams<T> p)
{
    using L = Lattice<LAT>;
    using V = typename Pair<T>::type;
    constexpr int Q = L::Q;
    constexpr bool REST = L::K0 == 1;  // lattices without a rest velocity gather every population
    static_assert(!MASS || sizeof(T) == 4, "the pair kernels are FP32");
    await_previous_grid();
    const uint32_t lb = grid_block(p.reverse);
    const uint32_t c0 = lb * kBlock + 2 * threadIdx.x;
    const uint32_t step = *p.clock_in;
    if (blockIdx.x == 0 && threadIdx.x == 0) *p.clock_out = step + 1;
    const bool active = c0 < p.g.cells;  // cells is even: both nodes or neither
    T xs[2][S + 1];
    if (!MASS && !active) return;
    if (active) {
        T f[2][S][Q];
        if constexpr (REST) {
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const V r = *reinterpret_cast<const V*>(p.fin + (size_t)(s * Q) * p.g.cells + c0);
                f[0][s][0] = r.x;
                f[1][s][0] = r.y;
            }
        }
        const uint32_t hk = mix32(step * 0x9e3779b9u);
        // with an even nx the pair shares a row, so its sources that do not move along
        // x are an aligned pair too (offsets +-nx, +-nx ny or the wraps, or both nodes
        // bounce at the same wall)
        const bool pair_y = L::DIM >= 2 && (p.g.nx & 1) == 0;
        Neighbourhood h[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) h[j] = neighbourhood<L::DIM, false>(p.g, c0 + j);
        if (pair_y) load_pair_y<LAT, S, T>(p.fin, p.g.cells, c0, h[0], f);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const uint32_t cell = c0 + j;
            if (pair_y)
                pull<LAT, S, T, REST, true>(p.fin, p.g, cell, h[j], f[j], p.xb);
            else
                pull<LAT, S, T, REST, false>(p.fin, p.g, cell, h[j], f[j], p.xb);
            T xi[S + 1];
            mole_fractions<LAT, S, T>(f[j], xi);
            if (MASS) {
                check_range<S, T>(xi, p.status);
#pragma unroll
                for (int s = 0; s <= S; ++s) xs[j][s] = xi[s];
            }
            T L1[S][S], L2[S][S];
            T xl[S + 1];
            lambda_composition<S, T>(xi, p.co, p.relax, xl);
            relaxation_matrices<S, T>(xl, p.co.invD, T(1.0 / L::cs2()), p.relax, L1, L2);
            collide<LAT, S, T>(f[j], xi, L1, L2, hk ^ (cell * 0x27d4eb2du));
        }
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                V v;
                v.x = f[0][s][k];
                v.y = f[1][s][k];
                *reinterpret_cast<V*>(p.fout + (size_t)(s * Q + k) * p.g.cells + c0) = v;
            }
    }
    if constexpr (MASS) write_mass_partials_pair<S>(xs, active, p.mass, lb);
}

// Smallest grid stepped by the pair kernel: 2^21 nodes, whose populations
// (at least 2 x 2 x 3 x 4 B per node) no longer fit the 129 MB L2.
constexpr uint32_t kPairMinCells = 1u << 21;

// Whether the pair kernel takes a step of this solver (see k_step_pair).
template <int LAT, int S, typename T>
constexpr bool pair_kernel_lattice()
{
    return Lattice<LAT>::Q <= 7 && S <= 2 && sizeof(T) == 4;
}

// Mass partials of the current (post-collision) state without stepping.
template <int LAT, int S, typename T>
__global__ void __launch_bounds__(kBlock) k_mass(StepParams<T> p)
{
    constexpr int Q = Lattice<LAT>::Q;
    const uint32_t cell = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = cell < p.g.cells;
    T xi[S + 1];
    if (active) {
        T f[S][Q];
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int k = 0; k < Q; ++k) f[s][k] = p.fout[(size_t)(s * Q + k) * p.g.cells + cell];
        mole_fractions<LAT, S, T>(f, xi);
    }
    write_mass_partials<S>(xi, active, p.mass, blockIdx.x);
}

template <typename T>
struct FieldParams {
    const T* fprev;   // post-collision populations at t-1 (null at t = 0)
    T* fcur;          // post-collision populations at t (init writes, moments reads)
    const T* x_in;    // init: [S+1][stride]
    T* x_out;         // moments: [S+1][stride]
    T* J_out;         // moments: [S+1][dim][stride] or null
    T* G_out;         // moments: local gradients [S+1][dim][stride] or null
    Geom g;
    uint32_t c0, c1, stride;
    int relax;
    uint32_t* status;
    const T* xb;      // Dirichlet face compositions [6][S]
    Halo<T> halo;     // slab cuts: receive buffers of fprev's parity (moments), send buffers (init)
    Coeffs<T> co;
};

// f+_k^i(t = 0) = w_k xi_i (Sec. 4, initialisation); flags inputs that are not
// finite or do not sum to one.
template <int LAT, int S, typename T>
__global__ void __launch_bounds__(kBlock) k_init(FieldParams<T> p)
{
    using L = Lattice<LAT>;
    constexpr int Q = L::Q;
    const uint32_t i = blockIdx.x * kBlock + threadIdx.x;
    const uint32_t cell = p.c0 + i;
    if (cell >= p.c1) return;
    T xi[S + 1];
    double sum = 0.0;
    bool finite = true;
#pragma unroll
    for (int s = 0; s <= S; ++s) {
        xi[s] = p.x_in[(size_t)s * p.stride + i];
        sum += (double)xi[s];
        finite &= (bool)isfinite((double)xi[s]);
    }
    if (!finite || !(fabs(sum - 1.0) <= 1e-5)) atomicOr(p.status, LBMS_FLAG_INIT);
    // moving populations w_k xi; the rest population takes what is left of xi,
    // so that sum_k f_k = xi up to one rounding whatever the weights round to
    T f[S][Q];
#pragma unroll
    for (int s = 0; s < S; ++s) {
        T moving = T(0);
#pragma unroll
        for (int k = 1; k < Q; ++k) {
            const T fk = T(L::w(k)) * xi[s];
            moving += fk;
            f[s][k] = fk;
            p.fcur[(size_t)(s * Q + k) * p.g.cells + cell] = fk;
        }
        f[s][0] = xi[s] - moving;
        p.fcur[(size_t)(s * Q) * p.g.cells + cell] = f[s][0];
    }
    if (p.g.halo) {  // a slab: its cut layers also fill the send buffers
        const Neighbourhood h = neighbourhood<L::DIM>(p.g, cell);
        if (h.hal) pack_halo<LAT, S, T>(f, p.g, h, p.halo);
    }
}

// Mole fractions at t from the stored post-collision populations (the collision
// conserves each xi); fluxes J = (I - Lambda_1/2) m_1 and local gradients
// grad xi = -Lambda_1 m_1 / c_s^2 (Eq. xix) of the pre-collision populations at
// t, gathered again from the previous buffer.  Each output is optional.
template <int LAT, int S, typename T>
__global__ void __launch_bounds__(kBlock) k_moments(FieldParams<T> p)
{
    using L = Lattice<LAT>;
    constexpr int Q = L::Q;
    constexpr int DIM = L::DIM;
    const uint32_t i = blockIdx.x * kBlock + threadIdx.x;
    const uint32_t cell = p.c0 + i;
    if (cell >= p.c1) return;
    if (p.x_out) {
        T f[S][Q];
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int k = 0; k < Q; ++k) f[s][k] = p.fcur[(size_t)(s * Q + k) * p.g.cells + cell];
        T xi[S + 1];
        mole_fractions<LAT, S, T>(f, xi);
#pragma unroll
        for (int s = 0; s <= S; ++s) p.x_out[(size_t)s * p.stride + i] = xi[s];
    }
    if (!p.J_out && !p.G_out) return;
    T J[S + 1][DIM], G[S + 1][DIM];
#pragma unroll
    for (int s = 0; s <= S; ++s)
#pragma unroll
        for (int a = 0; a < DIM; ++a) J[s][a] = G[s][a] = T(0);
    if (p.fprev) {
        const Neighbourhood h = neighbourhood<Lattice<LAT>::DIM>(p.g, cell);
        T f[S][Q];
        pull<LAT, S, T>(p.fprev, p.g, cell, h, f, p.xb, &p.halo);
        T xi[S + 1];
        mole_fractions<LAT, S, T>(f, xi);
        T L1[S][S], L2[S][S];
        T xl[S + 1];
        lambda_composition<S, T>(xi, p.co, p.relax, xl);
        relaxation_matrices<S, T>(xl, p.co.invD, T(1.0 / L::cs2()), p.relax, L1, L2);
        flux_and_gradient<LAT, S, T>(f, L1, J, G);
    }
    if (p.J_out)
#pragma unroll
        for (int s = 0; s <= S; ++s)
#pragma unroll
            for (int a = 0; a < DIM; ++a) p.J_out[((size_t)s * DIM + a) * p.stride + i] = J[s][a];
    if (p.G_out)
#pragma unroll
        for (int s = 0; s <= S; ++s)
#pragma unroll
            for (int a = 0; a < DIM; ++a) p.G_out[((size_t)s * DIM + a) * p.stride + i] = G[s][a];
}

// `scale` multiplies the inverse diffusivities: 0.5 for the kernels that take
// the halved ones (relaxation_matrices), 1 for the adjoint.
template <typename T>
Coeffs<T> make_coeffs(const KArgs& a, double scale)
{
    Coeffs<T> c;
    for (int i = 0; i < LBMS_MAX_SPECIES; ++i) {
        for (int j = 0; j < LBMS_MAX_SPECIES; ++j) c.invD[i][j] = (T)(scale * a.invD[i][j]);
        c.xref[i] = (T)a.xref[i];
    }
    return c;
}

template <typename T>
Halo<T> make_halo(const KArgs& a)
{
    Halo<T> h;
    h.recv_lo = static_cast<const T*>(a.halo_recv[0]);
    h.recv_hi = static_cast<const T*>(a.halo_recv[1]);
    h.send_lo = static_cast<T*>(a.halo_send[0]);
    h.send_hi = static_cast<T*>(a.halo_send[1]);
    return h;
}

inline FastDiv make_fastdiv(uint32_t d)
{
    uint32_t l = 0;
    while ((1ull << l) < d) ++l;
    FastDiv f;
    f.s = 31 + l;
    f.m = ((1ull << f.s) + d - 1) / d;
    return f;
}

inline Geom make_geom(const KArgs& a)
{
    Geom g;
    g.nx = a.nx; g.ny = a.ny; g.nz = a.nz;
    g.nxy = (uint32_t)a.nx * (uint32_t)a.ny;
    g.cells = a.cells;
    g.noflux = a.noflux | a.dirichlet;
    g.dirichlet = a.dirichlet;
    g.halo = a.halo;
    g.plane = a.plane;
    g.origin = a.origin;
    g.dnx = make_fastdiv((uint32_t)a.nx);
    g.dny = make_fastdiv((uint32_t)a.ny);
    return g;
}

// HALO_STEPS selects the step kernels of slabs (grids with cut faces): the
// per-lattice translation units k_*.cu instantiate the others and kh_*.cu these,
// so that the two halves compile in parallel.
template <int LAT, int S, typename T, bool HALO_STEPS>
cudaError_t launch(Op op, const KArgs& a)
{
    if (op == OP_STEP || op == OP_STEP_MASS || op == OP_MASS) {
        StepParams<T> p;
        p.fin = static_cast<const T*>(a.fin);
        p.fout = static_cast<T*>(a.fout);
        p.g = make_geom(a);
        p.relax = a.relax;
        p.mass.partials = a.partials;
        p.mass.shift = a.fixed_shift;
        p.status = a.status;
        p.clock_in = a.clock_in;
        p.clock_out = a.clock_out;
        p.xb = static_cast<const T*>(a.xb);
        p.halo = make_halo<T>(a);
        // alternate steps take the grid from its end (undivided grids; measured
        // on one box against forward-only steps: D3Q7 256^3 +0.8 %, D3Q6 +0.5 to
        // 1.5 %, D2Q9 N = 5 +0.9 %, D2Q5 and D1Q3 +0.3 %, D3Q15 -0.2 %)
        p.reverse = HALO_STEPS ? 0 : a.reverse;
        p.co = make_coeffs<T>(a, 0.5);
        const uint32_t tb = a.step_block;
        const uint32_t blocks = (a.cells + tb - 1) / tb;
        if constexpr (HALO_STEPS) {
            // slabs step one exchange at a time: every step writes the mass
            // partials (one kernel variant instead of two)
            if (op == OP_STEP || op == OP_STEP_MASS)
                return launch_chained(k_step<LAT, S, T, true, true>, blocks, tb, a.stream, p);
            return cudaErrorInvalidValue;
        } else {
            if constexpr (pair_kernel_lattice<LAT, S, T>()) {
                // grids whose state stays in L2 keep one node per thread (more
                // threads for the latency-bound small grid)
                if (a.cells >= kPairMinCells && (a.cells & 1u) == 0 && tb == kBlock) {
                    if (op == OP_STEP)
                        return launch_chained(k_step_pair<LAT, S, T, false>, blocks, kBlock / 2, a.stream, p);
                    if (op == OP_STEP_MASS)
                        return launch_chained(k_step_pair<LAT, S, T, true>, blocks, kBlock / 2, a.stream, p);
                }
            }
            if (op == OP_STEP) return launch_chained(k_step<LAT, S, T, false, false>, blocks, tb, a.stream, p);
            if (op == OP_STEP_MASS) return launch_chained(k_step<LAT, S, T, true, false>, blocks, tb, a.stream, p);
            p.reverse = 0;
            k_mass<LAT, S, T><<<blocks, tb, 0, a.stream>>>(p);
            return cudaGetLastError();
        }
    }
    if constexpr (HALO_STEPS) {
        return cudaErrorInvalidValue;
    } else {
        FieldParams<T> p;
        p.fprev = static_cast<const T*>(a.fin);
        p.fcur = static_cast<T*>(a.fout);
        p.x_in = static_cast<const T*>(a.field_in);
        p.x_out = static_cast<T*>(a.field_x);
        p.J_out = static_cast<T*>(a.field_J);
        p.G_out = static_cast<T*>(a.field_G);
        p.g = make_geom(a);
        p.c0 = a.c0; p.c1 = a.c1; p.stride = a.stride;
        p.relax = a.relax;
        p.status = a.status;
        p.xb = static_cast<const T*>(a.xb);
        p.halo = make_halo<T>(a);
        p.co = make_coeffs<T>(a, 0.5);
        const uint32_t blocks = node_blocks(a.c1 - a.c0);
        if (blocks == 0) return cudaSuccess;
        if (op == OP_INIT)
            k_init<LAT, S, T><<<blocks, kBlock, 0, a.stream>>>(p);
        else
            k_moments<LAT, S, T><<<blocks, kBlock, 0, a.stream>>>(p);
        return cudaGetLastError();
    }
}

template <int LAT, typename T, bool HALO_STEPS>
cudaError_t dispatch_S(Op op, const KArgs& a)
{
    switch (a.n_species - 1) {
        case 1: return launch<LAT, 1, T, HALO_STEPS>(op, a);
        case 2: return launch<LAT, 2, T, HALO_STEPS>(op, a);
        case 3: return launch<LAT, 3, T, HALO_STEPS>(op, a);
        case 4: return launch<LAT, 4, T, HALO_STEPS>(op, a);
        case 5: return launch<LAT, 5, T, HALO_STEPS>(op, a);
        case 6: return launch<LAT, 6, T, HALO_STEPS>(op, a);
        case 7: return launch<LAT, 7, T, HALO_STEPS>(op, a);
        default: return cudaErrorInvalidValue;
    }
}

template <int LAT, bool HALO_STEPS>
cudaError_t dispatch_lattice(Op op, int dtype, const KArgs& a)
{
    return dtype == LBMS_F64 ? dispatch_S<LAT, double, HALO_STEPS>(op, a)
                             : dispatch_S<LAT, float, HALO_STEPS>(op, a);
}

// Whether an operation runs a slab's step kernels (kh_*.cu).
inline bool slab_step_op(Op op, const KArgs& a) { return a.halo && (op == OP_STEP || op == OP_STEP_MASS); }

}  // namespace lbms
