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
    T invD[LBMS_MAX_SPECIES][LBMS_MAX_SPECIES];
};

template <typename T>
struct StepParams {
    const T* __restrict__ fin;
    T* __restrict__ fout;
    int nx, ny, nz;
    uint32_t cells;
    uint32_t noflux;
    int relax;
    double2* partials;  // [blocks][S + 1] when mass partials are requested
    uint32_t* status;
    Coeffs<T> co;
};

__device__ __forceinline__ void node_coords(uint32_t cell, int nx, int ny, int& x, int& y, int& z)
{
    const uint32_t row = cell / (uint32_t)nx;
    x = (int)(cell - row * (uint32_t)nx);
    z = (int)(row / (uint32_t)ny);
    y = (int)(row - (uint32_t)z * (uint32_t)ny);
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

// Block-wide fixed-order reduction of one (sum, compensation) pair per thread;
// thread 0 returns the block total.  All threads of the block must call it.
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

// Per-block partial sums of the n = S + 1 mole fractions held by the threads.
template <int S>
__device__ __forceinline__ void write_mass_partials(const double (&v)[S + 1], double2* partials)
{
    __shared__ double2 red[kBlock / 32];
#pragma unroll
    for (int s = 0; s <= S; ++s) {
        double sum = v[s], comp = 0.0;
        block_reduce_pair(sum, comp, red);
        if (threadIdx.x == 0) partials[(size_t)blockIdx.x * (S + 1) + s] = make_double2(sum, comp);
    }
}

// One time step: pull-stream (Eq. 3-13b, bounce-back/periodic faces), mole
// fractions (Eq. 3-15), relaxation matrices (Eqs. 2-10, 3-26, 3-16), collision
// (Eq. 3-13a with f_eq of Eq. 3-3) and store of the post-collision populations.
template <int LAT, int S, typename T, bool MASS>
__global__ void __launch_bounds__(kBlock) k_step(StepParams<T> p)
{
    using L = Lattice<LAT>;
    constexpr int Q = L::Q;
    const uint32_t cell = blockIdx.x * kBlock + threadIdx.x;
    const bool active = cell < p.cells;
    T xi[S + 1];
    if (active) {
        int x, y, z;
        node_coords(cell, p.nx, p.ny, x, y, z);
        T f[S][Q];
        pull<LAT, S, T>(p.fin, p.cells, x, y, z, p.nx, p.ny, p.nz, cell, p.noflux, f);
        mole_fractions<LAT, S, T>(f, xi);
        check_range<S, T>(xi, p.status);
        T L1[S][S], L2[S][S];
        relaxation_matrices<S, T>(xi, p.co.invD, T(1.0 / L::cs2()), p.relax, L1, L2);
        collide<LAT, S, T>(f, xi, L1, L2, cell * 0x27d4eb2du);
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int k = 0; k < Q; ++k) p.fout[(size_t)(s * Q + k) * p.cells + cell] = f[s][k];
    }
    if (MASS) {
        double v[S + 1];
#pragma unroll
        for (int s = 0; s <= S; ++s) v[s] = active ? (double)xi[s] : 0.0;
        write_mass_partials<S>(v, p.partials);
    }
}

// Mass partials of the current (post-collision) state without stepping.
template <int LAT, int S, typename T>
__global__ void __launch_bounds__(kBlock) k_mass(StepParams<T> p)
{
    constexpr int Q = Lattice<LAT>::Q;
    const uint32_t cell = blockIdx.x * kBlock + threadIdx.x;
    double v[S + 1];
    if (cell < p.cells) {
        T f[S][Q];
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int k = 0; k < Q; ++k) f[s][k] = p.fout[(size_t)(s * Q + k) * p.cells + cell];
        T xi[S + 1];
        mole_fractions<LAT, S, T>(f, xi);
#pragma unroll
        for (int s = 0; s <= S; ++s) v[s] = (double)xi[s];
    } else {
#pragma unroll
        for (int s = 0; s <= S; ++s) v[s] = 0.0;
    }
    write_mass_partials<S>(v, p.partials);
}

template <typename T>
struct FieldParams {
    const T* fprev;   // post-collision populations at t-1 (null at t = 0)
    T* fcur;          // post-collision populations at t (init writes, moments reads)
    const T* x_in;    // init: [S+1][stride]
    T* x_out;         // moments: [S+1][stride]
    T* J_out;         // moments: [S+1][dim][stride] or null
    int nx, ny, nz;
    uint32_t cells, c0, c1, stride;
    uint32_t noflux;
    int relax;
    uint32_t* status;
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
#pragma unroll
    for (int s = 0; s < S; ++s) {
        T moving = T(0);
#pragma unroll
        for (int k = 1; k < Q; ++k) {
            const T fk = T(L::w(k)) * xi[s];
            moving += fk;
            p.fcur[(size_t)(s * Q + k) * p.cells + cell] = fk;
        }
        p.fcur[(size_t)(s * Q) * p.cells + cell] = xi[s] - moving;
    }
}

// Mole fractions at t from the stored post-collision populations (the collision
// conserves each xi), and fluxes J = (I - Lambda_1/2) m_1 of the pre-collision
// populations at t, gathered again from the previous buffer.
template <int LAT, int S, typename T>
__global__ void __launch_bounds__(kBlock) k_moments(FieldParams<T> p)
{
    using L = Lattice<LAT>;
    constexpr int Q = L::Q;
    constexpr int DIM = L::DIM;
    const uint32_t i = blockIdx.x * kBlock + threadIdx.x;
    const uint32_t cell = p.c0 + i;
    if (cell >= p.c1) return;
    {
        T f[S][Q];
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int k = 0; k < Q; ++k) f[s][k] = p.fcur[(size_t)(s * Q + k) * p.cells + cell];
        T xi[S + 1];
        mole_fractions<LAT, S, T>(f, xi);
#pragma unroll
        for (int s = 0; s <= S; ++s) p.x_out[(size_t)s * p.stride + i] = xi[s];
    }
    if (!p.J_out) return;
    T J[S + 1][DIM];
#pragma unroll
    for (int s = 0; s <= S; ++s)
#pragma unroll
        for (int a = 0; a < DIM; ++a) J[s][a] = T(0);
    if (p.fprev) {
        int x, y, z;
        node_coords(cell, p.nx, p.ny, x, y, z);
        T f[S][Q];
        pull<LAT, S, T>(p.fprev, p.cells, x, y, z, p.nx, p.ny, p.nz, cell, p.noflux, f);
        T xi[S + 1];
        mole_fractions<LAT, S, T>(f, xi);
        T L1[S][S], L2[S][S];
        relaxation_matrices<S, T>(xi, p.co.invD, T(1.0 / L::cs2()), p.relax, L1, L2);
        T m1[S][DIM];
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                T acc = T(0);
#pragma unroll
                for (int k = 1; k < Q; ++k) {
                    const int c = a == 0 ? L::cx(k) : (a == 1 ? L::cy(k) : L::cz(k));
                    if (c == 1) acc += f[s][k];
                    if (c == -1) acc -= f[s][k];
                }
                m1[s][a] = acc;
            }
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                T acc = m1[s][a];
#pragma unroll
                for (int j = 0; j < S; ++j) acc -= T(0.5) * L1[s][j] * m1[j][a];
                J[s][a] = acc;
                J[S][a] -= acc;
            }
    }
#pragma unroll
    for (int s = 0; s <= S; ++s)
#pragma unroll
        for (int a = 0; a < DIM; ++a) p.J_out[((size_t)s * DIM + a) * p.stride + i] = J[s][a];
}

template <typename T>
Coeffs<T> make_coeffs(const KArgs& a)
{
    Coeffs<T> c;
    for (int i = 0; i < LBMS_MAX_SPECIES; ++i)
        for (int j = 0; j < LBMS_MAX_SPECIES; ++j) c.invD[i][j] = (T)a.invD[i][j];
    return c;
}

template <int LAT, int S, typename T>
cudaError_t launch(Op op, const KArgs& a)
{
    if (op == OP_STEP || op == OP_STEP_MASS || op == OP_MASS) {
        StepParams<T> p;
        p.fin = static_cast<const T*>(a.fin);
        p.fout = static_cast<T*>(a.fout);
        p.nx = a.nx; p.ny = a.ny; p.nz = a.nz;
        p.cells = a.cells;
        p.noflux = a.noflux;
        p.relax = a.relax;
        p.partials = a.partials;
        p.status = a.status;
        p.co = make_coeffs<T>(a);
        const uint32_t blocks = node_blocks(a.cells);
        if (op == OP_STEP)
            k_step<LAT, S, T, false><<<blocks, kBlock, 0, a.stream>>>(p);
        else if (op == OP_STEP_MASS)
            k_step<LAT, S, T, true><<<blocks, kBlock, 0, a.stream>>>(p);
        else
            k_mass<LAT, S, T><<<blocks, kBlock, 0, a.stream>>>(p);
        return cudaGetLastError();
    }
    FieldParams<T> p;
    p.fprev = static_cast<const T*>(a.fin);
    p.fcur = static_cast<T*>(a.fout);
    p.x_in = static_cast<const T*>(a.field_in);
    p.x_out = static_cast<T*>(a.field_x);
    p.J_out = static_cast<T*>(a.field_J);
    p.nx = a.nx; p.ny = a.ny; p.nz = a.nz;
    p.cells = a.cells;
    p.c0 = a.c0; p.c1 = a.c1; p.stride = a.stride;
    p.noflux = a.noflux;
    p.relax = a.relax;
    p.status = a.status;
    p.co = make_coeffs<T>(a);
    const uint32_t blocks = node_blocks(a.c1 - a.c0);
    if (blocks == 0) return cudaSuccess;
    if (op == OP_INIT)
        k_init<LAT, S, T><<<blocks, kBlock, 0, a.stream>>>(p);
    else
        k_moments<LAT, S, T><<<blocks, kBlock, 0, a.stream>>>(p);
    return cudaGetLastError();
}

template <int LAT, typename T>
cudaError_t dispatch_S(Op op, const KArgs& a)
{
    switch (a.n_species - 1) {
        case 1: return launch<LAT, 1, T>(op, a);
        case 2: return launch<LAT, 2, T>(op, a);
        case 3: return launch<LAT, 3, T>(op, a);
        case 4: return launch<LAT, 4, T>(op, a);
        case 5: return launch<LAT, 5, T>(op, a);
        case 6: return launch<LAT, 6, T>(op, a);
        case 7: return launch<LAT, 7, T>(op, a);
        default: return cudaErrorInvalidValue;
    }
}

template <int LAT>
cudaError_t dispatch_lattice(Op op, int dtype, const KArgs& a)
{
    return dtype == LBMS_F64 ? dispatch_S<LAT, double>(op, a) : dispatch_S<LAT, float>(op, a);
}

}  // namespace lbms
