// Batched solves: many independent grids (each with its own size, faces and
// diffusivities) in one node space.  Instance i owns the global nodes
// [base_i, base_i + cells_i), with base_i a multiple of the block size, so
// every block belongs to exactly one instance; populations are
// f[(s * Q + k) * total_nodes + node].  Each instance runs the same per-node
// arithmetic as a single solve (same gather, solve, collision and
// stochastic-rounding key from its local node index and its own step
// counter), so a batched instance equals the single solve of that grid bit
// for bit.
#pragma once

#include "kernels.cuh"

namespace lbms {

// Per-instance descriptor (device).
struct BatchInst {
    Geom g;           // the instance's own grid and faces; g.cells = its node count
    uint32_t base;    // first global node (multiple of kBlock)
    uint32_t block0;  // first global block
    uint32_t nblocks;
    uint32_t pad;
};

enum BatchOp : int { BOP_STEP = 0, BOP_STEP_MASS = 1, BOP_INIT = 2, BOP_MOMENTS = 3, BOP_MASS = 4 };

// Everything a batched kernel may need, dtype-agnostic.
struct BArgs {
    const void* fin = nullptr;  // populations read (steps: t-1; moments: previous buffer or null)
    void* fout = nullptr;       // populations written (steps, init) or read (moments, mass)
    uint32_t total_nodes = 0;   // plane stride of the population buffers
    uint32_t block_begin = 0, block_end = 0;  // global block range of this launch
    const uint32_t* blk_inst = nullptr;       // [total_blocks] instance of each block
    const BatchInst* inst = nullptr;          // [count]
    const void* invD = nullptr;               // [count][n][n] 1/(2 D_ij), element type
    int n_species = 2;
    int relax = LBMS_RELAX_MAGIC;
    uint32_t* clock = nullptr;                // [count][2] step counters
    int parity = 0;                           // counter word read (= index of fin)
    int reverse = 0;                          // steps: blocks taken from the end of the range
    void* partials = nullptr;                 // [total_blocks][n]
    int fixed_shift = 32;
    uint32_t* status = nullptr;
    const void* field_in = nullptr;           // init: mole fractions
    void* field_x = nullptr;                  // moments: mole fractions
    void* field_J = nullptr;                  // moments: fluxes or null
    const long long* field_off = nullptr;     // [count] element offset of instance i's x block
    int nodes_per_thread = 1;                 // plain steps: 1 or 2 (k_batch_step_pair)
    const void* xb = nullptr;                 // [count][6][S] Dirichlet compositions
    bool dirichlet = false;                   // some instance has a Dirichlet face
    cudaStream_t stream = nullptr;
};

template <typename T>
struct InvDView {
    const T* p;
    int n;
    __device__ __forceinline__ const T* operator[](int i) const { return p + i * n; }
};

template <typename T>
struct BatchParams {
    const T* __restrict__ fin;
    T* __restrict__ fout;
    uint32_t total_nodes;
    uint32_t block_begin;
    const uint32_t* __restrict__ blk_inst;
    const BatchInst* __restrict__ inst;
    const T* __restrict__ invD;
    int relax;
    uint32_t* clock;
    int parity;
    int reverse;  // steps: blocks taken from the end of the launch's range (grid_block)
    MassOut mass;  // partials pointer already offset to block_begin
    uint32_t* status;
    const T* x_in;
    T* x_out;
    T* J_out;
    const long long* field_off;
};

// DIR: some instance of the batch has Dirichlet faces (kernels of batches
// without any are compiled without the anti-bounce-back code).
// The Dirichlet compositions xb ([count][6][S]) are an argument of their own:
// inside the parameter structure the extra member changed the register
// allocation of the kernels that do not use it.
template <int LAT, int S, typename T, bool MASS, bool DIR>
__global__ void __launch_bounds__(kBlock) k_batch_step(BatchParams<T> p, const T* __restrict__ xb)
{
    using L = Lattice<LAT>;
    constexpr int Q = L::Q;
    const uint32_t lb = grid_block(p.reverse);  // alternate steps take the blocks from the end
    const uint32_t blk = p.block_begin + lb;
    const uint32_t id = p.blk_inst[blk];
    const BatchInst d = p.inst[id];
    const uint32_t local = (blk - d.block0) * kBlock + threadIdx.x;
    const bool active = local < d.g.cells;
    uint32_t* clk = p.clock + 2 * id;
    const uint32_t step = clk[p.parity];
    if (blk == d.block0 && threadIdx.x == 0) clk[1 - p.parity] = step + 1;
    T xi[S + 1];
    if (active) {
        const Neighbourhood h = neighbourhood<Lattice<LAT>::DIM, false>(d.g, local);
        Geom plane = d.g;
        plane.cells = p.total_nodes;  // the gather's plane stride
        const uint32_t cell = d.base + local;
        T f[S][Q];
        pull<LAT, S, T>(p.fin, plane, cell, h, f, DIR ? xb + (size_t)id * 6 * S : static_cast<const T*>(nullptr));
        mole_fractions<LAT, S, T>(f, xi);
        if (MASS) check_range<S, T>(xi, p.status);  // once per step call
        const InvDView<T> iv{p.invD + (size_t)id * (S + 1) * (S + 1), S + 1};
        T L1[S][S], L2[S][S];
        relaxation_matrices<S, T>(xi, iv, T(1.0 / L::cs2()), p.relax, L1, L2);
        collide<LAT, S, T>(f, xi, L1, L2, mix32(step * 0x9e3779b9u) ^ (local * 0x27d4eb2du));
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int k = 0; k < Q; ++k) p.fout[(size_t)(s * Q + k) * p.total_nodes + cell] = f[s][k];
    }
    if (MASS) write_mass_partials<S>(xi, active, p.mass, lb);
}

// Two nodes per thread, as k_step_pair: blocks of kBlock / 2 threads cover one
// kBlock-node block of one instance; the pair's rest populations come in one
// load and every plane goes out in one store.  Instance sizes may be odd: the
// thread whose pair ends an odd instance takes its one node alone.
// 12 blocks of kBlock / 2 threads per SM (40 registers; on ternary D2Q5 with a
// 16-byte spill, which still measured 3 % faster than 10 blocks at 48 registers:
// the instance lookup at the start of every block leaves a latency that more
// resident blocks hide).  MASS: the last step of a call, which also tests the
// range and writes the block's mass partials (the 256-node blocks of
// k_batch_step, so the same integers).
template <int LAT, int S, typename T, bool DIR, bool MASS>
__global__ void __launch_bounds__(kBlock / 2, 12)
    k_batch_step_pair(BatchParams<T> p, const T* __restrict__ xb)
{
    using L = Lattice<LAT>;
    using V = typename Pair<T>::type;
    constexpr int Q = L::Q;
    constexpr bool REST = L::K0 == 1;  // lattices without a rest velocity gather every population
    const uint32_t lb = grid_block(p.reverse);
    const uint32_t blk = p.block_begin + lb;
    const uint32_t id = p.blk_inst[blk];
    const BatchInst d = p.inst[id];
    const uint32_t local0 = (blk - d.block0) * kBlock + 2 * threadIdx.x;
    uint32_t* clk = p.clock + 2 * id;
    const uint32_t step = clk[p.parity];
    if (blk == d.block0 && threadIdx.x == 0) clk[1 - p.parity] = step + 1;
    const bool active = local0 < d.g.cells;
    if (!MASS && !active) return;
    T xs[2][S + 1];  // MASS: the pair's mole fractions, zero where it has no node
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int s = 0; s <= S; ++s) xs[j][s] = T(0);
    if (active) {
        const bool both = local0 + 1 < d.g.cells;
        Geom plane = d.g;
        plane.cells = p.total_nodes;  // the gather's plane stride
        const uint32_t c0 = d.base + local0;
        const InvDView<T> iv{p.invD + (size_t)id * (S + 1) * (S + 1), S + 1};
        const uint32_t hk = mix32(step * 0x9e3779b9u);
        T f[2][S][Q];
        if constexpr (REST) {
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const V r = *reinterpret_cast<const V*>(p.fin + (size_t)(s * Q) * p.total_nodes + c0);
                f[0][s][0] = r.x;
                f[1][s][0] = r.y;
            }
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            if (j == 1 && !both) break;
            const uint32_t local = local0 + j;
            const Neighbourhood h = neighbourhood<Lattice<LAT>::DIM, false>(d.g, local);
            pull<LAT, S, T, REST>(p.fin, plane, c0 + j, h, f[j],
                                  DIR ? xb + (size_t)id * 6 * S : static_cast<const T*>(nullptr));
            T xi[S + 1];
            mole_fractions<LAT, S, T>(f[j], xi);
            if (MASS) {
                check_range<S, T>(xi, p.status);
#pragma unroll
                for (int s = 0; s <= S; ++s) xs[j][s] = xi[s];
            }
            T L1[S][S], L2[S][S];
            relaxation_matrices<S, T>(xi, iv, T(1.0 / L::cs2()), p.relax, L1, L2);
            collide<LAT, S, T>(f[j], xi, L1, L2, hk ^ (local * 0x27d4eb2du));
        }
        if (both) {
#pragma unroll
            for (int s = 0; s < S; ++s)
#pragma unroll
                for (int k = 0; k < Q; ++k) {
                    V v;
                    v.x = f[0][s][k];
                    v.y = f[1][s][k];
                    *reinterpret_cast<V*>(p.fout + (size_t)(s * Q + k) * p.total_nodes + c0) = v;
                }
        } else {
#pragma unroll
            for (int s = 0; s < S; ++s)
#pragma unroll
                for (int k = 0; k < Q; ++k) p.fout[(size_t)(s * Q + k) * p.total_nodes + c0] = f[0][s][k];
        }
    }
    if constexpr (MASS) write_mass_partials_pair<S>(xs, active, p.mass, lb);
}

// Batches take the two-nodes-per-thread shape on the lattices with Q <= 5 (the
// batched 3D lattices keep one node per thread).
template <int LAT, int S, typename T>
constexpr bool batch_pair_lattice()
{
    return Lattice<LAT>::Q <= 5 && S <= 2 && sizeof(T) == 4;
}

template <int LAT, int S, typename T>
__global__ void __launch_bounds__(kBlock) k_batch_mass(BatchParams<T> p)
{
    constexpr int Q = Lattice<LAT>::Q;
    const uint32_t blk = p.block_begin + blockIdx.x;
    const BatchInst d = p.inst[p.blk_inst[blk]];
    const uint32_t local = (blk - d.block0) * kBlock + threadIdx.x;
    const bool active = local < d.g.cells;
    T xi[S + 1];
    if (active) {
        const uint32_t cell = d.base + local;
        T f[S][Q];
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int k = 0; k < Q; ++k) f[s][k] = p.fout[(size_t)(s * Q + k) * p.total_nodes + cell];
        mole_fractions<LAT, S, T>(f, xi);
    }
    write_mass_partials<S>(xi, active, p.mass, blockIdx.x);
}

// f+ = w_k xi at t = 0 for each instance, from its [n][cells] block of x_in.
template <int LAT, int S, typename T>
__global__ void __launch_bounds__(kBlock) k_batch_init(BatchParams<T> p)
{
    using L = Lattice<LAT>;
    constexpr int Q = L::Q;
    const uint32_t blk = p.block_begin + blockIdx.x;
    const uint32_t id = p.blk_inst[blk];
    const BatchInst d = p.inst[id];
    const uint32_t local = (blk - d.block0) * kBlock + threadIdx.x;
    if (local >= d.g.cells) return;
    const T* src = p.x_in + p.field_off[id];
    T xi[S + 1];
    double sum = 0.0;
    bool finite = true;
#pragma unroll
    for (int s = 0; s <= S; ++s) {
        xi[s] = src[(size_t)s * d.g.cells + local];
        sum += (double)xi[s];
        finite &= (bool)isfinite((double)xi[s]);
    }
    if (!finite || !(fabs(sum - 1.0) <= 1e-5)) atomicOr(p.status, LBMS_FLAG_INIT);
    const uint32_t cell = d.base + local;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        T moving = T(0);
#pragma unroll
        for (int k = 1; k < Q; ++k) {
            const T fk = T(L::w(k)) * xi[s];
            moving += fk;
            p.fout[(size_t)(s * Q + k) * p.total_nodes + cell] = fk;
        }
        p.fout[(size_t)(s * Q) * p.total_nodes + cell] = xi[s] - moving;
    }
}

// Mole fractions (and fluxes) of every instance into its blocks of x_out (and
// J_out, whose instance block starts at dim * field_off).
template <int LAT, int S, typename T>
__global__ void __launch_bounds__(kBlock) k_batch_moments(BatchParams<T> p, const T* __restrict__ xb)
{
    using L = Lattice<LAT>;
    constexpr int Q = L::Q;
    constexpr int DIM = L::DIM;
    const uint32_t blk = p.block_begin + blockIdx.x;
    const uint32_t id = p.blk_inst[blk];
    const BatchInst d = p.inst[id];
    const uint32_t local = (blk - d.block0) * kBlock + threadIdx.x;
    if (local >= d.g.cells) return;
    const uint32_t cell = d.base + local;
    const size_t cells = d.g.cells;
    {
        T f[S][Q];
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int k = 0; k < Q; ++k) f[s][k] = p.fout[(size_t)(s * Q + k) * p.total_nodes + cell];
        T xi[S + 1];
        mole_fractions<LAT, S, T>(f, xi);
        T* xo = p.x_out + p.field_off[id];
#pragma unroll
        for (int s = 0; s <= S; ++s) xo[(size_t)s * cells + local] = xi[s];
    }
    if (!p.J_out) return;
    T J[S + 1][DIM], G[S + 1][DIM];
#pragma unroll
    for (int s = 0; s <= S; ++s)
#pragma unroll
        for (int a = 0; a < DIM; ++a) J[s][a] = T(0);
    if (p.fin) {
        const Neighbourhood h = neighbourhood<Lattice<LAT>::DIM, false>(d.g, local);
        Geom plane = d.g;
        plane.cells = p.total_nodes;
        T f[S][Q];
        pull<LAT, S, T>(p.fin, plane, cell, h, f, xb + (size_t)id * 6 * S);
        T xi[S + 1];
        mole_fractions<LAT, S, T>(f, xi);
        const InvDView<T> iv{p.invD + (size_t)id * (S + 1) * (S + 1), S + 1};
        T L1[S][S], L2[S][S];
        relaxation_matrices<S, T>(xi, iv, T(1.0 / L::cs2()), p.relax, L1, L2);
        flux_and_gradient<LAT, S, T>(f, L1, J, G);
    }
    T* Jo = p.J_out + (size_t)DIM * p.field_off[id];
#pragma unroll
    for (int s = 0; s <= S; ++s)
#pragma unroll
        for (int a = 0; a < DIM; ++a) Jo[((size_t)s * DIM + a) * cells + local] = J[s][a];
}

template <int LAT, int S, typename T>
cudaError_t batch_launch(BatchOp op, const BArgs& a)
{
    BatchParams<T> p;
    p.fin = static_cast<const T*>(a.fin);
    p.fout = static_cast<T*>(a.fout);
    p.total_nodes = a.total_nodes;
    p.block_begin = a.block_begin;
    p.blk_inst = a.blk_inst;
    p.inst = a.inst;
    p.invD = static_cast<const T*>(a.invD);
    p.relax = a.relax;
    p.clock = a.clock;
    p.parity = a.parity;
    p.reverse = a.reverse;
    const size_t rec = sizeof(T) == 8 ? sizeof(double2) : sizeof(long long);
    p.mass.partials = a.partials ? static_cast<char*>(a.partials) + (size_t)a.block_begin * (S + 1) * rec
                                 : nullptr;
    p.mass.shift = a.fixed_shift;
    p.status = a.status;
    p.x_in = static_cast<const T*>(a.field_in);
    p.x_out = static_cast<T*>(a.field_x);
    p.J_out = static_cast<T*>(a.field_J);
    p.field_off = a.field_off;
    const T* xb = static_cast<const T*>(a.xb);
    const uint32_t blocks = a.block_end - a.block_begin;
    if (blocks == 0) return cudaSuccess;
    switch (op) {
        case BOP_STEP:
            if constexpr (batch_pair_lattice<LAT, S, T>()) {
                if (a.nodes_per_thread == 2) {
                    if (a.dirichlet)
                        k_batch_step_pair<LAT, S, T, true, false><<<blocks, kBlock / 2, 0, a.stream>>>(p, xb);
                    else
                        k_batch_step_pair<LAT, S, T, false, false><<<blocks, kBlock / 2, 0, a.stream>>>(p, nullptr);
                    break;
                }
            }
            if (a.dirichlet)
                k_batch_step<LAT, S, T, false, true><<<blocks, kBlock, 0, a.stream>>>(p, xb);
            else
                k_batch_step<LAT, S, T, false, false><<<blocks, kBlock, 0, a.stream>>>(p, nullptr);
            break;
        case BOP_STEP_MASS:
            if constexpr (batch_pair_lattice<LAT, S, T>()) {
                if (a.nodes_per_thread == 2) {
                    if (a.dirichlet)
                        k_batch_step_pair<LAT, S, T, true, true><<<blocks, kBlock / 2, 0, a.stream>>>(p, xb);
                    else
                        k_batch_step_pair<LAT, S, T, false, true><<<blocks, kBlock / 2, 0, a.stream>>>(p, nullptr);
                    break;
                }
            }
            if (a.dirichlet)
                k_batch_step<LAT, S, T, true, true><<<blocks, kBlock, 0, a.stream>>>(p, xb);
            else
                k_batch_step<LAT, S, T, true, false><<<blocks, kBlock, 0, a.stream>>>(p, nullptr);
            break;
        case BOP_INIT: k_batch_init<LAT, S, T><<<blocks, kBlock, 0, a.stream>>>(p); break;
        case BOP_MOMENTS: k_batch_moments<LAT, S, T><<<blocks, kBlock, 0, a.stream>>>(p, xb); break;
        default: k_batch_mass<LAT, S, T><<<blocks, kBlock, 0, a.stream>>>(p); break;
    }
    return cudaGetLastError();
}

template <int LAT, typename T>
cudaError_t batch_dispatch_S(BatchOp op, const BArgs& a)
{
    switch (a.n_species - 1) {
        case 1: return batch_launch<LAT, 1, T>(op, a);
        case 2: return batch_launch<LAT, 2, T>(op, a);
        case 3: return batch_launch<LAT, 3, T>(op, a);
        case 4: return batch_launch<LAT, 4, T>(op, a);
        case 5: return batch_launch<LAT, 5, T>(op, a);
        case 6: return batch_launch<LAT, 6, T>(op, a);
        case 7: return batch_launch<LAT, 7, T>(op, a);
        default: return cudaErrorInvalidValue;
    }
}

template <int LAT>
cudaError_t batch_dispatch_lattice(BatchOp op, int dtype, const BArgs& a)
{
    return dtype == LBMS_F64 ? batch_dispatch_S<LAT, double>(op, a) : batch_dispatch_S<LAT, float>(op, a);
}

cudaError_t batch_dispatch_d2q5(BatchOp op, int dtype, const BArgs& a);
cudaError_t batch_dispatch_d2q9(BatchOp op, int dtype, const BArgs& a);
cudaError_t batch_dispatch_d3q7(BatchOp op, int dtype, const BArgs& a);
cudaError_t batch_dispatch_d3q15(BatchOp op, int dtype, const BArgs& a);
cudaError_t batch_dispatch_d1q3(BatchOp op, int dtype, const BArgs& a);
cudaError_t batch_dispatch_d2q4(BatchOp op, int dtype, const BArgs& a);
cudaError_t batch_dispatch_d3q6(BatchOp op, int dtype, const BArgs& a);

}  // namespace lbms
