// Internal interface between the host runtime (lbms.cu) and the per-lattice
// kernel translation units (k_d2q5.cu, k_d2q9.cu, k_d3q7.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lbms.h"

namespace lbms {

constexpr int kBlock = 256;  // threads per block of every node kernel

// Kernel selector for the per-lattice dispatchers.
enum Op : int {
    OP_STEP = 0,       // one stream-collide step fin -> fout
    OP_STEP_MASS = 1,  // the same, also writing per-block mass partials
    OP_INIT = 2,       // f+ = w_k xi from a mole-fraction chunk
    OP_MOMENTS = 3,    // xi (and J) of a cell range into a field chunk
    OP_MASS = 4        // per-block mass partials of the current state only
};

// Everything a node kernel may need, dtype-agnostic; the dispatcher converts
// the coefficients to the kernel's type.
struct KArgs {
    const void* fin = nullptr;  // populations read (step: t-1 post-collision; moments: previous buffer or null)
    void* fout = nullptr;       // populations written (step, init) or read (moments, mass: current buffer)
    const void* field_in = nullptr;  // init: mole-fraction chunk [n][stride]
    void* field_x = nullptr;         // moments: mole-fraction chunk [n][stride]
    void* field_J = nullptr;         // moments: flux chunk [n][dim][stride] or null
    void* field_G = nullptr;         // moments: local-gradient chunk [n][dim][stride] or null
    int nx = 1, ny = 1, nz = 1;
    uint32_t cells = 0;
    uint32_t c0 = 0, c1 = 0, stride = 0;  // cell range [c0, c1) and field stride (init, moments)
    uint32_t step_block = kBlock;         // threads per block of the step and mass kernels
    uint32_t noflux = 0;                  // bit f set: face f is no-flux (x-, x+, y-, y+, z-, z+)
    uint32_t dirichlet = 0;               // bit f set: face f is Dirichlet (fixed composition)
    const void* xb = nullptr;             // Dirichlet compositions [6][S] in the solver's dtype
    uint32_t halo = 0;                    // bit f set: face f is a slab cut (faces of the split axis)
    uint32_t plane = 1;                   // nodes per layer of the split axis
    uint32_t origin = 0;                  // global index of node 0 (slab offset; rounding key)
    const void* halo_recv[2] = {nullptr, nullptr};  // receive buffers (low, high face) of the read parity
    void* halo_send[2] = {nullptr, nullptr};        // send buffers (low, high face)
    int relax = LBMS_RELAX_MAGIC;
    int n_species = 2;
    double invD[LBMS_MAX_SPECIES][LBMS_MAX_SPECIES] = {};  // 1 / D_ij
    double xref[LBMS_MAX_SPECIES] = {};                    // reference composition (frozen mode)
    void* partials = nullptr;  // [blocks][n]: int64 fixed point (FP32) or double2 (FP64)
    int fixed_shift = 32;      // fraction bits of the FP32 fixed-point mass partials
    uint32_t* status = nullptr;
    const uint32_t* clock_in = nullptr;  // step counter read by a step
    uint32_t* clock_out = nullptr;       // step counter written by a step
    int reverse = 0;                     // step: blocks take the grid from its end
    cudaStream_t stream = nullptr;
};

// Per-lattice dispatchers: launch `op` for S = n_species - 1 and dtype.
// Return cudaSuccess or the launch error.
cudaError_t dispatch_d2q5(Op op, int dtype, const KArgs& a);
cudaError_t dispatch_d2q9(Op op, int dtype, const KArgs& a);
cudaError_t dispatch_d3q7(Op op, int dtype, const KArgs& a);
cudaError_t dispatch_d3q15(Op op, int dtype, const KArgs& a);
cudaError_t dispatch_d1q3(Op op, int dtype, const KArgs& a);
cudaError_t dispatch_d2q4(Op op, int dtype, const KArgs& a);
cudaError_t dispatch_d3q6(Op op, int dtype, const KArgs& a);
// The step kernels of slabs (cut faces), one translation unit per lattice
// (kh_*.cu); the dispatchers above forward to them.
cudaError_t dispatch_halo_d2q5(Op op, int dtype, const KArgs& a);
cudaError_t dispatch_halo_d2q9(Op op, int dtype, const KArgs& a);
cudaError_t dispatch_halo_d3q7(Op op, int dtype, const KArgs& a);
cudaError_t dispatch_halo_d3q15(Op op, int dtype, const KArgs& a);
cudaError_t dispatch_halo_d1q3(Op op, int dtype, const KArgs& a);
cudaError_t dispatch_halo_d2q4(Op op, int dtype, const KArgs& a);
cudaError_t dispatch_halo_d3q6(Op op, int dtype, const KArgs& a);

// Number of blocks a node kernel over `cells` nodes is launched with.
inline uint32_t node_blocks(uint32_t cells) { return (cells + kBlock - 1) / kBlock; }

// Threads per block of a solver's step and mass kernels: grids too small to give
// every SM of the device two blocks of kBlock threads run blocks of 64, so that
// the per-node work (FP64 in particular, whose pipes are narrow on GB300) is
// spread over all SMs instead of a few.  `sms` is the device's multiprocessor
// count (device_sm_count).
constexpr uint32_t kSmallBlock = 64;
inline uint32_t step_block_for(uint32_t cells, int sms)
{
    return (uint64_t)cells < 2ull * (uint64_t)sms * kBlock ? kSmallBlock : kBlock;
}
inline uint32_t step_blocks(uint32_t cells, int sms)
{
    const uint32_t tb = step_block_for(cells, sms);
    return (cells + tb - 1) / tb;
}

// Multiprocessor count of the current device (cudaDevAttrMultiProcessorCount),
// looked up once per device and clamped to kMaxSms.
constexpr int kMaxSms = 8192;
cudaError_t device_sm_count(int* sms);

// Mass-partial slots a workspace reserves for a grid: enough for the block
// partition of step_blocks on any device of up to kMaxSms SMs, so that
// workspace sizes do not depend on the device they are computed on.
inline uint32_t partial_slots(uint32_t cells)
{
    return (uint64_t)cells < 2ull * kMaxSms * kBlock ? (cells + kSmallBlock - 1) / kSmallBlock
                                                    : (cells + kBlock - 1) / kBlock;
}

// True if the runtime reports p as device (or managed) memory of this process.
bool is_device_ptr(const void* p);

// The address under which kernels read and write pinned host memory (with
// unified addressing every pinned allocation is mapped into the device's
// address space), or null for pageable host memory and for device memory.
// Kernels then move host fields directly over the host link, without staging
// copies.
void* pinned_alias(const void* p);

// Helpers of the host runtime shared with lbms_mass_noalloc (mass_noalloc.cu):
// fraction bits of the FP32 fixed-point mass partials for a grid, the final
// reduction of per-block partials into n doubles, and the thread's message for
// lbms_last_error(NULL).
int mass_fixed_shift(uint32_t cells);
cudaError_t launch_mass_reduce(int dtype, const void* partials, uint32_t blocks, int n, int shift,
                               double* out, cudaStream_t stream);
int set_call_error(int code, const char* fmt, ...);

}  // namespace lbms
