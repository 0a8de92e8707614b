// lbms_mass_noalloc: species totals of a population field for callers that
// cannot allocate device memory.
//
// Some callers of this library may not call cudaMalloc at all: real-time or
// embedded loops whose device memory is fixed at start-up (an allocation can
// block for an unbounded time or fail), plug-ins inside host frameworks whose
// device memory belongs to the framework's own pool, and monitoring code that
// inspects a buffer someone else owns without a solver handle.  lbms_mass needs
// a solver handle and its caller-provided workspace; this entry point needs
// neither.  Its scratch (one partial sum per block and species) lives in the
// file-scope device array below, which every GPU that loads the library holds
// until the process exits.
//
// The array's device address is looked up once per device and cached for the
// life of the process, so resetting a device (cudaDeviceReset) while the
// library stays loaded is not supported by this entry point.
#include <mutex>

#include "lbms_internal.h"

namespace {

// 4 MiB of scratch: per-block partials (8 bytes per block and species for F32
// solvers, 16 for F64) followed by a 256-byte slot for results bound for host
// memory.
constexpr size_t kScratchBytes = size_t(4) << 20;
constexpr size_t kResultBytes = 256;
constexpr size_t kPartialBytes = kScratchBytes - kResultBytes;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_mass_scratch[kScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device with that device current.
int scratch_on_current_device(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return lbms::set_call_error(LBMS_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return lbms::set_call_error(LBMS_EINVAL, "device %d is beyond the %d supported", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_mass_scratch);
        if (e != cudaSuccess)
            return lbms::set_call_error(LBMS_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return LBMS_OK;
}

}  // namespace

extern "C" int lbms_mass_noalloc(int lattice, int n_species, const int grid[3], int dtype,
                                 const void* populations, double* mass_out, void* cuda_stream)
{
    using namespace lbms;
    set_call_error(LBMS_OK, "");
    if (lbms_workspace_size(lattice, n_species, grid, dtype) == 0)
        return set_call_error(LBMS_EINVAL, "invalid lattice/species/grid/dtype combination");
    if (!populations || !mass_out) return set_call_error(LBMS_EINVAL, "populations and mass_out must not be NULL");
    const uint32_t cells = (uint32_t)((size_t)grid[0] * grid[1] * grid[2]);
    const size_t record = dtype == LBMS_F64 ? 16 : 8;
    // grids whose partials cannot fit even with the coarsest block partition are
    // refused before anything touches the device
    if ((size_t)node_blocks(cells) * n_species * record > kPartialBytes)
        return set_call_error(LBMS_EINVAL,
                              "grid too large for lbms_mass_noalloc: %u nodes x %d species need more "
                              "than the %zu bytes of static scratch (use lbms_mass with a workspace)",
                              cells, n_species, kPartialBytes);
    // the kernel reads populations on the device: a host pointer is refused
    // before any launch
    if (!is_device_ptr(populations))
        return set_call_error(LBMS_EINVAL, "populations must be device memory");
    int sms = 0;
    cudaError_t e = device_sm_count(&sms);
    if (e != cudaSuccess) return set_call_error(LBMS_ECUDA, "device query: %s", cudaGetErrorString(e));
    // the block partition of a solver's own mass kernel, so that both entry
    // points run the same reduction (the FP64 compensated sums depend on it)
    const uint32_t blocks = step_blocks(cells, sms);
    const size_t need = (size_t)blocks * n_species * record;
    if (need > kPartialBytes)
        return set_call_error(LBMS_EINVAL,
                              "grid too large for lbms_mass_noalloc: %u nodes x %d species need %zu bytes of "
                              "scratch, the static area holds %zu (use lbms_mass with a workspace)",
                              cells, n_species, need, kPartialBytes);
    void* scratch = nullptr;
    int rc = scratch_on_current_device(&scratch);
    if (rc != LBMS_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    KArgs a;
    a.nx = grid[0]; a.ny = grid[1]; a.nz = grid[2];
    a.cells = cells;
    a.step_block = step_block_for(cells, sms);
    a.n_species = n_species;
    a.fout = const_cast<void*>(populations);  // read only by the mass kernel
    a.partials = scratch;
    a.fixed_shift = mass_fixed_shift(cells);
    a.stream = st;
    e = lattice == LBMS_D2Q5    ? dispatch_d2q5(OP_MASS, dtype, a)
        : lattice == LBMS_D2Q9  ? dispatch_d2q9(OP_MASS, dtype, a)
        : lattice == LBMS_D3Q7  ? dispatch_d3q7(OP_MASS, dtype, a)
        : lattice == LBMS_D3Q15 ? dispatch_d3q15(OP_MASS, dtype, a)
        : lattice == LBMS_D1Q3  ? dispatch_d1q3(OP_MASS, dtype, a)
        : lattice == LBMS_D2Q4  ? dispatch_d2q4(OP_MASS, dtype, a)
                                : dispatch_d3q6(OP_MASS, dtype, a);
    if (e != cudaSuccess) return set_call_error(LBMS_ECUDA, "mass kernel: %s", cudaGetErrorString(e));
    const bool host_out = !is_device_ptr(mass_out);
    double* dst = host_out ? reinterpret_cast<double*>(static_cast<char*>(scratch) + kPartialBytes) : mass_out;
    e = launch_mass_reduce(dtype, scratch, blocks, n_species, a.fixed_shift, dst, st);
    if (e != cudaSuccess) return set_call_error(LBMS_ECUDA, "mass reduction: %s", cudaGetErrorString(e));
    if (host_out) {
        e = cudaMemcpyAsync(mass_out, dst, sizeof(double) * n_species, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return set_call_error(LBMS_ECUDA, "copy to host: %s", cudaGetErrorString(e));
    }
    return LBMS_OK;
}
