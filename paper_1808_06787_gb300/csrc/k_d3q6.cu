// Kernel instantiations for the D3Q6 lattice (all S = 1..7, float and double).
#include "kernels.cuh"

namespace lbms {

cudaError_t dispatch_d3q6(Op op, int dtype, const KArgs& a)
{
    if (slab_step_op(op, a)) return dispatch_halo_d3q6(op, dtype, a);
    return dispatch_lattice<LBMS_D3Q6, false>(op, dtype, a);
}

}  // namespace lbms
