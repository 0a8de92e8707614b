// Kernel instantiations for the D1Q3 lattice (all S = 1..7, float and double).
#include "kernels.cuh"

namespace lbms {

cudaError_t dispatch_d1q3(Op op, int dtype, const KArgs& a)
{
    if (slab_step_op(op, a)) return dispatch_halo_d1q3(op, dtype, a);
    return dispatch_lattice<LBMS_D1Q3, false>(op, dtype, a);
}

}  // namespace lbms
