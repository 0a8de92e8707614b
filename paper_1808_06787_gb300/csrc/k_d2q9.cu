// Kernel instantiations for the D2Q9 lattice (all S = 1..7, float and double).
#include "kernels.cuh"

namespace lbms {

cudaError_t dispatch_d2q9(Op op, int dtype, const KArgs& a)
{
    if (slab_step_op(op, a)) return dispatch_halo_d2q9(op, dtype, a);
    return dispatch_lattice<LBMS_D2Q9, false>(op, dtype, a);
}

}  // namespace lbms
