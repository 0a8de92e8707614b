// Kernel instantiations for the D2Q5 lattice (all S = 1..7, float and double).
#include "kernels.cuh"

namespace lbms {

cudaError_t dispatch_d2q5(Op op, int dtype, const KArgs& a)
{
    if (slab_step_op(op, a)) return dispatch_halo_d2q5(op, dtype, a);
    return dispatch_lattice<LBMS_D2Q5, false>(op, dtype, a);
}

}  // namespace lbms
