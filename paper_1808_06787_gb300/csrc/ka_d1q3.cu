// Adjoint kernel instantiations for the D1Q3 lattice (S = 1..4, float and double).
#include "adjoint.cuh"

namespace lbms {

cudaError_t adj_dispatch_d1q3(AdjOp op, int dtype, const AArgs& a)
{
    return adj_dispatch_lattice<LBMS_D1Q3>(op, dtype, a);
}

}  // namespace lbms
