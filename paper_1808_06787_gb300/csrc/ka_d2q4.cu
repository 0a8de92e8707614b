// Adjoint kernel instantiations for the D2Q4 lattice (S = 1..4, float and double).
#include "adjoint.cuh"

namespace lbms {

cudaError_t adj_dispatch_d2q4(AdjOp op, int dtype, const AArgs& a)
{
    return adj_dispatch_lattice<LBMS_D2Q4>(op, dtype, a);
}

}  // namespace lbms
