// Adjoint kernel instantiations for the D3Q6 lattice (S = 1..4, float and double).
#include "adjoint.cuh"

namespace lbms {

cudaError_t adj_dispatch_d3q6(AdjOp op, int dtype, const AArgs& a)
{
    return adj_dispatch_lattice<LBMS_D3Q6>(op, dtype, a);
}

}  // namespace lbms
