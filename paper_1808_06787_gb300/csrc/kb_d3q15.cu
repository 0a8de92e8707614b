// Batched-solve kernel instantiations for the D3Q15 lattice (S = 1..7, float and double).
#include "batch.cuh"

namespace lbms {

cudaError_t batch_dispatch_d3q15(BatchOp op, int dtype, const BArgs& a)
{
    return batch_dispatch_lattice<LBMS_D3Q15>(op, dtype, a);
}

}  // namespace lbms
