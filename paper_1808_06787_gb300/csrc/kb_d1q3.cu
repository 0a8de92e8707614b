// Batched-solve kernel instantiations for the D1Q3 lattice (S = 1..7, float and double).
#include "batch.cuh"

namespace lbms {

cudaError_t batch_dispatch_d1q3(BatchOp op, int dtype, const BArgs& a)
{
    return batch_dispatch_lattice<LBMS_D1Q3>(op, dtype, a);
}

}  // namespace lbms
