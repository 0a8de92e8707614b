// Batched-solve kernel instantiations for the D2Q4 lattice (S = 1..7, float and double).
#include "batch.cuh"

namespace lbms {

cudaError_t batch_dispatch_d2q4(BatchOp op, int dtype, const BArgs& a)
{
    return batch_dispatch_lattice<LBMS_D2Q4>(op, dtype, a);
}

}  // namespace lbms
