// Batched-solve kernel instantiations for the D2Q5 lattice (S = 1..7, float and double).
#include "batch.cuh"

namespace lbms {

cudaError_t batch_dispatch_d2q5(BatchOp op, int dtype, const BArgs& a)
{
    return batch_dispatch_lattice<LBMS_D2Q5>(op, dtype, a);
}

}  // namespace lbms
