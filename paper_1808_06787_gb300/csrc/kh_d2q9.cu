// Step kernels of slabs (grids with cut faces) for the D2Q9 lattice (all S = 1..7,
// float and double).
#include "kernels.cuh"

namespace lbms {

cudaError_t dispatch_halo_d2q9(Op op, int dtype, const KArgs& a)
{
    return dispatch_lattice<LBMS_D2Q9, true>(op, dtype, a);
}

}  // namespace lbms
