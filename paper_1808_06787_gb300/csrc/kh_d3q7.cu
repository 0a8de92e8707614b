// Step kernels of slabs (grids with cut faces) for the D3Q7 lattice (all S = 1..7,
// float and double).
#include "kernels.cuh"

namespace lbms {

cudaError_t dispatch_halo_d3q7(Op op, int dtype, const KArgs& a)
{
    return dispatch_lattice<LBMS_D3Q7, true>(op, dtype, a);
}

}  // namespace lbms
