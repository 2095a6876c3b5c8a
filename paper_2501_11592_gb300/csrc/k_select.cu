// Selection step of one OMP / CLOMP iteration (Methods, "Coefficients learning
// on OMP": the position of the largest |A^T r| among unselected atoms is OR-ed
// into the mask), plus the Gram column of the new atom for the fit.  One warp
// per signal.
#include "k_select.cuh"

namespace cs {
namespace {

// One warp per signal, striding over the batch (the grid is sized to the
// resident capacity of the GPU, so no partial last wave).
template <int MCH>
__global__ void __launch_bounds__(256) k_select(IterArgs a) {
    pdl_wait();
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < a.B; b += nwarps)
        select_one<MCH>(a, b);
    pdl_trigger();   // after the work: the successor only overlaps our tail
}

}  // namespace

template <int MCH>
void launch_select_m(const IterArgs& a, cudaStream_t s) {
    const int grid = resident_grid((const void*)k_select<MCH>, 256, ceil_div(a.B, 8));
    launch_pdl(k_select<MCH>, dim3(grid), dim3(256), 0, s, a);
}

cudaError_t launch_select(const IterArgs& a, cudaStream_t s) {
    switch (row_chunks(a.mp)) {
        case 1: launch_select_m<1>(a, s); break;
        case 2: launch_select_m<2>(a, s); break;
        case 3:
        case 4: launch_select_m<4>(a, s); break;
        default: launch_select_m<8>(a, s); break;
    }
    return cudaGetLastError();
}

}  // namespace cs
