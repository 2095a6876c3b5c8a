// OMP least squares (Table "s forward block", OMP row: pinv of A(:,Mask)) as
// an incremental float64 Cholesky update, and the residual + stopping test of
// Eq. 2 shared by OMP and CLOMP.  The Cholesky runs one thread per signal so
// that every float64 lane does useful work on a part whose float64 rate is
// low; the residual runs one warp per signal (coalesced column gathers).
#include "k_chol.cuh"
#include "k_resid.cuh"

namespace cs {
namespace {

__global__ void __launch_bounds__(32) k_chol(IterArgs a) {
    pdl_wait();      // no early trigger: the successor launches when this grid completes
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= a.B) return;
    chol_update(a, b);
}


template <int MCH>
__global__ void __launch_bounds__(256) k_resid(IterArgs a) {
    pdl_wait();
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < a.B; b += nwarps)
        resid_one<MCH>(a, b);
    pdl_trigger();
}

}  // namespace

cudaError_t launch_chol(const IterArgs& a, cudaStream_t s) {
    // one warp per CTA spreads the float64 work over as many SMs as possible
    return launch_pdl(k_chol, dim3(ceil_div(a.B, 32)), dim3(32), 0, s, a);
}


template <int MCH>
void launch_resid_m(const IterArgs& a, cudaStream_t s) {
    const int grid = resident_grid((const void*)k_resid<MCH>, 256, ceil_div(a.B, 8));
    launch_pdl(k_resid<MCH>, dim3(grid), dim3(256), 0, s, a);
}

cudaError_t launch_resid(const IterArgs& a, cudaStream_t s) {
    switch (row_chunks(a.mp)) {
        case 1: launch_resid_m<1>(a, s); break;
        case 2: launch_resid_m<2>(a, s); break;
        case 3:
        case 4: launch_resid_m<4>(a, s); break;
        default: launch_resid_m<8>(a, s); break;
    }
    return cudaGetLastError();
}


}  // namespace cs
