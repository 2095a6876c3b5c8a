// OMP least squares (Table "s forward block", OMP row: pinv of A(:,Mask)) as
// an incremental float64 Cholesky update, and the residual + stopping test of
// Eq. 2 shared by OMP and CLOMP.  Both run one warp per signal: the Cholesky
// update as two matrix-vector products over the lanes (k_chol.cuh), the
// residual with coalesced column gathers.
#include "k_chol.cuh"
#include "k_resid.cuh"

namespace cs {
namespace {

template <int NP>
__global__ void __launch_bounds__(256) k_chol(IterArgs a) {
    pdl_wait();      // no early trigger: the successor launches when this grid completes
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < a.B; b += nwarps)
        chol_update<NP>(a, b);
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
    if (a.kmax == 32) {
        const int grid = resident_grid((const void*)k_chol<1>, 256, ceil_div(a.B, 8));
        return launch_pdl(k_chol<1>, dim3(grid), dim3(256), 0, s, a);
    }
    const int grid = resident_grid((const void*)k_chol<2>, 256, ceil_div(a.B, 8));
    return launch_pdl(k_chol<2>, dim3(grid), dim3(256), 0, s, a);
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
