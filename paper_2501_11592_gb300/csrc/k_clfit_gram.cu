// CLOMP coefficient fit (Methods, "Coefficients learning on OMP", structure 1):
// T Adam steps on 1/2 ||y - A(s .* Mask)||^2, with the gradient evaluated in
// Gram form G s - b.
#include "k_fit.cuh"

namespace cs {
namespace {

// ------------------------------------------- CLOMP: Gram-form Adam fit -----
template <int KT, int LPS>
__global__ void __launch_bounds__(128) k_clfit_gram(IterArgs a, ClArgs c, int iter) {
    constexpr int P = 32 / LPS;
    __shared__ __align__(16) float sh_s[4][P * KT];
    __shared__ float2 sh_tab[kAdamStaged];
    const float2* tab = stage_adam(c, sh_tab);   // solve constants: safe before the wait
    __syncthreads();
    pdl_wait();
    const int w = threadIdx.x >> 5;
    // warps stride over units of P signals (resident-sized grid)
    const int units = ceil_div(a.B, P);
    for (int u = blockIdx.x * 4 + w; u < units; u += gridDim.x * 4)
        if constexpr (KT <= 32) fit_grid<KT>(a, c, u, c.tau0, sh_s[w], tab);
        else fit_unit<KT, LPS>(a, c, u, c.tau0, sh_s[w], tab);
    pdl_trigger();
}

}  // namespace

cudaError_t launch_clfit_gram(const IterArgs& a, const ClArgs& c, int iter, cudaStream_t s) {
    // every live signal holds exactly `iter` atoms before this fit, so the
    // support after it has iter + 1 <= KT atoms; one signal per warp
    const int kt = round_up(iter + 1, 8);
#define CS_GRAM_LAUNCH(KT_, LPS_)                                                              \
    launch_pdl(k_clfit_gram<KT_, LPS_>,                                                         \
               dim3(resident_grid((const void*)k_clfit_gram<KT_, LPS_>, 128, ceil_div(a.B, 4 * (32 / LPS_)))), \
               dim3(128), 0, s, a, c, iter)
    switch (kt) {
        case 8: CS_GRAM_LAUNCH(8, 32); break;
        case 16: CS_GRAM_LAUNCH(16, 32); break;
        case 24: CS_GRAM_LAUNCH(24, 32); break;
        case 32: CS_GRAM_LAUNCH(32, 32); break;
        case 40: CS_GRAM_LAUNCH(40, 32); break;
        case 48: CS_GRAM_LAUNCH(48, 32); break;
        case 56: CS_GRAM_LAUNCH(56, 32); break;
        default: CS_GRAM_LAUNCH(64, 32); break;
    }
#undef CS_GRAM_LAUNCH
    return cudaGetLastError();
}


}  // namespace cs
