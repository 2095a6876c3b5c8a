// Fused per-iteration update of CLOMP in Gram form: selection, Adam fit and
// residual of one iteration (Methods, "Coefficients learning on OMP") in one
// launch.  One warp per signal: it selects the new atom, runs the Adam fit
// (lane q owns coordinate q), then forms the residual.  (Packing several
// small-support signals into one warp, as the stand-alone fit does, would
// serialise their selection and residual steps.)  Fusing removes
// two kernel boundaries per iteration -- the ramp-up and tail of the
// stand-alone kernels -- and re-reads nothing between the three steps but
// the few values one lane hands to another.
#include "k_fit.cuh"
#include "k_resid.cuh"
#include "k_select.cuh"

namespace cs {
namespace {

template <int MCH, int KT, int LPS>
__global__ void __launch_bounds__(128) k_update_clomp(IterArgs a, ClArgs c, int iter) {
    constexpr int P = 32 / LPS;
    __shared__ __align__(16) float sh_s[4][P * KT];
    __shared__ float2 sh_tab[kAdamStaged];
    const float2* tab = stage_adam(c, sh_tab);   // solve constants: safe before the wait
    __syncthreads();
    pdl_wait();
    const int w = threadIdx.x >> 5;
    const int units = ceil_div(a.B, P);
    for (int u = blockIdx.x * 4 + w; u < units; u += gridDim.x * 4) {
        for (int sb = 0; sb < P; ++sb) {
            const int b = u * P + sb;
            if (b < a.B) select_one<MCH>(a, b);
        }
        __syncwarp();      // Gram rows and support written by other lanes
        if constexpr (KT <= 32) fit_grid<KT>(a, c, u, c.tau0, sh_s[w], tab);
        else fit_unit<KT, LPS>(a, c, u, c.tau0, sh_s[w], tab);
        __syncwarp();      // coefficients and n_iter written by other lanes
        for (int sb = 0; sb < P; ++sb) {
            const int b = u * P + sb;
            if (b < a.B) resid_one<MCH>(a, b);
        }
    }
    pdl_trigger();   // after the work: the successor only overlaps our tail
}

template <int MCH, int KT, int LPS>
void launch_one(const IterArgs& a, const ClArgs& c, int iter, cudaStream_t s) {
    const int grid = resident_grid((const void*)k_update_clomp<MCH, KT, LPS>, 128,
                                   ceil_div(a.B, 4 * (32 / LPS)));
    launch_pdl(k_update_clomp<MCH, KT, LPS>, dim3(grid), dim3(128), 0, s, a, c, iter);
}

template <int MCH>
void launch_m(const IterArgs& a, const ClArgs& c, int iter, cudaStream_t s) {
    switch (round_up(iter + 1, 8)) {
        case 8: launch_one<MCH, 8, 32>(a, c, iter, s); break;
        case 16: launch_one<MCH, 16, 32>(a, c, iter, s); break;
        case 24: launch_one<MCH, 24, 32>(a, c, iter, s); break;
        case 32: launch_one<MCH, 32, 32>(a, c, iter, s); break;
        case 40: launch_one<MCH, 40, 32>(a, c, iter, s); break;
        case 48: launch_one<MCH, 48, 32>(a, c, iter, s); break;
        case 56: launch_one<MCH, 56, 32>(a, c, iter, s); break;
        default: launch_one<MCH, 64, 32>(a, c, iter, s); break;
    }
}

}  // namespace

bool update_clomp_fused_supported(const IterArgs& a) { return row_chunks(a.mp) <= 2; }

cudaError_t launch_update_clomp(const IterArgs& a, const ClArgs& c, int iter, cudaStream_t s) {
    if (row_chunks(a.mp) == 1) launch_m<1>(a, c, iter, s);
    else if (row_chunks(a.mp) == 2) launch_m<2>(a, c, iter, s);
    else return cudaErrorNotSupported;
    return cudaGetLastError();
}

}  // namespace cs
