// K4 / K5: the CL fit as a forward / adjoint kernel pair (with the adjoint
// optionally fused with one Adam step), operating directly on the caller's
// A through an index gather of the support columns -- A_S is never
// materialised.
//
// Methods, "Coefficients learning on OMP": s is masked, passed through a
// fixed fully connected layer A to give y' = A (s .* Mask), and learned by
// back-propagating the residual loss.  With L = 1/2 ||y - y'||^2:
//   forward:  r = y - A_S s_S,  L = 1/2 r.r
//   adjoint:  dL/ds_S = -A_S^T r
// One warp per signal; lanes run over the rows of A (coalesced column reads).
#include <cmath>

#include "cs_internal.cuh"

namespace cs {
namespace {

__global__ void __launch_bounds__(256)
k_clfit_forward(const float* __restrict__ A, int m, int lda, const int32_t* __restrict__ S,
                const float* __restrict__ Sv, int t, int lds, const float* __restrict__ Y,
                int ldy, int B, float* __restrict__ R, int ldr, float* __restrict__ loss) {
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= B) return;
    const int32_t* sb = S + (size_t)b * lds;
    const float* vb = Sv + (size_t)b * lds;
    float ss = 0.f;
    for (int i = lane; i < m; i += 32) {
        float r = Y[(size_t)b * ldy + i];
        for (int q = 0; q < t; ++q) r = fmaf(-A[(size_t)sb[q] * lda + i], vb[q], r);
        R[(size_t)b * ldr + i] = r;
        ss = fmaf(r, r, ss);
    }
    ss = warp_sum(ss);
    if (lane == 0 && loss) loss[b] = 0.5f * ss;
}

__global__ void __launch_bounds__(256)
k_clfit_adjoint(const float* __restrict__ A, int m, int lda, const int32_t* __restrict__ S,
                float* __restrict__ Sv, int t, int lds, const float* __restrict__ R, int ldr,
                int B, float* __restrict__ grad, float* __restrict__ mom, float* __restrict__ vel,
                float c1, float c2, float beta1, float beta2, float eps, int adam) {
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= B) return;
    const int32_t* sb = S + (size_t)b * lds;
    const float* rb = R + (size_t)b * ldr;
    for (int q = 0; q < t; ++q) {
        const float* col = A + (size_t)sb[q] * lda;
        float acc = 0.f;
        for (int i = lane; i < m; i += 32) acc = fmaf(col[i], rb[i], acc);
        const float g = -warp_sum(acc);
        if (lane == 0) {
            const size_t o = (size_t)b * lds + q;
            if (grad) grad[o] = g;
            if (adam) {
                const float mo = fmaf(beta1, mom[o], (1.f - beta1) * g);
                const float ve = fmaf(beta2, vel[o], (1.f - beta2) * g * g);
                mom[o] = mo;
                vel[o] = ve;
                Sv[o] -= c1 * mo / fmaf(sqrtf(ve), c2, eps);
            }
        }
    }
}

}  // namespace

cudaError_t launch_clfit_forward(const float* A, int m, int lda, const int32_t* S, const float* Sv,
                                 int t, int lds, const float* Y, int ldy, int batch, float* R,
                                 int ldr, float* loss, cudaStream_t s) {
    k_clfit_forward<<<ceil_div(batch, 8), 256, 0, s>>>(A, m, lda, S, Sv, t, lds, Y, ldy, batch, R,
                                                       ldr, loss);
    return cudaGetLastError();
}

cudaError_t launch_clfit_adjoint(const float* A, int m, int lda, const int32_t* S, float* Sv,
                                 int t, int lds, const float* R, int ldr, int batch, float* grad,
                                 float* mom, float* vel, int tau, float lr, float beta1,
                                 float beta2, float eps, int adam, cudaStream_t s) {
    float c1 = 0.f, c2 = 0.f;
    if (adam) {
        // bias corrections in float64 from the float32 hyper-parameters
        c1 = (float)((double)lr / (1.0 - std::pow((double)beta1, (double)tau)));
        c2 = (float)(1.0 / std::sqrt(1.0 - std::pow((double)beta2, (double)tau)));
    }
    k_clfit_adjoint<<<ceil_div(batch, 8), 256, 0, s>>>(A, m, lda, S, Sv, t, lds, R, ldr, batch,
                                                       grad, mom, vel, c1, c2, beta1, beta2, eps,
                                                       adam);
    return cudaGetLastError();
}

}  // namespace cs
