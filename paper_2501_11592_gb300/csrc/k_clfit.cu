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
// One CTA per signal: the forward kernel spreads the rows over its threads,
// the adjoint the support atoms over its warps (coalesced column reads).
#include <cmath>

#include "cs_internal.cuh"

namespace cs {
namespace {

constexpr int CF_THREADS = 256;   // one CTA per signal
constexpr int CF_ROWS = 4;        // rows per thread per pass of the forward kernel

// Forward: thread j of the signal's CTA owns rows j, j + 256, ... of r and
// subtracts the support columns in support order (one fused multiply-add
// per term, as r = y - sum_q a_q s_q is written); the columns' indices and
// values are staged in shared memory 256 at a time, and four rows' loads are
// in flight per column.
__global__ void __launch_bounds__(CF_THREADS)
k_clfit_forward(const float* __restrict__ A, int m, int lda, const int32_t* __restrict__ S,
                const float* __restrict__ Sv, int t, int lds, const float* __restrict__ Y,
                int ldy, int B, float* __restrict__ R, int ldr, float* __restrict__ loss) {
    __shared__ int sj[CF_THREADS];
    __shared__ float sv[CF_THREADS];
    __shared__ float red[CF_THREADS / 32];
    const int b = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int32_t* sb = S + (size_t)b * lds;
    const float* vb = Sv + (size_t)b * lds;
    float ss = 0.f;
    for (int i0 = 0; i0 < m; i0 += CF_THREADS * CF_ROWS) {
        float r[CF_ROWS];
#pragma unroll
        for (int u = 0; u < CF_ROWS; ++u) {
            const int i = i0 + tid + CF_THREADS * u;
            r[u] = i < m ? Y[(size_t)b * ldy + i] : 0.f;
        }
        for (int q0 = 0; q0 < t; q0 += CF_THREADS) {
            const int qn = min(CF_THREADS, t - q0);
            __syncthreads();
            if (tid < qn) {
                sj[tid] = sb[q0 + tid];
                sv[tid] = vb[q0 + tid];
            }
            __syncthreads();
            for (int q = 0; q < qn; ++q) {
                const float* col = A + (size_t)sj[q] * lda;
                float a[CF_ROWS];
#pragma unroll
                for (int u = 0; u < CF_ROWS; ++u) {
                    const int i = i0 + tid + CF_THREADS * u;
                    a[u] = i < m ? col[i] : 0.f;
                }
#pragma unroll
                for (int u = 0; u < CF_ROWS; ++u) r[u] = fmaf(-a[u], sv[q], r[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < CF_ROWS; ++u) {
            const int i = i0 + tid + CF_THREADS * u;
            if (i < m) {
                R[(size_t)b * ldr + i] = r[u];
                ss = fmaf(r[u], r[u], ss);
            }
        }
    }
    ss = warp_sum(ss);
    if (lane == 0) red[warp] = ss;
    __syncthreads();
    if (tid == 0 && loss) {
        float tot = 0.f;
        for (int w = 0; w < CF_THREADS / 32; ++w) tot += red[w];
        loss[b] = 0.5f * tot;
    }
}

// Adjoint (+ Adam): warp w of the signal's CTA takes the support atoms
// w, w + 8, ...; for each, the lanes sum a_q . r over the rows (ascending per
// lane, then the warp tree) and lane 0 writes the gradient and the update.
__global__ void __launch_bounds__(CF_THREADS)
k_clfit_adjoint(const float* __restrict__ A, int m, int lda, const int32_t* __restrict__ S,
                float* __restrict__ Sv, int t, int lds, const float* __restrict__ R, int ldr,
                int B, float* __restrict__ grad, float* __restrict__ mom, float* __restrict__ vel,
                float c1, float c2, float beta1, float beta2, float eps, int adam) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int b = blockIdx.x;
    const int32_t* sb = S + (size_t)b * lds;
    const float* rb = R + (size_t)b * ldr;
    for (int q = warp; q < t; q += CF_THREADS / 32) {
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
    if (batch <= 0) return cudaSuccess;
    k_clfit_forward<<<batch, CF_THREADS, 0, s>>>(A, m, lda, S, Sv, t, lds, Y, ldy, batch, R, ldr, loss);
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
    if (batch <= 0) return cudaSuccess;
    k_clfit_adjoint<<<batch, CF_THREADS, 0, s>>>(A, m, lda, S, Sv, t, lds, R, ldr, batch, grad, mom, vel, c1,
                                                 c2, beta1, beta2, eps, adam);
    return cudaGetLastError();
}

}  // namespace cs
