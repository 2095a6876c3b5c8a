// Column-wise 2D output path: the image columns x = D s from the solver's
// sparse codes (Eq. 3 with the sparsifying basis D), and the two quality
// figures the paper reports for reconstructions, PSNR and SSIM (the index
// of Wang, Bovik, Sheikh and Simoncelli 2004: 11 x 11 Gaussian window of
// standard deviation 1.5, K1 = 0.01, K2 = 0.03, every window placed fully
// inside the image, averaged).
#include "k_common.cuh"

namespace cs {
namespace {

// One warp per signal: lanes own 32 consecutive rows of x at a time; the
// support indices and coefficients are read 32 at a time and broadcast by
// shuffles, so each D column is read as coalesced 128-byte rows.
__global__ void __launch_bounds__(256) k_synthesize(const float* __restrict__ D, int N, int n, int ldd,
                                                    const int* __restrict__ support,
                                                    const float* __restrict__ coef,
                                                    const int* __restrict__ n_iter, int k, int B,
                                                    float* __restrict__ X, int ldx) {
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= B) return;
    const int t = min(max(n_iter[b], 0), k);
    if (D == nullptr) {
        // no basis: the dense code itself (N = n), coefficients scattered
        // into a zeroed column (support entries are distinct)
        for (int i = lane; i < N; i += 32) X[(size_t)b * ldx + i] = 0.f;
        __syncwarp();
        for (int q = lane; q < t; q += 32) {
            const int j = support[(size_t)b * k + q];
            if (j >= 0 && j < n) X[(size_t)b * ldx + j] = coef[(size_t)b * k + q];
        }
        return;
    }
    for (int i0 = 0; i0 < N; i0 += 32) {
        const int i = i0 + lane;
        float acc = 0.f;
        for (int q0 = 0; q0 < t; q0 += 32) {
            const int q = q0 + lane;
            int j = (q < t) ? support[(size_t)b * k + q] : -1;
            const float c = (q < t) ? coef[(size_t)b * k + q] : 0.f;
            if (j >= n) j = -1;
            const int cnt = min(32, t - q0);
            for (int u = 0; u < cnt; ++u) {
                const int ju = __shfl_sync(FULL, j, u);
                const float cu = __shfl_sync(FULL, c, u);
                if (ju >= 0 && i < N) acc = fmaf(cu, D[(size_t)ju * ldd + i], acc);
            }
        }
        if (i < N) X[(size_t)b * ldx + i] = acc;
    }
}

constexpr int SSIM_R = 11;          // window size
constexpr int QT = 512;             // threads per image (the window loops are latency-bound)

// 1-D Gaussian factors of the window: weight (u, v) = g[u] g[v], unit sum
__constant__ float c_gauss[SSIM_R];

__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    for (int i = 0; i < QT / 32; ++i) r += sh[i];
    return r;
}

__device__ __forceinline__ float block_minmax(float v, float* sh, bool is_max) {
    for (int o = 16; o > 0; o >>= 1) {
        const float u = __shfl_xor_sync(FULL, v, o);
        v = is_max ? fmaxf(v, u) : fminf(v, u);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    float r = sh[0];
    for (int i = 1; i < QT / 32; ++i) r = is_max ? fmaxf(r, sh[i]) : fminf(r, sh[i]);
    return r;
}

// One block per image (H x W column-major, consecutive images).  Window
// statistics in float32: the weighted means first, then the centred second
// moments (no cancellation of E[x^2] - mean^2), and each window's index;
// the indices and the squared errors are summed in float64.
__global__ void __launch_bounds__(QT) k_image_quality(const float* __restrict__ X, const float* __restrict__ R,
                                                      int H, int W, float peak,
                                                      float* __restrict__ psnr, float* __restrict__ ssim) {
    __shared__ double shd[QT / 32];
    __shared__ float shf[QT / 32];
    const size_t off = (size_t)blockIdx.x * H * W;
    const float* x = X + off;
    const float* y = R + off;
    const int HW = H * W;

    double se = 0.0;
    float lo = __int_as_float(0x7f800000), hi = __int_as_float(0xff800000);
    for (int p = threadIdx.x; p < HW; p += QT) {
        const float d = x[p] - y[p];
        se += (double)d * (double)d;
        lo = fminf(lo, y[p]);
        hi = fmaxf(hi, y[p]);
    }
    se = block_sum(se, shd);
    lo = block_minmax(lo, shf, false);
    hi = block_minmax(hi, shf, true);
    const float L = peak > 0.f ? peak : hi - lo;
    const float C1 = (0.01f * L) * (0.01f * L), C2 = (0.03f * L) * (0.03f * L);

    const int ph = H - SSIM_R + 1, pw = W - SSIM_R + 1;
    double acc = 0.0;
    for (int p = threadIdx.x; p < ph * pw; p += QT) {
        const int r0 = p % ph, c0 = p / ph;   // consecutive threads: consecutive rows (coalesced)
        float mx = 0.f, my = 0.f;
        for (int v = 0; v < SSIM_R; ++v) {
            const float* xc = x + (size_t)(c0 + v) * H + r0;
            const float* yc = y + (size_t)(c0 + v) * H + r0;
            float sx = 0.f, sy = 0.f;
#pragma unroll
            for (int u = 0; u < SSIM_R; ++u) {
                sx = fmaf(c_gauss[u], xc[u], sx);
                sy = fmaf(c_gauss[u], yc[u], sy);
            }
            mx = fmaf(c_gauss[v], sx, mx);
            my = fmaf(c_gauss[v], sy, my);
        }
        float vx = 0.f, vy = 0.f, cxy = 0.f;
        for (int v = 0; v < SSIM_R; ++v) {
            const float* xc = x + (size_t)(c0 + v) * H + r0;
            const float* yc = y + (size_t)(c0 + v) * H + r0;
            float sxx = 0.f, syy = 0.f, sxy = 0.f;
#pragma unroll
            for (int u = 0; u < SSIM_R; ++u) {
                const float dx = xc[u] - mx, dy = yc[u] - my;
                sxx = fmaf(c_gauss[u] * dx, dx, sxx);
                syy = fmaf(c_gauss[u] * dy, dy, syy);
                sxy = fmaf(c_gauss[u] * dx, dy, sxy);
            }
            vx = fmaf(c_gauss[v], sxx, vx);
            vy = fmaf(c_gauss[v], syy, vy);
            cxy = fmaf(c_gauss[v], sxy, cxy);
        }
        // the window's index in float32 (its terms are float32 already),
        // summed over the windows in float64
        const float num = fmaf(2.f * mx, my, C1) * fmaf(2.f, cxy, C2);
        const float den = (fmaf(mx, mx, my * my) + C1) * ((vx + vy) + C2);
        acc += (double)(num / den);
    }
    acc = block_sum(acc, shd);
    if (threadIdx.x == 0) {
        const double mse = se / HW;
        psnr[blockIdx.x] = (mse == 0.0) ? __int_as_float(0x7f800000)
                                        : (float)(10.0 * log10((double)L * (double)L / mse));
        ssim[blockIdx.x] = (float)(acc / ((double)ph * pw));
    }
}

}  // namespace

cudaError_t launch_synthesize(const float* D, int N, int n, int ldd, const int* support, const float* coef,
                              const int* n_iter, int k, int B, float* X, int ldx, cudaStream_t s) {
    if (B <= 0) return cudaSuccess;
    k_synthesize<<<ceil_div(B, 8), 256, 0, s>>>(D, N, n, ldd, support, coef, n_iter, k, B, X, ldx);
    return cudaGetLastError();
}

cudaError_t launch_image_quality(const float* X, const float* R, int H, int W, int count, float peak,
                                 float* psnr, float* ssim, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    float win[SSIM_R];
    double g[SSIM_R], sum = 0.0;
    for (int u = 0; u < SSIM_R; ++u) {
        const double d = u - (SSIM_R - 1) / 2.0;
        g[u] = exp(-d * d / (2.0 * 1.5 * 1.5));
        sum += g[u];
    }
    for (int u = 0; u < SSIM_R; ++u) win[u] = (float)(g[u] / sum);
    cudaError_t e = cudaMemcpyToSymbolAsync(c_gauss, win, sizeof(win), 0, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    k_image_quality<<<count, QT, 0, s>>>(X, R, H, W, peak, psnr, ssim);
    return cudaGetLastError();
}

}  // namespace cs
