// Total-variation prior of Eq. 5 in the Gram-form CL fit.  For x = D s the
// prior w TV(x) = (w/N) ||Delta D_S s_S||^2 (Delta: the (N-1) x N first
// difference) is quadratic in s, with gradient lambda (Delta D)_S^T
// (Delta D)_S s_S, lambda = 2w/N.  So the fit keeps its form g = G s - b with
// G = A_S^T A_S + lambda T_S, T = (Delta D)^T (Delta D): the prior enters the
// solve once, as lambda T added to the Gram matrix A^T A from which every
// support Gram matrix is gathered.
#include "cs_internal.cuh"

#include <algorithm>

namespace cs {
namespace {

// E[j][i] = D[i+1, j] - D[i, j] for i < N-1 (zero up to the padded length
// Ep): the differenced waveform of atom j.  D == nullptr: atom j is the unit
// vector e_j (N = n).
__global__ void k_tv_diff(const float* __restrict__ D, int N, int ldd, int n, float* __restrict__ E, int Ep) {
    const int j = blockIdx.y;
    if (j >= n) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Ep; i += gridDim.x * blockDim.x) {
        float v = 0.f;
        if (i < N - 1) {
            if (D) v = D[(size_t)j * ldd + i + 1] - D[(size_t)j * ldd + i];
            else v = (float)((i + 1 == j) ? 1 : 0) - (float)((i == j) ? 1 : 0);
        }
        E[(size_t)j * Ep + i] = v;
    }
}

__global__ void k_axpy(float* __restrict__ y, const float* __restrict__ x, float alpha, size_t len) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (size_t)gridDim.x * blockDim.x)
        y[i] = fmaf(alpha, x[i], y[i]);
}

}  // namespace

cudaError_t launch_tv_prior(const float* D, int N, int ldd, int n, float lambda, float* E, int Ep, float* T,
                            float* GA, cudaStream_t s) {
    dim3 g1(ceil_div(Ep, 256), n);
    k_tv_diff<<<g1, 256, 0, s>>>(D, N, ldd, n, E, Ep);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_gram_tiled(E, Ep, n, T, s);
    if (e != cudaSuccess) return e;
    const size_t len = (size_t)n * n;
    const int blocks = (int)std::min<size_t>((len + 255) / 256, 4096);
    k_axpy<<<blocks, 256, 0, s>>>(GA, T, lambda, len);
    return cudaGetLastError();
}

}  // namespace cs
