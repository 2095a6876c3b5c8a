// K0: float32 SIMT correlation C^T = R^T A with a fused masked |c| argmax.
//
// The residual-injection branch of CLOMP (Methods, "Coefficients learning on
// OMP") feeds r^T through a fully connected layer whose fixed weights are A,
// giving A^T r for every signal at once; plain OMP then keeps the position of
// the largest |A^T r| among unselected atoms.  Here the output tile is
// 128 signals x 128 atoms, K = m runs in steps of 16 through double-buffered
// shared memory, and each thread owns an 8 x 8 register tile.  C never leaves
// the chip: the epilogue masks selected atoms (bitset), takes |c| and reduces
// to one (|c|, atom) pair per signal and atom tile, lowest atom on ties.
#include "cs_internal.cuh"

namespace cs {
namespace {

constexpr int BM = 128, BN = kCorrFp32TileN, BK = 16, PAD = 4;

// DENSE: write C^T (B x n, row stride ldd) instead of the argmax epilogue.
// status (optional): tiles of signals that have all stopped are skipped.
template <bool DENSE>
__global__ void __launch_bounds__(256, 2)
k_corr_fp32(const float* __restrict__ R32, const float* __restrict__ A32, int mp, int B, int n,
            const uint32_t* __restrict__ mask, int nw, const int* __restrict__ status,
            float* __restrict__ cand_val, int* __restrict__ cand_idx, int nch,
            float* __restrict__ dense, int ldd) {
    __shared__ __align__(16) float As[2][BK][BM + PAD];
    __shared__ __align__(16) float Bs[2][BK][BN + PAD];
    __shared__ int any_live;

    pdl_wait();
    const int tid = threadIdx.x;
    const int b0 = blockIdx.x * BM;
    const int j0 = blockIdx.y * BN;

    if (tid == 0) any_live = 0;
    __syncthreads();
    if (tid < BM) {
        const int b = b0 + tid;
        if (b < B && (status == nullptr || status[b] < 0)) any_live = 1;
    }
    __syncthreads();
    if (!any_live) return;

    const int ty = tid >> 4, tx = tid & 15;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    const int nk = ceil_div(mp, BK);
    float4 ra[2], rb[2];
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);

    auto gload = [&](int kt) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int e = tid + 256 * h;
            const int row = e >> 2;
            const int kk = kt * BK + (e & 3) * 4;
            const int sig = b0 + row, atom = j0 + row;
            ra[h] = (sig < B && kk < mp) ? *reinterpret_cast<const float4*>(R32 + (size_t)sig * mp + kk) : zero4;
            rb[h] = (atom < n && kk < mp) ? *reinterpret_cast<const float4*>(A32 + (size_t)atom * mp + kk) : zero4;
        }
    };
    auto sstore = [&](int buf) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int e = tid + 256 * h;
            const int row = e >> 2;
            const int kq = (e & 3) * 4;
            As[buf][kq + 0][row] = ra[h].x;
            As[buf][kq + 1][row] = ra[h].y;
            As[buf][kq + 2][row] = ra[h].z;
            As[buf][kq + 3][row] = ra[h].w;
            Bs[buf][kq + 0][row] = rb[h].x;
            Bs[buf][kq + 1][row] = rb[h].y;
            Bs[buf][kq + 2][row] = rb[h].z;
            Bs[buf][kq + 3][row] = rb[h].w;
        }
    };

    gload(0);
    sstore(0);
    __syncthreads();
    for (int kt = 0; kt < nk; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < nk) gload(kt + 1);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + ty * 4]);
            const float4 c0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
            const float4 c1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tx * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        if (kt + 1 < nk) sstore(buf ^ 1);
        __syncthreads();
    }

    if constexpr (DENSE) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int sig = b0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
            if (sig >= B) continue;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int atom = j0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
                if (atom < n) dense[(size_t)sig * ldd + atom] = acc[i][j];
            }
        }
    } else {
    // Epilogue: masked |c| argmax per signal over this atom tile.
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int sig = b0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
        float bv = -1.f;
        int bj = -1;
        if (sig < B) {
            const int a_lo = j0 + tx * 4, a_hi = j0 + 64 + tx * 4;
            const uint32_t w_lo = (a_lo < n) ? mask[(size_t)sig * nw + (a_lo >> 5)] : 0xffffffffu;
            const uint32_t w_hi = (a_hi < n) ? mask[(size_t)sig * nw + (a_hi >> 5)] : 0xffffffffu;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int atom = (j < 4 ? a_lo + j : a_hi + (j - 4));
                const uint32_t w = (j < 4 ? w_lo : w_hi);
                if (atom < n && !((w >> (atom & 31)) & 1u)) {
                    const float v = fabsf(acc[i][j]);
                    if (cand_better(v, atom, bv, bj)) { bv = v; bj = atom; }
                }
            }
        }
        // the 16 threads sharing `ty` form one half-warp
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
            if (cand_better(ov, oj, bv, bj)) { bv = ov; bj = oj; }
        }
        if (tx == 0 && sig < B) {
            cand_val[(size_t)sig * nch + blockIdx.y] = bv;
            cand_idx[(size_t)sig * nch + blockIdx.y] = bj;
        }
    }
    }
}

}  // namespace

cudaError_t launch_corr_fp32(const IterArgs& a, cudaStream_t s) {
    dim3 grid(ceil_div(a.B, BM), ceil_div(a.n, BN));
    return launch_pdl(k_corr_fp32<false>, grid, dim3(256), 0, s, a.R32, a.A32, a.mp, a.B, a.n, a.mask, a.nw,
                      a.status, a.cand_val, a.cand_idx, a.nch, (float*)nullptr, 0);
}

cudaError_t launch_corr_fp32_dense_live(const IterArgs& a, float* C, int ldc, cudaStream_t s) {
    dim3 grid(ceil_div(a.B, BM), ceil_div(a.n, BN));
    k_corr_fp32<true><<<grid, 256, 0, s>>>(a.R32, a.A32, a.mp, a.B, a.n, nullptr, 0, a.status, nullptr, nullptr, 1,
                                           C, ldc);
    return cudaGetLastError();
}

cudaError_t launch_corr_fp32_dense(const float* R32, const float* A32, int mp, int B, int n, float* C,
                                   int ldc, cudaStream_t s) {
    dim3 grid(ceil_div(B, BM), ceil_div(n, BN));
    k_corr_fp32<true><<<grid, 256, 0, s>>>(R32, A32, mp, B, n, nullptr, 0, nullptr, nullptr, nullptr, 1,
                                           C, ldc);
    return cudaGetLastError();
}

}  // namespace cs
