// Whole plain-OMP solves of small batches, one CTA per signal, one launch
// (the single-signal case is latency-bound: the per-iteration kernels would
// spend it in launches).  Each iteration of Eq. 2's greedy loop:
//   * correlation c = A^T r of every unselected atom, float32, k ascending
//     with one fused multiply-add per term -- the order of the batched
//     float32 correlation kernel, so the values are the same -- and the
//     masked argmax (lowest atom on ties): threads over atoms, A's columns
//     staged through shared memory a few K values at a time;
//   * warp 0 appends the atom (bitset, support, Gram column from A^T A,
//     a_j^T y), thread 0 runs the float64 Cholesky update and the
//     triangular solves on the factor held in shared memory (a dependent
//     chain of L2 round trips otherwise), warp 0 forms the residual and
//     the stop test.
// The append, Cholesky and residual are the batched path's own functions,
// so a solve gives the same bits either way.
#include "k_chol.cuh"
#include "k_resid.cuh"
#include "k_select.cuh"

namespace cs {
namespace {

constexpr int OF_THREADS = 256;
constexpr int OF_KC = 8;              // K values of A staged per step

template <int MCH>
__global__ void __launch_bounds__(OF_THREADS) k_omp_fused(IterArgs a) {
    __shared__ float sh_v[OF_THREADS / 32];
    __shared__ int sh_j[OF_THREADS / 32];
    __shared__ float sh_a[OF_KC][OF_THREADS + 1];   // A[q0 + q][j0 + atom], padded rows
    extern __shared__ double sh_chol[];   // L (kmax x kmax), z, x of the signal
    const int b = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float* r = a.R32 + (size_t)b * a.mp;
    uint32_t* mrow = a.mask + (size_t)b * a.nw;
    for (int it = 0; it < a.iters; ++it) {
        __syncthreads();                 // last iteration's residual, bitset and status
        if (a.status[b] >= 0) break;     // the same value for every thread
        const int t = a.n_iter[b];
        float bv = -1.f;
        int bj = -1;
        for (int j0 = 0; j0 < a.n; j0 += OF_THREADS) {
            // thread tid owns atom j0 + tid; the K values of the block's
            // atoms arrive OF_KC at a time through shared memory (coalesced
            // reads of A's columns), and each thread sums its own in
            // ascending k with one fused multiply-add per term
            const int j = j0 + tid;
            float acc = 0.f;
            for (int q0 = 0; q0 < a.mp; q0 += OF_KC) {
                __syncthreads();         // the previous chunk is consumed
                for (int e = tid; e < OF_KC * OF_THREADS; e += OF_THREADS) {
                    const int ja = j0 + e / OF_KC, q = q0 + e % OF_KC;
                    sh_a[e % OF_KC][e / OF_KC] = (ja < a.n && q < a.mp) ? a.A32[(size_t)ja * a.mp + q] : 0.f;
                }
                __syncthreads();
                const int qn = min(OF_KC, a.mp - q0);
                for (int q = 0; q < qn; ++q) acc = fmaf(r[q0 + q], sh_a[q][tid], acc);
            }
            if (j < a.n && !((mrow[j >> 5] >> (j & 31)) & 1u)) {
                const float v = fabsf(acc);
                if (cand_better(v, j, bv, bj)) {
                    bv = v;
                    bj = j;
                }
            }
        }
        warp_argmax(bv, bj);
        if (lane == 0) {
            sh_v[warp] = bv;
            sh_j[warp] = bj;
        }
        __syncthreads();
        if (warp == 0) {
            float v = lane < OF_THREADS / 32 ? sh_v[lane] : -1.f;
            int j = lane < OF_THREADS / 32 ? sh_j[lane] : -1;
            warp_argmax(v, j);
            if (j < 0) {                 // nothing left to select
                if (lane == 0) a.status[b] = CS_SIG_MAX_ITER;
            } else {
                if (lane == 0) mrow[j >> 5] |= 1u << (j & 31);
                float4 y[MCH];
                load_row<MCH>(a.Y32 + (size_t)b * a.mp, a.mp, y);
                append_atom<MCH>(a, b, t, j, y);
                __syncwarp();            // Gram column, dnorm, a_j^T y for thread 0
                if (lane == 0) {
                    double* Ls = sh_chol;
                    double* zs = Ls + (size_t)a.kmax * a.kmax;
                    chol_update_at(a, b, Ls, 1, zs, zs + a.kmax, 1);
                }
                __syncwarp();            // coefficients, n_iter, status for the warp
                resid_one<MCH>(a, b);
            }
        }
    }
}

template <int MCH>
void launch_m(const IterArgs& a, cudaStream_t s) {
    const size_t smem = sizeof(double) * ((size_t)a.kmax * a.kmax + 2 * (size_t)a.kmax);
    k_omp_fused<MCH><<<a.B, OF_THREADS, smem, s>>>(a);
}

}  // namespace

bool omp_fused_supported(const IterArgs& a) {
    return a.need_gcol && a.GA != nullptr && a.prec == CS_CORR_FP32 && row_chunks(a.mp) <= kMaxRowChunks;
}

cudaError_t launch_omp_fused(const IterArgs& a, cudaStream_t s) {
    if (!omp_fused_supported(a)) return cudaErrorNotSupported;
    if (a.B <= 0) return cudaSuccess;
    switch (row_chunks(a.mp)) {
        case 1: launch_m<1>(a, s); break;
        case 2: launch_m<2>(a, s); break;
        case 3:
        case 4: launch_m<4>(a, s); break;
        default: launch_m<8>(a, s); break;
    }
    return cudaGetLastError();
}

}  // namespace cs
