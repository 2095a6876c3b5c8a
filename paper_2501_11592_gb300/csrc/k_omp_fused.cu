// Whole plain-OMP solves of small batches, one CTA per signal, one launch
// (a single signal is latency-bound: the per-iteration kernels would spend
// it in launches and in round trips through L2).  Each iteration of Eq. 2's
// greedy loop:
//   * correlation c = A^T r of every unselected atom, float32, k ascending
//     with one fused multiply-add per term -- the order of the batched
//     float32 correlation kernel, so the values are the same -- and the
//     masked argmax (lowest atom on ties): threads over atoms, A held in
//     shared memory for the whole solve when it fits (else staged a few K
//     values at a time);
//   * warp 0 appends the atom (bitset, support, Gram column from A^T A,
//     a_j^T y), runs the float64 Cholesky update (k_chol.cuh), forms the
//     residual and applies the stop test.
// The signal's residual, y, support, coefficients, Gram column, bitset and
// Cholesky factor stay in shared memory for the whole solve; the outputs are
// written as they change.  Every step uses the batched path's arithmetic in
// the same order (the same device functions where they exist), so a solve
// gives the same bits either way.
#include "k_chol.cuh"
#include "k_resid.cuh"

namespace cs {
namespace {

constexpr int OF_THREADS = 256;
constexpr int OF_KC = 8;              // K values of A staged per step
constexpr int OF_MAX_SMEM = 200 * 1024;
constexpr size_t OF_STATIC = sizeof(float) * OF_KC * (OF_THREADS + 1) + 1024;

// Dynamic shared memory: W = L^{-T} by rows and by columns (2 K x K), z, x
// (float64) | r, y (mp floats) | Gram column, coefficients (K floats) |
// support (K ints) | bitset (nw words) | (when it fits) A itself, K-major
// with a padded row of n + 1 atoms.
__host__ __device__ inline size_t of_state(int K, int mp, int nw) {
    const size_t v = sizeof(double) * (2 * (size_t)K * K + 2 * (size_t)K) + sizeof(float) * (2 * (size_t)mp + 2 * (size_t)K) +
                     sizeof(int) * (size_t)K + sizeof(uint32_t) * (size_t)nw;
    return (v + 15) & ~(size_t)15;
}
__host__ __device__ inline size_t of_resident_a(int mp, int n) { return sizeof(float) * (size_t)mp * (n + 1); }
__host__ __device__ inline bool of_a_fits(int K, int mp, int nw, int n) {
    return of_state(K, mp, nw) + of_resident_a(mp, n) + OF_STATIC <= (size_t)OF_MAX_SMEM;
}

// Column j of the shared-memory A (sa[q * np1 + j]) row-sliced like load_row.
template <int MCH>
__device__ __forceinline__ void load_col_sa(const float* sa, int np1, int mp, int j, float4 (&v)[MCH]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < MCH; ++c) {
        const int i = 4 * (c * 32 + lane);
        v[c] = (i < mp) ? make_float4(sa[(size_t)i * np1 + j], sa[(size_t)(i + 1) * np1 + j],
                                      sa[(size_t)(i + 2) * np1 + j], sa[(size_t)(i + 3) * np1 + j])
                        : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// warp_dots32 with the columns read from the shared-memory A (the same sums
// in the same order, so the same values as the Gram table).
template <int MCH>
__device__ __forceinline__ float warp_dots32_sa(const float* sa, int np1, int mp, int my_atom,
                                                const float4 (&x)[MCH]) {
    const int lane = threadIdx.x & 31;
    float part[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) {
        const int j = __shfl_sync(FULL, my_atom, q);
        float acc = 0.f;
        if (j >= 0) {
#pragma unroll
            for (int c = 0; c < MCH; ++c) {
                const int i = 4 * (c * 32 + lane);
                if (i < mp) {
                    const float4 col = make_float4(sa[(size_t)i * np1 + j], sa[(size_t)(i + 1) * np1 + j],
                                                   sa[(size_t)(i + 2) * np1 + j], sa[(size_t)(i + 3) * np1 + j]);
                    acc += dot4(col, x[c]);
                }
            }
        }
        part[q] = acc;
    }
    warp_reduce_scatter32(part);
    return part[0];
}

// resid_vector_from (k_resid.cuh) with the columns read from the
// shared-memory A: the same fused multiply-adds in the same order.
template <int MCH>
__device__ __forceinline__ void resid_vector_sa(const float* sa, int np1, int mp, const int t, float4 (&r)[MCH],
                                                const int* sup, const float* x) {
    const int lane = threadIdx.x & 31;
    for (int q0 = 0; q0 < t; q0 += 32) {
        const int qn = min(32, t - q0);
        const int my_j = (lane < qn) ? sup[q0 + lane] : 0;
        const float my_x = (lane < qn) ? x[q0 + lane] : 0.f;
        for (int u0 = 0; u0 < qn; u0 += 4) {
            float4 v[4][MCH];
            float xq[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = __shfl_sync(FULL, my_j, u0 + u);
                xq[u] = __shfl_sync(FULL, my_x, u0 + u);
                if (u0 + u < qn) {
                    load_col_sa<MCH>(sa, np1, mp, j, v[u]);
                } else {
#pragma unroll
                    for (int c = 0; c < MCH; ++c) v[u][c] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int c = 0; c < MCH; ++c) {
                    r[c].x = fmaf(-v[u][c].x, xq[u], r[c].x);
                    r[c].y = fmaf(-v[u][c].y, xq[u], r[c].y);
                    r[c].z = fmaf(-v[u][c].z, xq[u], r[c].z);
                    r[c].w = fmaf(-v[u][c].w, xq[u], r[c].w);
                }
        }
    }
}

// A (m rows of leading dimension ld, zero rows up to mp) into sa[q * np1 + j]:
// consecutive threads take one column's consecutive rows (the stores hit
// distinct banks when np1 is odd), sixteen loads in flight per thread before
// their stores.
__device__ __forceinline__ void copy_a_to_sa(const float* __restrict__ A, int ld, int m, int mp, int n, float* sa,
                                             int np1) {
    constexpr int U = 16;
    const int total = n * mp;
    for (int e0 = threadIdx.x; e0 < total; e0 += U * OF_THREADS) {
        float v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * OF_THREADS;
            const int j = e / mp, q = e - (e / mp) * mp;
            v[u] = (e < total && q < m) ? A[(size_t)j * ld + q] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * OF_THREADS;
            if (e < total) sa[(size_t)(e % mp) * np1 + e / mp] = v[u];
        }
    }
}

// Ac / Yc non-null (A resident in shared memory): the solve reads the
// caller's A (leading dimension lda) and Y (ldy) itself and does the
// set-up of k_setup (same sums), so it is the only launch of the solve.
template <int MCH>
__global__ void __launch_bounds__(OF_THREADS) k_omp_fused(IterArgs a, const float* __restrict__ Ac, int lda,
                                                          const float* __restrict__ Yc, int ldy) {
    __shared__ float sh_v[OF_THREADS / 32];
    __shared__ int sh_j[OF_THREADS / 32];
    __shared__ float sh_a[OF_KC][OF_THREADS + 1];   // A[q0 + q][j0 + atom], padded rows
    __shared__ int sh_status, sh_t;
    extern __shared__ __align__(16) unsigned char sh_dyn[];
    const int K = a.kmax;
    double* Ws = reinterpret_cast<double*>(sh_dyn);
    double* zs = Ws + 2 * (size_t)K * K;
    double* xs = zs + K;
    float* rs = reinterpret_cast<float*>(xs + K);
    float* ys = rs + a.mp;
    float* gs = ys + a.mp;
    float* cs_ = gs + K;
    int* ss = reinterpret_cast<int*>(cs_ + K);
    uint32_t* ms = reinterpret_cast<uint32_t*>(ss + K);
    // A resident for the whole solve when it fits: sa[q * (n + 1) + j]
    const bool resident = of_a_fits(K, a.mp, a.nw, a.n);
    float* sa = reinterpret_cast<float*>(sh_dyn + of_state(K, a.mp, a.nw));
    const int np1 = a.n + 1;

    const int b = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool self = Ac != nullptr;     // only with A resident
    if (self) {
        // k_setup's work for this signal (warp 0, the same sums)
        if (warp == 0) {
            const float* y = Yc + (size_t)b * ldy;
            float ssq = 0.f;
            int finite = 1;
            for (int i = lane; i < a.mp; i += 32) {
                const float v = (i < a.m) ? y[i] : 0.f;
                finite &= isfinite(v) ? 1 : 0;
                ys[i] = v;
                rs[i] = v;
                ssq = fmaf(v, v, ssq);
            }
            for (int q = lane; q < a.k; q += 32) {
                a.support[(size_t)b * a.k + q] = -1;
                a.coef[(size_t)b * a.k + q] = 0.f;
            }
            ssq = warp_sum(ssq);
            finite = __all_sync(FULL, finite);
            if (lane == 0) {
                const float rho = sqrtf(ssq);
                int st;
                a.n_iter[b] = 0;
                if (!finite) {
                    st = CS_SIG_NONFINITE;
                    a.res_norm[b] = __int_as_float(0x7fffffff);
                } else {
                    a.res_norm[b] = rho;
                    st = ((double)rho <= a.tol) ? CS_SIG_REACHED_TOL : -1;
                }
                a.status[b] = st;
                sh_status = st;
                sh_t = 0;
            }
        }
        for (int w = tid; w < a.nw; w += OF_THREADS) ms[w] = 0u;
        copy_a_to_sa(Ac, lda, a.m, a.mp, a.n, sa, np1);
    } else {
        for (int i = tid; i < a.mp; i += OF_THREADS) {
            rs[i] = a.R32[(size_t)b * a.mp + i];
            ys[i] = a.Y32[(size_t)b * a.mp + i];
        }
        for (int w = tid; w < a.nw; w += OF_THREADS) ms[w] = a.mask[(size_t)b * a.nw + w];
        if (resident)
            copy_a_to_sa(a.A32, a.mp, a.mp, a.mp, a.n, sa, np1);
        if (tid == 0) {
            sh_status = a.status[b];
            sh_t = a.n_iter[b];
        }
    }
    for (int it = 0; it < a.iters; ++it) {
        __syncthreads();                 // last iteration's residual, bitset and status
        if (sh_status >= 0) break;       // the same value for every thread
        const int t = sh_t;
        float bv = -1.f;
        int bj = -1;
        for (int j0 = 0; j0 < a.n; j0 += OF_THREADS) {
            // thread tid owns atom j0 + tid; the K values of the block's
            // atoms arrive OF_KC at a time through shared memory (coalesced
            // reads of A's columns), and each thread sums its own in
            // ascending k with one fused multiply-add per term
            const int j = j0 + tid;
            float acc = 0.f;
            if (resident) {
                if (j < a.n)
                    for (int q = 0; q < a.mp; ++q) acc = fmaf(rs[q], sa[(size_t)q * np1 + j], acc);
            } else for (int q0 = 0; q0 < a.mp; q0 += OF_KC) {
                __syncthreads();         // the previous chunk is consumed
                for (int e = tid; e < OF_KC * OF_THREADS; e += OF_THREADS) {
                    const int ja = j0 + e / OF_KC, q = q0 + e % OF_KC;
                    sh_a[e % OF_KC][e / OF_KC] = (ja < a.n && q < a.mp) ? a.A32[(size_t)ja * a.mp + q] : 0.f;
                }
                __syncthreads();
                const int qn = min(OF_KC, a.mp - q0);
                for (int q = 0; q < qn; ++q) acc = fmaf(rs[q0 + q], sh_a[q][tid], acc);
            }
            if (j < a.n && !((ms[j >> 5] >> (j & 31)) & 1u)) {
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
        if (warp != 0) continue;
        float v = lane < OF_THREADS / 32 ? sh_v[lane] : -1.f;
        int j = lane < OF_THREADS / 32 ? sh_j[lane] : -1;
        warp_argmax(v, j);
        if (j < 0) {                     // nothing left to select
            if (lane == 0) {
                a.status[b] = CS_SIG_MAX_ITER;
                sh_status = CS_SIG_MAX_ITER;
            }
            continue;
        }
        // ---- append atom j as support entry t (the batched append's arithmetic)
        if (lane == 0) {
            ms[j >> 5] |= 1u << (j & 31);
            ss[t] = j;
            a.support[(size_t)b * a.k + t] = j;
        }
        float4 aj[MCH], yv[MCH];
        if (resident) load_col_sa<MCH>(sa, np1, a.mp, j, aj);
        else load_row<MCH>(a.A32 + (size_t)j * a.mp, a.mp, aj);
        load_row<MCH>(ys, a.mp, yv);
        float dd = 0.f, by = 0.f;
#pragma unroll
        for (int c = 0; c < MCH; ++c) {
            dd += dot4(aj[c], aj[c]);
            by += dot4(aj[c], yv[c]);
        }
        dd = warp_sum(dd);               // the Gram table's a_j . a_j (same sums)
        by = warp_sum(by);
        __syncwarp();                    // the support entry
        if (resident) {
            // the Gram column formed here from the shared-memory A, in the
            // Gram table's arithmetic
            for (int i0 = 0; i0 < t; i0 += 32) {
                const int i = i0 + lane;
                const float g = warp_dots32_sa<MCH>(sa, np1, a.mp, i < t ? ss[i] : -1, aj);
                if (i < t) gs[i] = g;
            }
        } else {
            const float* garow = a.GA + (size_t)j * a.n;
            dd = garow[j];
            for (int i0 = 0; i0 < t; i0 += 32) {
                const int i = i0 + lane;
                if (i < t) gs[i] = garow[ss[i]];
            }
        }
        __syncwarp();                    // the Gram column
        // ---- float64 Cholesky update (the batched kernel's arithmetic)
        bool ok;
        if (K == 32) {
            float gl[1] = {lane < t ? gs[lane] : 0.f};
            ok = chol_warp<1>(t, K, gl, (double)dd, (double)by, Ws, Ws + (size_t)K * K, zs, xs, cs_);
        } else {
            float gl[2] = {lane < t ? gs[lane] : 0.f, lane + 32 < t ? gs[lane + 32] : 0.f};
            ok = chol_warp<2>(t, K, gl, (double)dd, (double)by, Ws, Ws + (size_t)K * K, zs, xs, cs_);
        }
        if (lane == 0) {
            if (!ok) {
                a.status[b] = CS_SIG_DEPENDENT;
                a.support[(size_t)b * a.k + t] = -1;
                sh_status = CS_SIG_DEPENDENT;
            } else {
                sh_t = t + 1;
                a.n_iter[b] = t + 1;
            }
        }
        __syncwarp();
        if (sh_status >= 0) continue;    // dependent atom
        const int t1 = t + 1;
        for (int i = lane; i < t1; i += 32) a.coef[(size_t)b * a.k + i] = cs_[i];
        // ---- residual r = y - A_S x_S, its norm, the stop test (the batched
        // residual's arithmetic)
        float4 rv[MCH];
#pragma unroll
        for (int c = 0; c < MCH; ++c) rv[c] = yv[c];
        if (resident) resid_vector_sa<MCH>(sa, np1, a.mp, t1, rv, ss, cs_);
        else resid_vector_from<MCH>(a, t1, rv, ss, cs_);
        float sq = 0.f;
        float4* R = reinterpret_cast<float4*>(rs);
#pragma unroll
        for (int c = 0; c < MCH; ++c) {
            const int i4 = c * 32 + lane;
            if (i4 * 4 < a.mp) {
                R[i4] = rv[c];
                sq += dot4(rv[c], rv[c]);
            }
        }
        sq = warp_sum(sq);
        if (lane == 0) {
            const float rho = sqrtf(sq);
            stop_test(a, b, t1, rho);
            // the status stop_test wrote, without reading it back
            sh_status = ((double)rho <= a.tol) ? CS_SIG_REACHED_TOL
                        : (t1 >= a.k) ? CS_SIG_REACHED_K : (t1 >= a.iters) ? CS_SIG_MAX_ITER : -1;
        }
    }
}

template <int MCH>
cudaError_t launch_m(const IterArgs& a, const float* Ac, int lda, const float* Yc, int ldy, cudaStream_t s) {
    const cudaError_t attr = set_smem_limit((const void*)k_omp_fused<MCH>, OF_MAX_SMEM);
    if (attr != cudaSuccess) return attr;
    const size_t smem = of_state(a.kmax, a.mp, a.nw) +
                        (of_a_fits(a.kmax, a.mp, a.nw, a.n) ? of_resident_a(a.mp, a.n) : 0);
    k_omp_fused<MCH><<<a.B, OF_THREADS, smem, s>>>(a, Ac, lda, Yc, ldy);
    return cudaGetLastError();
}

}  // namespace

bool omp_fused_supported(const IterArgs& a) {
    return a.need_gcol && a.prec == CS_CORR_FP32 && row_chunks(a.mp) <= kMaxRowChunks &&
           of_state(a.kmax, a.mp, a.nw) + OF_STATIC <= (size_t)OF_MAX_SMEM &&
           (a.GA != nullptr || of_a_fits(a.kmax, a.mp, a.nw, a.n));
}

bool omp_fused_self_contained(const IterArgs& a) {
    return omp_fused_supported(a) && of_a_fits(a.kmax, a.mp, a.nw, a.n);
}

cudaError_t launch_omp_fused(const IterArgs& a, const float* A, int lda, const float* Y, int ldy, cudaStream_t s) {
    if (!omp_fused_supported(a) || (A != nullptr && !omp_fused_self_contained(a))) return cudaErrorNotSupported;
    if (a.B <= 0) return cudaSuccess;
    switch (row_chunks(a.mp)) {
        case 1: return launch_m<1>(a, A, lda, Y, ldy, s);
        case 2: return launch_m<2>(a, A, lda, Y, ldy, s);
        case 3:
        case 4: return launch_m<4>(a, A, lda, Y, ldy, s);
        default: return launch_m<8>(a, A, lda, Y, ldy, s);
    }
}

}  // namespace cs
