// OMP least squares (Table "s forward block", OMP row: pinv of A(:,Mask)) as
// an incremental float64 Cholesky update of one signal, run by one warp and
// shared by the batched kernel (state in global memory) and the fused
// small-batch solve (state in shared memory) (internal header).
//
// With L L^T = A_S^T A_S the solve keeps W = L^{-T} (upper triangular)
// instead of L.  Adding atom a with Gram column g = A_S^T a, d = ||a||^2 and
// b_t = a^T y:
//   l    = L^{-1} g = W^T g            (the new row of L, a matrix-vector product)
//   L_tt = sqrt(d - l.l)               (only 1 / L_tt is formed, see rsqrt_f64)
//   z_t  = (b_t - l.z) / L_tt          (forward substitution of L z = A_S^T y, one row)
//   w    = [-W l; 1] / L_tt            (the new column of W = L'^{-T})
//   x   += z_t w                       (x = W z = (A_S^T A_S)^{-1} A_S^T y)
// Every step is a product over the lanes' entries with no serial triangular
// solve, so the 32 lanes share the float64 work.  W is stored twice, by rows
// (Wr[i*K + p] = W_ip) and by columns (Wc[p*K + i] = W_ip), so that both
// products read consecutive addresses across the lanes.
#pragma once

#include "k_common.cuh"

namespace cs {
namespace {

// 1/sqrt(x) in float64 for x > 0 without the float64 square root and
// division (long sequences on this GPU's narrow float64 unit): the float32
// estimate rsqrtf refined by two Newton-Raphson steps y <- y (3/2 - x y^2 / 2),
// each of which doubles the number of correct bits (about 22 -> 44 -> 53).
// Outside float32's normal range the float64 operations are used instead.
__device__ __forceinline__ double rsqrt_f64(double x) {
    const float xf = (float)x;
    if (!(xf >= 0x1p-125f && xf <= 0x1p125f)) return 1.0 / sqrt(x);
    double y = (double)rsqrtf(xf);
    const double hx = 0.5 * x;
    y = y * fma(-hx * y, y, 1.5);
    y = y * fma(-hx * y, y, 1.5);
    return y;
}

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;   // the same value on every lane (each step adds a commutative pair)
}

// One warp, NP = K/32 entries per lane (entry e of lane q is index q + 32e).
// g[e]: the Gram column entry of that index (0 past t); d, bt as above; W
// (both layouts, K x K), z and x (K) of this signal; coef[0..t] receives x
// as float.  Returns false (the same on every lane) for a dependent atom
// (pivot below 2^-20 d, or NaN), leaving the state untouched.  The caller
// synchronises the warp before other lanes read what this wrote.
template <int NP>
__device__ __forceinline__ bool chol_warp(const int t, const int K, const float (&g)[NP], const double d,
                                          const double bt, double* __restrict__ Wr, double* __restrict__ Wc,
                                          double* __restrict__ z, double* __restrict__ x, float* __restrict__ coef) {
    static_assert(NP == 1 || NP == 2, "K is 32 or 64");
    const int lane = threadIdx.x & 31;
    // l = W^T g: l_p = sum_{i <= p} W_ip g_i, i ascending
    double l[NP];
#pragma unroll
    for (int e = 0; e < NP; ++e) l[e] = 0.0;
    // eight rows' loads are issued before their multiply-adds (the loads
    // are independent; the sums stay in ascending i)
#pragma unroll
    for (int h = 0; h < NP; ++h) {
        const int i1 = min(t, 32 * (h + 1));
        for (int i0 = 32 * h; i0 < i1; i0 += 8) {
            double wv[8][NP];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = i0 + u;
#pragma unroll
                for (int e = h; e < NP; ++e) {
                    const int p = lane + 32 * e;
                    wv[u][e] = (i < i1 && i <= p && p < t) ? Wr[(size_t)i * K + p] : 0.0;
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = i0 + u;
                const double gi = (double)__shfl_sync(0xffffffffu, g[h], i & 31);
#pragma unroll
                for (int e = h; e < NP; ++e) {
                    const int p = lane + 32 * e;
                    if (i < i1 && i <= p && p < t) l[e] = fma(wv[u][e], gi, l[e]);
                }
            }
        }
    }
    double ssq = 0.0, lz = 0.0;
#pragma unroll
    for (int e = 0; e < NP; ++e) {
        const int p = lane + 32 * e;
        if (p < t) {
            ssq = fma(l[e], l[e], ssq);
            lz = fma(l[e], z[p], lz);
        }
    }
    ssq = warp_sum_f64(ssq);
    lz = warp_sum_f64(lz);
    const double piv = d - ssq;
    if (!(piv > 0x1p-20 * d)) return false;
    const double rinv = rsqrt_f64(piv);    // 1 / L_tt
    const double zt = (bt - lz) * rinv;
    // u = W l: u_i = sum_{p >= i} W_ip l_p, p ascending
    double u[NP];
#pragma unroll
    for (int e = 0; e < NP; ++e) u[e] = 0.0;
#pragma unroll
    for (int h = 0; h < NP; ++h) {
        const int p1 = min(t, 32 * (h + 1));
        for (int p0 = 32 * h; p0 < p1; p0 += 8) {
            double wv[8][NP];
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                const int p = p0 + v;
#pragma unroll
                for (int e = 0; e <= h; ++e) {
                    const int i = lane + 32 * e;
                    wv[v][e] = (p < p1 && i <= p) ? Wc[(size_t)p * K + i] : 0.0;
                }
            }
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                const int p = p0 + v;
                const double lp = __shfl_sync(0xffffffffu, l[h], p & 31);
#pragma unroll
                for (int e = 0; e <= h; ++e) {
                    const int i = lane + 32 * e;
                    if (p < p1 && i <= p) u[e] = fma(wv[v][e], lp, u[e]);
                }
            }
        }
    }
    // the new column of W, and x += z_t w
#pragma unroll
    for (int e = 0; e < NP; ++e) {
        const int i = lane + 32 * e;
        if (i < t) {
            const double w = -u[e] * rinv;
            Wr[(size_t)i * K + t] = w;
            Wc[(size_t)t * K + i] = w;
            const double xi = fma(zt, w, x[i]);
            x[i] = xi;
            coef[i] = (float)xi;
        } else if (i == t) {
            Wr[(size_t)t * K + t] = rinv;
            Wc[(size_t)t * K + t] = rinv;
            z[t] = zt;
            const double xt = zt * rinv;
            x[t] = xt;
            coef[t] = (float)xt;
        }
    }
    return true;
}

// The batched layout: per signal b, W by rows then by columns at
// L + b * 2K^2, z and x at b*K, the Gram column gcol[b*K + i]; status,
// support and n_iter updated in place.  One warp.
template <int NP>
__device__ __forceinline__ void chol_update(const IterArgs& a, const int b) {
    const int lane = threadIdx.x & 31;
    if (a.status[b] >= 0) return;
    const int t = a.n_iter[b];
    const int K = a.kmax;
    float g[NP];
#pragma unroll
    for (int e = 0; e < NP; ++e) {
        const int i = lane + 32 * e;
        g[e] = (i < t) ? a.gcol[(size_t)b * K + i] : 0.f;
    }
    double* Wr = a.L + (size_t)b * 2 * K * K;
    const bool ok = chol_warp<NP>(t, K, g, (double)a.dnorm[b], (double)a.bt[b], Wr, Wr + (size_t)K * K,
                                  a.z + (size_t)b * K, a.x64 + (size_t)b * K, a.coef + (size_t)b * a.k);
    if (lane == 0) {
        if (!ok) {
            a.status[b] = CS_SIG_DEPENDENT;
            a.support[(size_t)b * a.k + t] = -1;
        } else {
            a.n_iter[b] = t + 1;
        }
    }
}

}  // namespace
}  // namespace cs
