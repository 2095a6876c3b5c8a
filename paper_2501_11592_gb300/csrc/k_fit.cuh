// CLOMP coefficient fit in Gram form for one unit of P = 32/LPS signals (one
// warp), shared by the stand-alone fit kernel and the fused CLOMP update.
#pragma once

#include "k_common.cuh"

namespace cs {
namespace {

constexpr int kAdamStaged = 256;   // Adam factors staged in shared memory per fit

// Gradient of 1/2||y - A_S s||^2 written as G s - b with G = A_S^T A_S and
// b = A_S^T y maintained per signal by the selection step.  The warp holds
// P = 32/LPS signals, LPS lanes each; lane q of a signal owns coordinates q,
// q+LPS, ... (rows of G in registers, packed in pairs for fp32x2 FMAs).
// KT >= the support size (a multiple of 8, chosen per iteration by the
// host), so the matvec runs over KT columns only.  sh_s_w: this warp's
// P x KT shared-memory vector; sh_c1 / sh_c2: the staged Adam factors.
template <int KT, int LPS>
__device__ __forceinline__ void fit_unit(const IterArgs& a, const ClArgs& c, const int u,
                                         float* sh_s_w, const float* sh_c1, const float* sh_c2,
                                         const bool staged) {
    constexpr int P = 32 / LPS;
    constexpr int NQ = (KT + LPS - 1) / LPS;
    constexpr int KP = KT / 2;
    const int lane = threadIdx.x & 31;
    const int sub = lane / LPS, ql = lane % LPS;
    const int b = u * P + sub;
    const bool live = b < a.B && a.status[b] < 0;
    if (!__any_sync(0xffffffffu, live)) return;
    const int sz = live ? a.n_iter[b] + 1 : 0;
    const int K = a.kmax;
    const float* Gb = a.G + (size_t)(live ? b : 0) * K * K;

    unsigned long long gp[NQ][KP];                // row q of G as (G[q][2p], G[q][2p+1])
    float s[NQ], mo[NQ], ve[NQ], bb[NQ];
#pragma unroll
    for (int h = 0; h < NQ; ++h) {
        const int q = ql + LPS * h;
        const bool on = q < sz;
#pragma unroll
        for (int pp = 0; pp < KP; ++pp) {
            const float g0 = (on && 2 * pp < sz) ? Gb[(size_t)q * K + 2 * pp] : 0.f;
            const float g1 = (on && 2 * pp + 1 < sz) ? Gb[(size_t)q * K + 2 * pp + 1] : 0.f;
            gp[h][pp] = pack2(g0, g1);
        }
        s[h] = on ? a.coef[(size_t)b * a.k + q] : 0.f;
        mo[h] = (on && !c.reset) ? a.am[(size_t)b * K + q] : 0.f;
        ve[h] = (on && !c.reset) ? a.av[(size_t)b * K + q] : 0.f;
        bb[h] = on ? a.bvec[(size_t)b * K + q] : 0.f;
    }
    const float omb1 = 1.f - c.beta1, omb2 = 1.f - c.beta2;
    float* my_s = sh_s_w + sub * KT;
    unsigned long long nb[NQ];                // (-b_q, 0): initial partial sums
#pragma unroll
    for (int h = 0; h < NQ; ++h) nb[h] = pack2(-bb[h], 0.f);
#pragma unroll 2
    for (int step = 0; step < c.steps; ++step) {
#pragma unroll
        for (int h = 0; h < NQ; ++h)
            if (ql + LPS * h < KT) my_s[ql + LPS * h] = s[h];
        __syncwarp();
        // g = G s - b: packed fp32x2 FMAs, two pairs of partial sums per row
        unsigned long long g2[NQ][2];
#pragma unroll
        for (int h = 0; h < NQ; ++h) {
            g2[h][0] = nb[h];
            g2[h][1] = 0ull;
        }
#pragma unroll
        for (int p4 = 0; p4 < KT; p4 += 4) {
            const float4 sv = *reinterpret_cast<const float4*>(&my_s[p4]);
            const unsigned long long s01 = pack2(sv.x, sv.y), s23 = pack2(sv.z, sv.w);
#pragma unroll
            for (int h = 0; h < NQ; ++h) {
                g2[h][0] = ffma2(gp[h][p4 / 2], s01, g2[h][0]);
                g2[h][1] = ffma2(gp[h][p4 / 2 + 1], s23, g2[h][1]);
            }
        }
        __syncwarp();
        const float c1 = staged ? sh_c1[step] : c.tab[c.tau0 + step];
        const float c2 = staged ? sh_c2[step] : c.tab[c.tab_len + c.tau0 + step];
        // Coordinates beyond the support have zero rows, zero b and zero
        // state, so the update leaves them at exactly zero: no masking.
#pragma unroll
        for (int h = 0; h < NQ; ++h) {
            float g0, g1, g2v, g3;
            unpack2(g2[h][0], g0, g1);
            unpack2(g2[h][1], g2v, g3);
            const float gq = (g0 + g1) + (g2v + g3);
            mo[h] = fmaf(c.beta1, mo[h], omb1 * gq);
            ve[h] = fmaf(c.beta2, ve[h], omb2 * gq * gq);
            // sqrt(v) as v * rsqrt(v) (0 stays 0), approximate reciprocal
            const float rt = ve[h] * rsqrtf(fmaxf(ve[h], 1e-37f));
            s[h] -= c1 * mo[h] * rcp_approx(fmaf(rt, c2, c.eps));
        }
    }
    if (live) {
#pragma unroll
        for (int h = 0; h < NQ; ++h) {
            const int q = ql + LPS * h;
            if (q < sz) {
                a.coef[(size_t)b * a.k + q] = s[h];
                a.am[(size_t)b * K + q] = mo[h];
                a.av[(size_t)b * K + q] = ve[h];
            }
        }
        if (ql == 0) {
            a.tau[b] = c.tau0 + c.steps;
            a.n_iter[b] = sz;
        }
    }
}

// Stage this fit's Adam factors lr/(1-b1^tau), 1/sqrt(1-b2^tau) for the steps
// tau0+1 .. tau0+steps (call from every thread, then __syncthreads).
__device__ __forceinline__ bool stage_adam(const ClArgs& c, float* sh_c1, float* sh_c2) {
    const bool staged = c.steps <= kAdamStaged;
    if (staged)
        for (int i = threadIdx.x; i < c.steps; i += blockDim.x) {
            sh_c1[i] = c.tab[c.tau0 + i];
            sh_c2[i] = c.tab[c.tab_len + c.tau0 + i];
        }
    return staged;
}

}  // namespace
}  // namespace cs
