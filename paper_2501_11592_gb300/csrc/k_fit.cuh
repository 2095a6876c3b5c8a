// CLOMP coefficient fit in Gram form (one warp per signal, or per unit of
// small-support signals), shared by the stand-alone fit kernel, the fused
// CLOMP update and the persistent solve.
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
// P x KT shared-memory vector; tab: the Adam factor pairs of this fit's
// steps (staged in shared memory or in the global table); tau0: the Adam step
// counter before the fit.
template <int KT, int LPS>
__device__ __forceinline__ void fit_unit(const IterArgs& a, const ClArgs& c, const int u, const int tau0,
                                         float* sh_s_w, const float2* tab) {
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
        const float2 cc = tab[step];
        const float c1 = cc.x, c2 = cc.y;
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
            a.tau[b] = tau0 + c.steps;
            a.n_iter[b] = sz;
        }
    }
}

// Reduction of the RB row partials p[] over the 4 lanes j = lane % 4 of a
// row block; afterwards lane j holds the sum of row RB*i + grid_row(j).
template <int RB>
__device__ __forceinline__ float grid_reduce(float (&p)[RB]) {
    const int j = threadIdx.x & 3;
    if constexpr (RB == 4) {
        // transposing: exchange half of the partials per stage
        const bool up = (j & 2) != 0;
        const float k0 = up ? p[2] : p[0], k1 = up ? p[3] : p[1];
        const float d0 = up ? p[0] : p[2], d1 = up ? p[1] : p[3];
        const float r0 = k0 + __shfl_xor_sync(0xffffffffu, d0, 2);
        const float r1 = k1 + __shfl_xor_sync(0xffffffffu, d1, 2);
        const bool up1 = (j & 1) != 0;
        return (up1 ? r1 : r0) + __shfl_xor_sync(0xffffffffu, up1 ? r0 : r1, 1);
    } else if constexpr (RB == 2) {
        const bool up = (j & 2) != 0;
        const float r = (up ? p[1] : p[0]) + __shfl_xor_sync(0xffffffffu, up ? p[0] : p[1], 2);
        return r + __shfl_xor_sync(0xffffffffu, r, 1);
    } else {
        // RB = 1 or 3: butterfly sums, then lane j picks row j
        float out = 0.f;
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            float v = p[r] + __shfl_xor_sync(0xffffffffu, p[r], 2);
            v += __shfl_xor_sync(0xffffffffu, v, 1);
            out = (r == (RB == 1 ? 0 : j)) ? v : out;
        }
        return out;
    }
}

// Row (within the block of lane (i, j)) whose sum grid_reduce leaves in lane
// j, and whether lane j is the one lane that owns that coordinate.
template <int RB>
__device__ __forceinline__ int grid_row(int j) {
    return RB == 4 ? j : RB == 2 ? (j >> 1) : RB == 1 ? 0 : (j < 3 ? j : 0);
}
template <int RB>
__device__ __forceinline__ bool grid_owner(int j) {
    return RB == 4 ? true : RB == 2 ? ((j & 1) == 0) : RB == 1 ? (j == 0) : (j < 3);
}

// Gram-form Adam fit of signal b by one warp for supports of KT <= 32 atoms
// (KT in {8, 16, 24, 32}, >= the support size).  The gradient G s - b is a
// KT x KT matvec per step; its cost on this machine is the movement of s to
// the lanes, not the FMAs.  So lane (i, j) = (lane / 4, lane % 4) keeps the
// RB x CB block of G (rows RB*i.., columns CB*j.., RB = KT/8, CB = KT/4) in
// registers, reads only the CB entries of s it needs from shared memory, and
// the four lanes of a row block finish the row sums with shuffles.  Each
// coordinate q = RB*i + grid_row(j) is owned (Adam state, update) by one
// lane.  Coordinates beyond the support have zero rows, zero b and zero
// state, so the update leaves them at exactly zero.  coef_copy (optional)
// receives the coefficients as well; support_size (optional) overrides the
// one-new-atom size n_iter + 1.
template <int KT>
__device__ __forceinline__ void fit_grid(const IterArgs& a, const ClArgs& c, const int b, const int tau0,
                                         float* sh_s_w, const float2* tab, float* coef_copy = nullptr,
                                         const int support_size = 0) {
    static_assert(KT % 8 == 0 && KT >= 8 && KT <= 32, "fit_grid: KT in {8, 16, 24, 32}");
    constexpr int RB = KT / 8, CB = KT / 4, CP = CB / 2;
    const int lane = threadIdx.x & 31, i = lane >> 2, j = lane & 3;
    if (b >= a.B || a.status[b] >= 0) return;
    const int sz = support_size > 0 ? support_size : a.n_iter[b] + 1;
    const int K = a.kmax;
    const float* Gb = a.G + (size_t)b * K * K;
    unsigned long long gp[RB][CP];
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        const int row = RB * i + r;
#pragma unroll
        for (int cp = 0; cp < CP; ++cp) {
            const int col = CB * j + 2 * cp;
            const float g0 = (row < sz && col < sz) ? Gb[(size_t)row * K + col] : 0.f;
            const float g1 = (row < sz && col + 1 < sz) ? Gb[(size_t)row * K + col + 1] : 0.f;
            gp[r][cp] = pack2(g0, g1);
        }
    }
    const bool own = grid_owner<RB>(j);
    const int q = RB * i + grid_row<RB>(j);
    const bool on = own && q < sz;
    float s = on ? a.coef[(size_t)b * a.k + q] : 0.f;
    float mo = (on && !c.reset) ? a.am[(size_t)b * K + q] : 0.f;
    float ve = (on && !c.reset) ? a.av[(size_t)b * K + q] : 0.f;
    const float bb = on ? a.bvec[(size_t)b * K + q] : 0.f;
    const float omb1 = 1.f - c.beta1, omb2 = 1.f - c.beta2;
#pragma unroll 2
    for (int step = 0; step < c.steps; ++step) {
        if (own) sh_s_w[q] = s;
        __syncwarp();
        unsigned long long sp[CP];
        if constexpr (CB % 4 == 0) {
#pragma unroll
            for (int h = 0; h < CB / 4; ++h) {
                const float4 v = *reinterpret_cast<const float4*>(&sh_s_w[CB * j + 4 * h]);
                sp[2 * h] = pack2(v.x, v.y);
                sp[2 * h + 1] = pack2(v.z, v.w);
            }
        } else {
#pragma unroll
            for (int h = 0; h < CP; ++h) {
                const float2 v = *reinterpret_cast<const float2*>(&sh_s_w[CB * j + 2 * h]);
                sp[h] = pack2(v.x, v.y);
            }
        }
        __syncwarp();
        float pr[RB];
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            unsigned long long acc = 0ull;
#pragma unroll
            for (int cp = 0; cp < CP; ++cp) acc = ffma2(gp[r][cp], sp[cp], acc);
            float lo, hi;
            unpack2(acc, lo, hi);
            pr[r] = lo + hi;
        }
        const float gq = grid_reduce<RB>(pr) - bb;
        const float2 cc = tab[step];
        const float c1 = cc.x, c2 = cc.y;
        mo = fmaf(c.beta1, mo, omb1 * gq);
        ve = fmaf(c.beta2, ve, omb2 * gq * gq);
        // sqrt(v) as v * rsqrt(v) (0 stays 0), approximate reciprocal
        const float rt = ve * rsqrtf(fmaxf(ve, 1e-37f));
        s -= c1 * mo * rcp_approx(fmaf(rt, c2, c.eps));
    }
    if (on) {
        a.coef[(size_t)b * a.k + q] = s;
        if (coef_copy) coef_copy[q] = s;
        a.am[(size_t)b * K + q] = mo;
        a.av[(size_t)b * K + q] = ve;
    }
    if (lane == 0) {
        a.tau[b] = tau0 + c.steps;
        a.n_iter[b] = sz;
    }
}

// Stage this fit's Adam factor pairs (lr/(1-b1^tau), 1/sqrt(1-b2^tau)) for the
// steps tau0+1 .. tau0+steps (call from every thread, then __syncthreads);
// returns the staged copy, or the global table when it is too long.
__device__ __forceinline__ const float2* stage_adam(const ClArgs& c, float2* sh_tab) {
    if (c.steps > kAdamStaged) return c.tab + c.tau0;
    for (int i = threadIdx.x; i < c.steps; i += blockDim.x) sh_tab[i] = c.tab[c.tau0 + i];
    return sh_tab;
}

}  // namespace
}  // namespace cs
