// Selection step of one OMP / CLOMP iteration for one signal (one warp),
// shared by the stand-alone selection kernel and the fused CLOMP update.
#pragma once

#include "k_common.cuh"

namespace cs {
namespace {

// Append atom bj as the (t+1)-th support atom of signal b (one warp): the
// support entry and, when the fit needs them, the new Gram row / column and
// A_S^T y entry (OMP: gcol, dnorm, bt for the Cholesky update; CLOMP Gram
// form: G and bvec).  y: the signal, row-sliced like load_row.
template <int MCH>
__device__ __forceinline__ void append_atom(const IterArgs& a, const int b, const int t, const int bj,
                                            const float4 (&y)[MCH]) {
    const int lane = threadIdx.x & 31;
    if (lane == 0) a.support[(size_t)b * a.k + t] = bj;
    if (a.need_gcol || a.need_gram) {
        float4 aj[MCH];
        load_row<MCH>(a.A32 + (size_t)bj * a.mp, a.mp, aj);
        float dd = 0.f, by = 0.f;
#pragma unroll
        for (int c = 0; c < MCH; ++c) {
            dd += dot4(aj[c], aj[c]);
            by += dot4(aj[c], y[c]);
        }
        dd = warp_sum(dd);
        by = warp_sum(by);
        const int* sup = a.support + (size_t)b * a.k;
        const float* garow = a.GA ? a.GA + (size_t)bj * a.n : nullptr;
        if (garow) dd = garow[bj];     // same arithmetic as the other Gram entries
        for (int i0 = 0; i0 < t; i0 += 32) {
            const int i = i0 + lane;
            const int ji = (i < t) ? sup[i] : -1;
            const float g = garow ? (ji >= 0 ? garow[ji] : 0.f) : warp_dots32<MCH>(a.A32, a.mp, ji, aj);
            if (i < t) {
                if (a.need_gcol) a.gcol[(size_t)b * a.kmax + i] = g;
                if (a.need_gram) {
                    float* G = a.G + (size_t)b * a.kmax * a.kmax;
                    G[(size_t)t * a.kmax + i] = g;
                    G[(size_t)i * a.kmax + t] = g;
                }
            }
        }
        if (lane == 0) {
            a.dnorm[b] = dd;
            a.bt[b] = by;
            if (a.need_gram) {
                a.G[((size_t)b * a.kmax + t) * a.kmax + t] = dd;
                a.bvec[(size_t)b * a.kmax + t] = by;
            }
        }
    }
}

template <int MCH>
__device__ __forceinline__ void select_one(const IterArgs& a, const int b) {
    const int lane = threadIdx.x & 31;
    if (a.status[b] >= 0) return;
    const int t = a.n_iter[b];
    const uint32_t* msk = a.mask + (size_t)b * a.nw;

    float4 r[MCH];
    load_row<MCH>(a.R32 + (size_t)b * a.mp, a.mp, r);

    float bv = -1.f;
    int bj = -1;
    const int ncand = a.nch * a.topc;
    const float* cv = a.cand_val + (size_t)b * ncand;
    const int* ci = a.cand_idx + (size_t)b * ncand;

    if (a.prec == CS_CORR_FP32) {
        // exact float32 argmax: one (|c|, atom) per atom tile
        for (int e = lane; e < ncand; e += 32) {
            const int j = ci[e];
            const float v = cv[e];
            if (cand_better(v, j, bv, bj)) { bv = v; bj = j; }
        }
        warp_argmax(bv, bj);
    } else {
        // low-precision candidates (the two best atoms of every 16-atom group,
        // bf16 |c|): merge to the 8 best (larger |c|, then lower index) and
        // re-score those in float32.
        // bit q of `taken` marks candidate e = 32 q + lane as already merged.
        // Up to 128 candidates (n <= 1024) are held in registers, more are
        // re-read from L1 in every round.
        constexpr int PLR = 4;
        uint32_t taken = 0;
        int mine[kTopcMax];
        if (ncand <= 32 * PLR) {
            float lvv[PLR];
            int ljj[PLR];
#pragma unroll
            for (int q = 0; q < PLR; ++q) {
                const int e = q * 32 + lane;
                lvv[q] = e < ncand ? cv[e] : -1.f;
                ljj[q] = e < ncand ? ci[e] : -1;
            }
#pragma unroll
            for (int rk = 0; rk < kTopcMax; ++rk) {
                float lv = -1.f;
                int lj = -1, lq = 0;
#pragma unroll
                for (int q = 0; q < PLR; ++q)
                    if (!((taken >> q) & 1u) && cand_better(lvv[q], ljj[q], lv, lj)) {
                        lv = lvv[q]; lj = ljj[q]; lq = q;
                    }
                float wv = lv;
                int wj = lj;
                warp_argmax(wv, wj);
                mine[rk] = wj;
                if (wj >= 0 && wj == lj) taken |= 1u << lq;
            }
        } else {
#pragma unroll
            for (int rk = 0; rk < kTopcMax; ++rk) {
                float lv = -1.f;
                int lj = -1, lq = -1;
                for (int q = 0, e = lane; e < ncand; ++q, e += 32) {
                    if ((taken >> q) & 1u) continue;
                    const float v = cv[e];
                    const int j = ci[e];
                    if (cand_better(v, j, lv, lj)) { lv = v; lj = j; lq = q; }
                }
                float wv = lv;
                int wj = lj;
                warp_argmax(wv, wj);
                mine[rk] = wj;
                if (wj >= 0 && wj == lj) taken |= 1u << lq;
            }
        }
        // float32 re-score of the merged candidates: loads of all 8 columns
        // first, then one warp sum each
        {
            float part[kTopcMax];
#pragma unroll
            for (int rk = 0; rk < kTopcMax; ++rk) {
                part[rk] = 0.f;
                const int j = mine[rk];
                if (j >= 0) {
                    const float4* col = reinterpret_cast<const float4*>(a.A32 + (size_t)j * a.mp);
#pragma unroll
                    for (int c = 0; c < MCH; ++c) {
                        const int i4 = c * 32 + lane;
                        if (i4 * 4 < a.mp) part[rk] += dot4(col[i4], r[c]);
                    }
                }
            }
#pragma unroll
            for (int rk = 0; rk < kTopcMax; ++rk) {
                const float v = fabsf(warp_sum(part[rk]));
                if (cand_better(v, mine[rk], bv, bj)) { bv = v; bj = mine[rk]; }
            }
        }
        // Certificate.  For every atom |c_bf16 - c| <= delta (bf16 rounding
        // of both operands, 2u + u^2 with u = 2^-8; a generous m 2^-22 for the
        // tensor-core fp32 accumulation; m 2^-23 for the fp32 re-score; times
        // ||a||_max ||r||; FP8: see below).  An atom that was not re-scored can only beat the
        // float32 winner if its bf16 |c| exceeds bv - delta: such "suspects"
        // are candidates ranked 9th or lower above that threshold, and the
        // other atoms of any group whose third value (cand_bound) is above
        // it.  Suspects are re-scored in float32; usually there are none.
        const float rn = a.res_norm[b];
        float delta;
        if (a.prec == CS_CORR_FP8) {
            // FP8: with the quantisation-error norms of the operands,
            // |c8 - c| <= ||a - sa A8|| ||sr R8|| + ||a|| ||r - sr R8||
            //            + m (2^-22 + 2^-23) ||sa A8|| ||sr R8||
            // (accumulation, the two scalings, the fp32 re-score), where
            // ||sa A8|| <= max||a|| + ea_max and ||sr R8|| <= ||r|| + er.
            const float ea = *a.ea_max, er = a.er[b], cm = *a.colnorm_max;
            delta = (ea * (rn + er) + cm * er + (float)a.m * (0x1p-22f + 0x1p-23f) * (cm + ea) * (rn + er)) * 1.01f;
        } else {
            delta = (0x1p-7f + 0x1p-16f + (float)a.m * (0x1p-22f + 0x1p-23f)) * (*a.colnorm_max) * rn * 1.01f;
        }
        const float theta = bv - delta;
        bool any_suspect = false;
        for (int q = 0, e0 = 0; e0 < ncand; ++q, e0 += 32) {
            const int e = e0 + lane;
            const int jq = (e < ncand && !((taken >> q) & 1u) && cv[e] > theta) ? ci[e] : -1;
            if (__any_sync(FULL, jq >= 0)) {
                any_suspect = true;
                float v = fabsf(warp_dots32<MCH>(a.A32, a.mp, jq, r));
                int jj = jq;
                warp_argmax(v, jj);
                if (cand_better(v, jj, bv, bj)) { bv = v; bj = jj; }
            }
        }
        const int ngroups = a.nch * (a.topc / 2);     // two candidates per 16-atom group
        const float* cb = a.cand_bound + (size_t)b * ngroups;
        for (int g0 = 0; g0 < ngroups; g0 += 32) {
            const int g = g0 + lane;
            unsigned sus = __ballot_sync(FULL, g < ngroups && cb[g] > theta);
            while (sus) {
                any_suspect = true;
                const int gg = g0 + __ffs(sus) - 1;
                sus &= sus - 1;
                const int j = gg * kTcGroup + (lane & (kTcGroup - 1));
                const bool ok = lane < kTcGroup && j < a.n && !((msk[j >> 5] >> (j & 31)) & 1u);
                float v = fabsf(warp_dots32<MCH>(a.A32, a.mp, ok ? j : -1, r));
                int jj = ok ? j : -1;
                warp_argmax(v, jj);
                if (cand_better(v, jj, bv, bj)) { bv = v; bj = jj; }
            }
        }
        if (any_suspect && lane == 0) atomicAdd(&a.counters[0], 1u);
    }

    if (bj < 0) {   // nothing left to select
        if (lane == 0) a.status[b] = CS_SIG_MAX_ITER;
        return;
    }
    if (lane == 0) a.mask[(size_t)b * a.nw + (bj >> 5)] |= (1u << (bj & 31));
    float4 y[MCH];
    load_row<MCH>(a.Y32 + (size_t)b * a.mp, a.mp, y);
    append_atom<MCH>(a, b, t, bj, y);
}

}  // namespace
}  // namespace cs
