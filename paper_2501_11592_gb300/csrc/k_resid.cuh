// Residual r = y - A_S s_S, its norm and the stopping test of Eq. 2 for one
// signal (one warp), shared by the stand-alone residual kernel and the fused
// CLOMP update.
#pragma once

#include "k_common.cuh"

namespace cs {
namespace {

// ------------------------------------------------ residual + stop test -----
// r <- r - A_S s_S for the t support atoms `sup` with coefficients `x` (one
// warp; r enters holding y, row-sliced like load_row).
template <int MCH>
__device__ __forceinline__ void resid_vector_from(const IterArgs& a, const int t, float4 (&r)[MCH],
                                                  const int* sup, const float* x) {
    const int lane = threadIdx.x & 31;
    // Columns in selection order (the oracle's order).  Lane q loads support
    // index and coefficient q once; the indices are then broadcast by
    // shuffles, so up to 4 columns' loads are in flight before their FMAs.
    for (int q0 = 0; q0 < t; q0 += 32) {
        const int qn = min(32, t - q0);
        const int my_j = (lane < qn) ? sup[q0 + lane] : 0;
        const float my_x = (lane < qn) ? x[q0 + lane] : 0.f;
        for (int u0 = 0; u0 < qn; u0 += 4) {
            float4 v[4][MCH];
            float xq[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = __shfl_sync(0xffffffffu, my_j, u0 + u);
                xq[u] = __shfl_sync(0xffffffffu, my_x, u0 + u);
                const float4* col = reinterpret_cast<const float4*>(a.A32 + (size_t)j * a.mp);
#pragma unroll
                for (int c = 0; c < MCH; ++c) {
                    const int i4 = c * 32 + lane;
                    v[u][c] = (u0 + u < qn && i4 * 4 < a.mp) ? col[i4] : make_float4(0.f, 0.f, 0.f, 0.f);
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

// r <- r - A_S s_S for signal b, support and coefficients from its outputs.
template <int MCH>
__device__ __forceinline__ void resid_vector(const IterArgs& a, const int b, const int t, float4 (&r)[MCH]) {
    resid_vector_from<MCH>(a, t, r, a.support + (size_t)b * a.k, a.coef + (size_t)b * a.k);
}

// Stopping test of Eq. 2 after t atoms (lane 0 of the signal's warp).
__device__ __forceinline__ void stop_test(const IterArgs& a, const int b, const int t, const float rho) {
    a.res_norm[b] = rho;
    if ((double)rho <= a.tol) a.status[b] = CS_SIG_REACHED_TOL;
    else if (t >= a.k) a.status[b] = CS_SIG_REACHED_K;
    else if (t >= a.iters) a.status[b] = CS_SIG_MAX_ITER;
}

template <int MCH>
__device__ __forceinline__ void resid_one(const IterArgs& a, const int b) {
    const int lane = threadIdx.x & 31;
    if (a.status[b] >= 0) return;
    const int t = a.n_iter[b];
    float4 r[MCH];
    load_row<MCH>(a.Y32 + (size_t)b * a.mp, a.mp, r);
    resid_vector<MCH>(a, b, t, r);
    float ss = 0.f;
    float4* R = reinterpret_cast<float4*>(a.R32 + (size_t)b * a.mp);
#pragma unroll
    for (int c = 0; c < MCH; ++c) {
        const int i4 = c * 32 + lane;
        if (i4 * 4 < a.mp) {
            R[i4] = r[c];
            ss += dot4(r[c], r[c]);
        }
    }
    if (a.R16) {
        // bf16 copy for the tensor-core correlation (row stride mh >= mp rounded to 8)
        __nv_bfloat16* R16 = a.R16 + (size_t)b * a.mh;
#pragma unroll
        for (int c = 0; c < MCH; ++c) {
            const int i = (c * 32 + lane) * 4;
            if (i < a.mp) {
                __nv_bfloat162 lo = __floats2bfloat162_rn(r[c].x, r[c].y);
                __nv_bfloat162 hi = __floats2bfloat162_rn(r[c].z, r[c].w);
                *reinterpret_cast<__nv_bfloat162*>(R16 + i) = lo;
                *reinterpret_cast<__nv_bfloat162*>(R16 + i + 2) = hi;
            }
        }
    }
    if (a.R8) {
        // FP8 copy for the FP8 tensor-core correlation: per-signal scale and
        // quantisation-error norm; entries past mp keep the set-up's zeros
        float amax = 0.f;
#pragma unroll
        for (int c = 0; c < MCH; ++c)
            if ((c * 32 + lane) * 4 < a.mp)
                amax = fmaxf(fmaxf(fabsf(r[c].x), fabsf(r[c].y)), fmaxf(fmaxf(fabsf(r[c].z), fabsf(r[c].w)), amax));
        const float sc = fp8_scale(warp_max(amax));
        float e2 = 0.f;
        uint8_t* R8 = a.R8 + (size_t)b * a.mq;
#pragma unroll
        for (int c = 0; c < MCH; ++c) {
            const int i = (c * 32 + lane) * 4;
            if (i < a.mp) {
                const float v[4] = {r[c].x, r[c].y, r[c].z, r[c].w};
                uint32_t packed = 0;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const uint32_t q = fp8_e4m3(v[u] / sc);
                    const float d = v[u] - sc * fp8_e4m3_value(q);
                    e2 = fmaf(d, d, e2);
                    packed |= q << (8 * u);
                }
                *reinterpret_cast<uint32_t*>(R8 + i) = packed;
            }
        }
        e2 = warp_sum(e2);
        if (lane == 0) {
            a.sr[b] = sc;
            a.er[b] = sqrtf(e2);
        }
    }
    ss = warp_sum(ss);
    if (lane == 0) stop_test(a, b, t, sqrtf(ss));
}

}  // namespace
}  // namespace cs
