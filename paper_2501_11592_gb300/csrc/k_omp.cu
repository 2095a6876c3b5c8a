// OMP least squares (Table "s forward block", OMP row: pinv of A(:,Mask)) as
// an incremental float64 Cholesky update, and the residual + stopping test of
// Eq. 2 shared by OMP and CLOMP.  The Cholesky runs one thread per signal so
// that every float64 lane does useful work on a part whose float64 rate is
// low; the residual runs one warp per signal (coalesced column gathers).
#include "k_common.cuh"

namespace cs {
namespace {

// ---------------------------------------------- OMP: Cholesky update -------
// Row t of L with L L^T = A_S^T A_S:  L[0:t,0:t] l = g,  L_tt = sqrt(d - l.l);
// then z_t = (a_j^T y - l.z)/L_tt and x = L^{-T} z.  float64 throughout.
__global__ void __launch_bounds__(32) k_chol(IterArgs a) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= a.B) return;
    if (a.status[b] >= 0) return;
    const int t = a.n_iter[b];
    const size_t B = (size_t)a.B;
    const int K = a.kmax;
    double* L = a.L + b;                 // L[(i*K + p)*B]
#define LAT(i, p) L[((size_t)(i) * K + (p)) * B]
    const double d = (double)a.dnorm[b];
    double ssq = 0.0;
    for (int i = 0; i < t; ++i) {
        double s = (double)a.gcol[(size_t)i * B + b];
        for (int p = 0; p < i; ++p) s -= LAT(i, p) * LAT(t, p);
        const double li = s / LAT(i, i);
        LAT(t, i) = li;
        ssq += li * li;
    }
    const double piv = d - ssq;
    if (!(piv > 0x1p-20 * d)) {     // dependent atom (also catches NaN)
        a.status[b] = CS_SIG_DEPENDENT;
        a.support[(size_t)b * a.k + t] = -1;
        return;
    }
    const double ltt = sqrt(piv);
    LAT(t, t) = ltt;
    double zt = (double)a.bt[b];
    for (int i = 0; i < t; ++i) zt -= LAT(t, i) * a.z[(size_t)i * B + b];
    zt /= ltt;
    a.z[(size_t)t * B + b] = zt;
    for (int i = t; i >= 0; --i) {
        double s = a.z[(size_t)i * B + b];
        for (int p = i + 1; p <= t; ++p) s -= LAT(p, i) * a.x64[(size_t)p * B + b];
        const double xi = s / LAT(i, i);
        a.x64[(size_t)i * B + b] = xi;
        a.coef[(size_t)b * a.k + i] = (float)xi;
    }
    a.n_iter[b] = t + 1;
#undef LAT
}


// ------------------------------------------------ residual + stop test -----
template <int MCH>
__device__ __forceinline__ void resid_one(const IterArgs& a, const int b) {
    const int lane = threadIdx.x & 31;
    if (a.status[b] >= 0) return;
    const int t = a.n_iter[b];
    float4 r[MCH];
    load_row<MCH>(a.Y32 + (size_t)b * a.mp, a.mp, r);
    const int* sup = a.support + (size_t)b * a.k;
    const float* x = a.coef + (size_t)b * a.k;
    // Columns in selection order (the oracle's order).  Lane q loads support
    // index and coefficient q once; the indices are then broadcast by
    // shuffles, so up to 8 columns' loads are in flight before their FMAs.
    for (int q0 = 0; q0 < t; q0 += 32) {
        const int qn = min(32, t - q0);
        const int my_j = (lane < qn) ? sup[q0 + lane] : 0;
        const float my_x = (lane < qn) ? x[q0 + lane] : 0.f;
        for (int u0 = 0; u0 < qn; u0 += 8) {
            float4 v[8][MCH];
            float xq[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
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
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int c = 0; c < MCH; ++c) {
                    r[c].x = fmaf(-v[u][c].x, xq[u], r[c].x);
                    r[c].y = fmaf(-v[u][c].y, xq[u], r[c].y);
                    r[c].z = fmaf(-v[u][c].z, xq[u], r[c].z);
                    r[c].w = fmaf(-v[u][c].w, xq[u], r[c].w);
                }
        }
    }
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
    ss = warp_sum(ss);
    if (lane == 0) {
        const float rho = sqrtf(ss);
        a.res_norm[b] = rho;
        if ((double)rho <= a.tol) a.status[b] = CS_SIG_REACHED_TOL;
        else if (t >= a.k) a.status[b] = CS_SIG_REACHED_K;
        else if (t >= a.iters) a.status[b] = CS_SIG_MAX_ITER;
    }
}


template <int MCH>
__global__ void __launch_bounds__(256) k_resid(IterArgs a) {
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < a.B; b += nwarps)
        resid_one<MCH>(a, b);
}

}  // namespace

cudaError_t launch_chol(const IterArgs& a, cudaStream_t s) {
    // one warp per CTA spreads the float64 work over as many SMs as possible
    k_chol<<<ceil_div(a.B, 32), 32, 0, s>>>(a);
    return cudaGetLastError();
}


template <int MCH>
void launch_resid_m(const IterArgs& a, cudaStream_t s) {
    const int grid = resident_grid((const void*)k_resid<MCH>, 256, ceil_div(a.B, 8));
    k_resid<MCH><<<grid, 256, 0, s>>>(a);
}

cudaError_t launch_resid(const IterArgs& a, cudaStream_t s) {
    switch (row_chunks(a.mp)) {
        case 1: launch_resid_m<1>(a, s); break;
        case 2: launch_resid_m<2>(a, s); break;
        case 3:
        case 4: launch_resid_m<4>(a, s); break;
        default: launch_resid_m<8>(a, s); break;
    }
    return cudaGetLastError();
}


}  // namespace cs
