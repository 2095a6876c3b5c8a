// Per-signal kernels of one OMP / CLOMP iteration (everything except the
// correlation GEMM): selection, coefficient fit, residual and stopping test.
//
// Paper steps (Methods, "Coefficients learning on OMP"; Eq. 2):
//   select  -- argmax |A^T r| over unselected atoms, Mask |= new atom;
//   fit     -- OMP: least squares on A(:,Mask) (Table "s forward block");
//              CLOMP: Adam on 1/2 ||y - A(s .* Mask)||^2, s learnable;
//   resid   -- r = y - A_S s_S, stop on |S| = k, ||r|| <= tol or R iterations.
// Parallel layout: one warp per signal for the float32 gathers over m, one
// thread per signal for the float64 triangular solves (so every float64 lane
// does useful work on a part whose float64 rate is low), one CTA per signal
// for the gather-form CL fit.
#include "cs_internal.cuh"

namespace cs {
namespace {

constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------- set-up --

// Copy A (caller layout, lda) into the padded float32 layout and, when A16 is
// given, its bf16 copy; record max_j ||a_j||_2.  One warp per column.
__global__ void k_prep_A(const float* __restrict__ A, int lda, int m, int n, int mp, int mh,
                         float* __restrict__ A32, __nv_bfloat16* __restrict__ A16,
                         float* colnorm_max) {
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= n) return;
    const float* a = A + (size_t)j * lda;
    float ss = 0.f;
    for (int i = lane; i < mp; i += 32) {
        const float v = (i < m) ? a[i] : 0.f;
        A32[(size_t)j * mp + i] = v;
        ss = fmaf(v, v, ss);
    }
    if (A16) {
        for (int i = lane; i < mh; i += 32)
            A16[(size_t)j * mh + i] = __float2bfloat16_rn(i < m ? a[i] : 0.f);
    }
    ss = warp_sum(ss);
    if (lane == 0 && colnorm_max) {
        // non-negative floats order like their bit patterns
        atomicMax(reinterpret_cast<unsigned int*>(colnorm_max), __float_as_uint(sqrtf(ss)));
    }
}

// Copy caller residuals (m x B, leading dimension ldr) into the padded
// float32 and/or bf16 row layouts used by the correlation kernels.
__global__ void k_prep_R(const float* __restrict__ R, int ldr, int m, int B, int mp, int mh,
                         float* __restrict__ R32, __nv_bfloat16* __restrict__ R16) {
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= B) return;
    const float* r = R + (size_t)b * ldr;
    if (R32)
        for (int i = lane; i < mp; i += 32) R32[(size_t)b * mp + i] = (i < m) ? r[i] : 0.f;
    if (R16)
        for (int i = lane; i < mh; i += 32) R16[(size_t)b * mh + i] = __float2bfloat16_rn(i < m ? r[i] : 0.f);
}

// Per-signal initial state: r = y, s = 0, empty support, status "running".
__global__ void k_setup(IterArgs a, const float* __restrict__ Y, int ldy, int clomp) {
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= a.B) return;
    const float* y = Y + (size_t)b * ldy;
    float ss = 0.f;
    int finite = 1;
    for (int i = lane; i < a.mp; i += 32) {
        const float v = (i < a.m) ? y[i] : 0.f;
        finite &= isfinite(v) ? 1 : 0;
        a.Y32[(size_t)b * a.mp + i] = v;
        a.R32[(size_t)b * a.mp + i] = v;
        ss = fmaf(v, v, ss);
    }
    if (a.R16)
        for (int i = lane; i < a.mh; i += 32)
            a.R16[(size_t)b * a.mh + i] = __float2bfloat16_rn(i < a.m ? y[i] : 0.f);
    for (int w = lane; w < a.nw; w += 32) a.mask[(size_t)b * a.nw + w] = 0u;
    for (int q = lane; q < a.k; q += 32) {
        a.support[(size_t)b * a.k + q] = -1;
        a.coef[(size_t)b * a.k + q] = 0.f;
    }
    if (clomp) {
        for (int q = lane; q < a.kmax; q += 32) {
            a.am[(size_t)b * a.kmax + q] = 0.f;
            a.av[(size_t)b * a.kmax + q] = 0.f;
        }
    }
    ss = warp_sum(ss);
    finite = __all_sync(FULL, finite);
    if (lane == 0) {
        const float rho = sqrtf(ss);
        a.n_iter[b] = 0;
        a.tau[b] = 0;
        if (!finite) {
            a.status[b] = CS_SIG_NONFINITE;
            a.res_norm[b] = __int_as_float(0x7fffffff);
        } else {
            a.res_norm[b] = rho;
            a.status[b] = ((double)rho <= a.tol) ? CS_SIG_REACHED_TOL : -1;
        }
    }
}

// Adam bias-correction factors for tau = 1..len, evaluated in float64 from
// the float32 hyper-parameters and rounded once:
//   tab[tau-1]       = lr / (1 - beta1^tau)
//   tab[len + tau-1] = 1 / sqrt(1 - beta2^tau)
__global__ void k_adam_table(float* tab, int len, float lr, float beta1, float beta2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    const double tau = (double)(i + 1);
    tab[i] = (float)((double)lr / (1.0 - pow((double)beta1, tau)));
    tab[len + i] = (float)(1.0 / sqrt(1.0 - pow((double)beta2, tau)));
}

// ------------------------------------------------------------- selection --

template <int MCH>
__device__ __forceinline__ void load_row(const float* __restrict__ base, int mp, float4 (&v)[MCH]) {
    const int lane = threadIdx.x & 31;
    const float4* p = reinterpret_cast<const float4*>(base);
#pragma unroll
    for (int c = 0; c < MCH; ++c) {
        const int i4 = c * 32 + lane;
        v[c] = (i4 * 4 < mp) ? p[i4] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// Warp-cooperative dot products of up to 32 columns of A32 (atom index
// held by lane q, -1 = none) with the row-sliced vector x; lane q returns
// the full dot for its column.
template <int MCH>
__device__ __forceinline__ float warp_dots32(const float* __restrict__ A32, int mp, int my_atom,
                                             const float4 (&x)[MCH]) {
    const int lane = threadIdx.x & 31;
    float part[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) {
        const int j = __shfl_sync(FULL, my_atom, q);
        float acc = 0.f;
        if (j >= 0) {
            const float4* col = reinterpret_cast<const float4*>(A32 + (size_t)j * mp);
#pragma unroll
            for (int c = 0; c < MCH; ++c) {
                const int i4 = c * 32 + lane;
                if (i4 * 4 < mp) acc += dot4(col[i4], x[c]);
            }
        }
        part[q] = acc;
    }
    warp_reduce_scatter32(part);
    return part[0];
}

template <int MCH>
__global__ void __launch_bounds__(256) k_select(IterArgs a) {
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= a.B) return;
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
        // low-precision candidates: re-score every listed atom in float32
        for (int e0 = 0; e0 < ncand; e0 += 32) {
            const int e = e0 + lane;
            const int j = (e < ncand) ? ci[e] : -1;
            const float c = warp_dots32<MCH>(a.A32, a.mp, j, r);
            const float v = fabsf(c);
            if (cand_better(v, j, bv, bj)) { bv = v; bj = j; }
        }
        warp_argmax(bv, bj);
        // Certificate: atoms missing from a full list have bf16 |c| at most
        // that list's last entry U; with |c_bf16 - c| <= delta for every atom,
        // no unlisted atom can beat the float32 winner if |c*| > U + delta.
        float U = -1.f;
        for (int ch = lane; ch < a.nch; ch += 32) {
            const int last = ch * a.topc + a.topc - 1;
            if (ci[last] >= 0) U = fmaxf(U, cv[last]);
        }
        U = fmaxf(U, __shfl_xor_sync(FULL, U, 16));
        U = fmaxf(U, __shfl_xor_sync(FULL, U, 8));
        U = fmaxf(U, __shfl_xor_sync(FULL, U, 4));
        U = fmaxf(U, __shfl_xor_sync(FULL, U, 2));
        U = fmaxf(U, __shfl_xor_sync(FULL, U, 1));
        // delta: bf16 rounding of both operands (2u + u^2, u = 2^-8), float32
        // accumulation of m terms (m 2^-22, generous for the tensor-core
        // adder) and the float32 re-score (m 2^-23), times ||a||_max ||r||.
        const float rn = a.res_norm[b];
        const float delta = (0x1p-7f + 0x1p-16f + (float)a.m * (0x1p-22f + 0x1p-23f)) *
                            (*a.colnorm_max) * rn * 1.01f;
        if (U >= 0.f && !(bv - U > delta)) {
            // fallback: exact float32 scan of every unselected atom
            if (lane == 0) atomicAdd(&a.counters[0], 1u);
            for (int j0 = 0; j0 < a.n; j0 += 32) {
                const int j = j0 + lane;
                const bool ok = (j < a.n) && !((msk[j >> 5] >> (j & 31)) & 1u);
                const float c = warp_dots32<MCH>(a.A32, a.mp, ok ? j : -1, r);
                float v = fabsf(c);
                int jj = ok ? j : -1;
                warp_argmax(v, jj);
                if (cand_better(v, jj, bv, bj)) { bv = v; bj = jj; }
            }
        }
    }

    if (bj < 0) {   // nothing left to select
        if (lane == 0) a.status[b] = CS_SIG_MAX_ITER;
        return;
    }
    if (lane == 0) {
        a.support[(size_t)b * a.k + t] = bj;
        a.mask[(size_t)b * a.nw + (bj >> 5)] |= (1u << (bj & 31));
    }

    if (a.need_gcol || a.need_gram) {
        float4 aj[MCH], y[MCH];
        load_row<MCH>(a.A32 + (size_t)bj * a.mp, a.mp, aj);
        load_row<MCH>(a.Y32 + (size_t)b * a.mp, a.mp, y);
        float dd = 0.f, by = 0.f;
#pragma unroll
        for (int c = 0; c < MCH; ++c) {
            dd += dot4(aj[c], aj[c]);
            by += dot4(aj[c], y[c]);
        }
        dd = warp_sum(dd);
        by = warp_sum(by);
        const int* sup = a.support + (size_t)b * a.k;
        for (int i0 = 0; i0 < t; i0 += 32) {
            const int i = i0 + lane;
            const int ji = (i < t) ? sup[i] : -1;
            const float g = warp_dots32<MCH>(a.A32, a.mp, ji, aj);
            if (i < t) {
                if (a.need_gcol) a.gcol[(size_t)i * a.B + b] = g;
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

// ---------------------------------------------- OMP: Cholesky update -------
// Row t of L with L L^T = A_S^T A_S:  L[0:t,0:t] l = g,  L_tt = sqrt(d - l.l);
// then z_t = (a_j^T y - l.z)/L_tt and x = L^{-T} z.  float64 throughout.
__global__ void __launch_bounds__(128) k_chol(IterArgs a) {
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
__global__ void __launch_bounds__(256) k_resid(IterArgs a) {
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= a.B) return;
    if (a.status[b] >= 0) return;
    const int t = a.n_iter[b];
    float4 r[MCH];
    load_row<MCH>(a.Y32 + (size_t)b * a.mp, a.mp, r);
    const int* sup = a.support + (size_t)b * a.k;
    const float* x = a.coef + (size_t)b * a.k;
    for (int q = 0; q < t; ++q) {
        const int j = sup[q];
        const float xq = x[q];
        const float4* col = reinterpret_cast<const float4*>(a.A32 + (size_t)j * a.mp);
#pragma unroll
        for (int c = 0; c < MCH; ++c) {
            const int i4 = c * 32 + lane;
            if (i4 * 4 < a.mp) {
                const float4 v = col[i4];
                r[c].x = fmaf(-v.x, xq, r[c].x);
                r[c].y = fmaf(-v.y, xq, r[c].y);
                r[c].z = fmaf(-v.z, xq, r[c].z);
                r[c].w = fmaf(-v.w, xq, r[c].w);
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

// ------------------------------------------- CLOMP: Gram-form Adam fit -----
// Gradient of 1/2||y - A_S s||^2 written as G s - b with G = A_S^T A_S and
// b = A_S^T y maintained per signal by k_select.  One warp per signal; lane
// q owns coordinates q, q+32 (rows of G in registers).
template <int KMAX>
__global__ void __launch_bounds__(256) k_clfit_gram(IterArgs a, ClArgs c, int iter) {
    constexpr int NQ = KMAX / 32;
    __shared__ __align__(16) float sh_s[8][KMAX];
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int b = blockIdx.x * 8 + w;
    if (b >= a.B) return;
    if (a.status[b] >= 0) return;
    const int t = a.n_iter[b];
    const int sz = t + 1;
    const int K = a.kmax;
    const float* Gb = a.G + (size_t)b * K * K;

    float grow[NQ][KMAX];
    float s[NQ], mo[NQ], ve[NQ], bb[NQ];
#pragma unroll
    for (int h = 0; h < NQ; ++h) {
        const int q = lane + 32 * h;
        const bool on = q < sz;
#pragma unroll
        for (int p = 0; p < KMAX; ++p) grow[h][p] = (on && p < sz) ? Gb[(size_t)q * K + p] : 0.f;
        s[h] = on ? a.coef[(size_t)b * a.k + q] : 0.f;
        mo[h] = (on && !c.reset) ? a.am[(size_t)b * K + q] : 0.f;
        ve[h] = (on && !c.reset) ? a.av[(size_t)b * K + q] : 0.f;
        bb[h] = on ? a.bvec[(size_t)b * K + q] : 0.f;
    }
    int tau = c.reset ? 0 : a.tau[b];
    const float omb1 = 1.f - c.beta1, omb2 = 1.f - c.beta2;
    for (int step = 0; step < c.steps; ++step) {
#pragma unroll
        for (int h = 0; h < NQ; ++h) sh_s[w][lane + 32 * h] = s[h];
        __syncwarp();
        float g[NQ];
#pragma unroll
        for (int h = 0; h < NQ; ++h) g[h] = -bb[h];
#pragma unroll
        for (int p4 = 0; p4 < KMAX; p4 += 4) {
            const float4 sv = *reinterpret_cast<const float4*>(&sh_s[w][p4]);
#pragma unroll
            for (int h = 0; h < NQ; ++h) {
                g[h] = fmaf(grow[h][p4 + 0], sv.x, g[h]);
                g[h] = fmaf(grow[h][p4 + 1], sv.y, g[h]);
                g[h] = fmaf(grow[h][p4 + 2], sv.z, g[h]);
                g[h] = fmaf(grow[h][p4 + 3], sv.w, g[h]);
            }
        }
        __syncwarp();
        ++tau;
        const float c1 = c.tab[tau - 1], c2 = c.tab[c.tab_len + tau - 1];
#pragma unroll
        for (int h = 0; h < NQ; ++h) {
            if (lane + 32 * h < sz) {
                mo[h] = fmaf(c.beta1, mo[h], omb1 * g[h]);
                ve[h] = fmaf(c.beta2, ve[h], omb2 * g[h] * g[h]);
                s[h] -= c1 * mo[h] / fmaf(sqrtf(ve[h]), c2, c.eps);
            }
        }
    }
#pragma unroll
    for (int h = 0; h < NQ; ++h) {
        const int q = lane + 32 * h;
        if (q < sz) {
            a.coef[(size_t)b * a.k + q] = s[h];
            a.am[(size_t)b * K + q] = mo[h];
            a.av[(size_t)b * K + q] = ve[h];
        }
    }
    if (lane == 0) {
        a.tau[b] = tau;
        a.n_iter[b] = sz;
    }
}

// ------------------------------------------ CLOMP: gather-form Adam fit ----
// The literal CL fit: each step forms r = y - A_S s (forward through the
// fixed layer) and g = -A_S^T r (its adjoint), then one Adam step.  One CTA
// per signal; thread i holds rows i, i+NTH, ... of A_S in registers, so the
// gathered columns are read once per iteration and reused for all steps.
template <int KMAX, int RPT>
__global__ void __launch_bounds__(256) k_clfit_gather(IterArgs a, ClArgs c, int iter) {
    constexpr int NQ = KMAX / 32;
    __shared__ __align__(16) float sh_s[KMAX];
    __shared__ float red[8][KMAX];
    __shared__ int sh_j[KMAX];
    const int b = blockIdx.x;
    if (a.status[b] >= 0) return;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int nth = blockDim.x, nwarp = nth >> 5;
    const int t = a.n_iter[b];
    const int sz = t + 1;
    const int K = a.kmax;

    for (int q = tid; q < KMAX; q += nth) {
        sh_j[q] = (q < sz) ? a.support[(size_t)b * a.k + q] : -1;
        sh_s[q] = (q < sz) ? a.coef[(size_t)b * a.k + q] : 0.f;
    }
    __syncthreads();
    float arow[RPT][KMAX];
    float yv[RPT];
#pragma unroll
    for (int rr = 0; rr < RPT; ++rr) {
        const int i = tid + rr * nth;
        const bool on = i < a.m;
        yv[rr] = on ? a.Y32[(size_t)b * a.mp + i] : 0.f;
#pragma unroll
        for (int q = 0; q < KMAX; ++q) {
            const int j = sh_j[q];
            arow[rr][q] = (on && j >= 0) ? a.A32[(size_t)j * a.mp + i] : 0.f;
        }
    }
    float s[NQ], mo[NQ], ve[NQ];
#pragma unroll
    for (int h = 0; h < NQ; ++h) {
        const int q = lane + 32 * h;
        const bool on = (w == 0) && q < sz;
        s[h] = on ? sh_s[q] : 0.f;
        mo[h] = (on && !c.reset) ? a.am[(size_t)b * K + q] : 0.f;
        ve[h] = (on && !c.reset) ? a.av[(size_t)b * K + q] : 0.f;
    }
    int tau = c.reset ? 0 : a.tau[b];
    const float omb1 = 1.f - c.beta1, omb2 = 1.f - c.beta2;

    for (int step = 0; step < c.steps; ++step) {
        float part[NQ][32];
#pragma unroll
        for (int h = 0; h < NQ; ++h)
#pragma unroll
            for (int q = 0; q < 32; ++q) part[h][q] = 0.f;
#pragma unroll
        for (int rr = 0; rr < RPT; ++rr) {
            float res = yv[rr];
#pragma unroll
            for (int q = 0; q < KMAX; ++q) res = fmaf(-arow[rr][q], sh_s[q], res);
#pragma unroll
            for (int h = 0; h < NQ; ++h)
#pragma unroll
                for (int q = 0; q < 32; ++q) part[h][q] = fmaf(arow[rr][32 * h + q], res, part[h][q]);
        }
#pragma unroll
        for (int h = 0; h < NQ; ++h) {
            warp_reduce_scatter32(part[h]);
            red[w][32 * h + lane] = part[h][0];
        }
        __syncthreads();
        ++tau;
        if (w == 0) {
            const float c1 = c.tab[tau - 1], c2 = c.tab[c.tab_len + tau - 1];
#pragma unroll
            for (int h = 0; h < NQ; ++h) {
                const int q = lane + 32 * h;
                float g = 0.f;
                for (int ww = 0; ww < nwarp; ++ww) g += red[ww][q];
                g = -g;
                if (q < sz) {
                    mo[h] = fmaf(c.beta1, mo[h], omb1 * g);
                    ve[h] = fmaf(c.beta2, ve[h], omb2 * g * g);
                    s[h] -= c1 * mo[h] / fmaf(sqrtf(ve[h]), c2, c.eps);
                }
                sh_s[q] = s[h];
            }
        }
        __syncthreads();
    }
    if (w == 0) {
#pragma unroll
        for (int h = 0; h < NQ; ++h) {
            const int q = lane + 32 * h;
            if (q < sz) {
                a.coef[(size_t)b * a.k + q] = s[h];
                a.am[(size_t)b * K + q] = mo[h];
                a.av[(size_t)b * K + q] = ve[h];
            }
        }
        if (lane == 0) {
            a.tau[b] = tau;
            a.n_iter[b] = sz;
        }
    }
}

int row_chunks(int mp) { return ceil_div(mp, 128); }

}  // namespace

cudaError_t launch_prep_A(const float* A, int lda, int m, int n, int mp, int mh, float* A32,
                          __nv_bfloat16* A16, float* colnorm_max, cudaStream_t s) {
    if (colnorm_max) {
        cudaError_t e = cudaMemsetAsync(colnorm_max, 0, sizeof(float), s);
        if (e != cudaSuccess) return e;
    }
    k_prep_A<<<ceil_div(n, 8), 256, 0, s>>>(A, lda, m, n, mp, mh, A32, A16, colnorm_max);
    return cudaGetLastError();
}

cudaError_t launch_prep_R(const float* R, int ldr, int m, int B, int mp, int mh, float* R32,
                          __nv_bfloat16* R16, cudaStream_t s) {
    k_prep_R<<<ceil_div(B, 8), 256, 0, s>>>(R, ldr, m, B, mp, mh, R32, R16);
    return cudaGetLastError();
}

cudaError_t launch_setup(const IterArgs& a, const float* Y, int ldy, int clomp, cudaStream_t s) {
    k_setup<<<ceil_div(a.B, 8), 256, 0, s>>>(a, Y, ldy, clomp);
    return cudaGetLastError();
}

cudaError_t launch_adam_table(float* tab, int len, float lr, float beta1, float beta2,
                              cudaStream_t s) {
    if (len <= 0) return cudaSuccess;
    k_adam_table<<<ceil_div(len, 256), 256, 0, s>>>(tab, len, lr, beta1, beta2);
    return cudaGetLastError();
}

#define CS_DISPATCH_MCH(MP, KERNEL, GRID, BLOCK, STREAM, ...)                     \
    do {                                                                          \
        switch (row_chunks(MP)) {                                                 \
            case 1: KERNEL<1><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__); break;    \
            case 2: KERNEL<2><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__); break;    \
            case 3:                                                               \
            case 4: KERNEL<4><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__); break;    \
            default: KERNEL<8><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__); break;   \
        }                                                                         \
    } while (0)

cudaError_t launch_select(const IterArgs& a, cudaStream_t s) {
    CS_DISPATCH_MCH(a.mp, k_select, ceil_div(a.B, 8), 256, s, a);
    return cudaGetLastError();
}

cudaError_t launch_chol(const IterArgs& a, cudaStream_t s) {
    k_chol<<<ceil_div(a.B, 128), 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_resid(const IterArgs& a, cudaStream_t s) {
    CS_DISPATCH_MCH(a.mp, k_resid, ceil_div(a.B, 8), 256, s, a);
    return cudaGetLastError();
}

cudaError_t launch_clfit_gram(const IterArgs& a, const ClArgs& c, int iter, cudaStream_t s) {
    if (a.kmax <= 32)
        k_clfit_gram<32><<<ceil_div(a.B, 8), 256, 0, s>>>(a, c, iter);
    else
        k_clfit_gram<64><<<ceil_div(a.B, 8), 256, 0, s>>>(a, c, iter);
    return cudaGetLastError();
}

cudaError_t launch_clfit_gather(const IterArgs& a, const ClArgs& c, int iter, cudaStream_t s) {
    const int nth = a.m <= 256 ? round_up(a.m, 32) : 256;
    const int rpt = ceil_div(a.m, nth);
    if (a.kmax <= 32) {
        if (rpt == 1) k_clfit_gather<32, 1><<<a.B, nth, 0, s>>>(a, c, iter);
        else if (rpt == 2) k_clfit_gather<32, 2><<<a.B, nth, 0, s>>>(a, c, iter);
        else k_clfit_gather<32, 4><<<a.B, nth, 0, s>>>(a, c, iter);
    } else {
        if (rpt == 1) k_clfit_gather<64, 1><<<a.B, nth, 0, s>>>(a, c, iter);
        else if (rpt == 2) k_clfit_gather<64, 2><<<a.B, nth, 0, s>>>(a, c, iter);
        else k_clfit_gather<64, 4><<<a.B, nth, 0, s>>>(a, c, iter);
    }
    return cudaGetLastError();
}

}  // namespace cs
