// OMP least squares (Table "s forward block", OMP row: pinv of A(:,Mask)) as
// an incremental float64 Cholesky update of one signal, shared by the
// one-thread-per-signal kernel and the fused small-batch solve
// (internal header).
#pragma once

#include "k_common.cuh"

namespace cs {
namespace {

// Row t of L with L L^T = A_S^T A_S:  L[0:t,0:t] l = g,  L_tt = sqrt(d - l.l);
// then z_t = (a_j^T y - l.z)/L_tt and x = L^{-T} z, written (as float) to
// coef[0..t].  float64 throughout; one thread.  g_i = g[i * gs]; L (K x K),
// z and x at element strides ls and vs.  Returns false for a dependent atom
// (pivot below 2^-20 d, or NaN), leaving coef untouched.
__device__ __forceinline__ bool chol_core(const int t, const int K, const float* g, const size_t gs,
                                          const double d, const double bt, double* L, const size_t ls,
                                          double* zv, double* xv, const size_t vs, float* coef) {
#define LAT(i, p) L[((size_t)(i) * K + (p)) * ls]
    double ssq = 0.0;
    for (int i = 0; i < t; ++i) {
        double s = (double)g[(size_t)i * gs];
        for (int p = 0; p < i; ++p) s -= LAT(i, p) * LAT(t, p);
        const double li = s / LAT(i, i);
        LAT(t, i) = li;
        ssq += li * li;
    }
    const double piv = d - ssq;
    if (!(piv > 0x1p-20 * d)) return false;
    const double ltt = sqrt(piv);
    LAT(t, t) = ltt;
    double zt = bt;
    for (int i = 0; i < t; ++i) zt -= LAT(t, i) * zv[(size_t)i * vs];
    zt /= ltt;
    zv[(size_t)t * vs] = zt;
    for (int i = t; i >= 0; --i) {
        double s = zv[(size_t)i * vs];
        for (int p = i + 1; p <= t; ++p) s -= LAT(p, i) * xv[(size_t)p * vs];
        const double xi = s / LAT(i, i);
        xv[(size_t)i * vs] = xi;
        coef[i] = (float)xi;
    }
    return true;
#undef LAT
}

// The batched layout: L[(i*K + p)*B + b], z[i*B + b], x[i*B + b], the Gram
// column gcol[i*B + b]; status, support and n_iter updated in place.
__device__ __forceinline__ void chol_update(const IterArgs& a, const int b) {
    if (a.status[b] >= 0) return;
    const int t = a.n_iter[b];
    const size_t B = (size_t)a.B;
    if (!chol_core(t, a.kmax, a.gcol + b, B, (double)a.dnorm[b], (double)a.bt[b], a.L + b, B, a.z + b, a.x64 + b, B,
                   a.coef + (size_t)b * a.k)) {
        a.status[b] = CS_SIG_DEPENDENT;
        a.support[(size_t)b * a.k + t] = -1;
        return;
    }
    a.n_iter[b] = t + 1;
}

}  // namespace
}  // namespace cs
