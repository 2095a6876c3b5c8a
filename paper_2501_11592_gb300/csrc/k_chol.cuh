// OMP least squares (Table "s forward block", OMP row: pinv of A(:,Mask)) as
// an incremental float64 Cholesky update of one signal, shared by the
// one-thread-per-signal kernel and the fused small-batch solve
// (internal header).
#pragma once

#include "k_common.cuh"

namespace cs {
namespace {

// Row t of L with L L^T = A_S^T A_S:  L[0:t,0:t] l = g,  L_tt = sqrt(d - l.l);
// then z_t = (a_j^T y - l.z)/L_tt and x = L^{-T} z.  float64 throughout; one
// thread.  A pivot below 2^-20 d marks a dependent atom (status 3).  L (K x K),
// z and x of the signal sit at element strides ls and vs (the batched layout
// interleaves signals; a single CTA keeps its signal's in shared memory).
__device__ __forceinline__ void chol_update_at(const IterArgs& a, const int b, double* L, const size_t ls,
                                               double* zv, double* xv, const size_t vs) {
    if (a.status[b] >= 0) return;
    const int t = a.n_iter[b];
    const size_t B = (size_t)a.B;
    const int K = a.kmax;
#define LAT(i, p) L[((size_t)(i) * K + (p)) * ls]
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
    for (int i = 0; i < t; ++i) zt -= LAT(t, i) * zv[(size_t)i * vs];
    zt /= ltt;
    zv[(size_t)t * vs] = zt;
    for (int i = t; i >= 0; --i) {
        double s = zv[(size_t)i * vs];
        for (int p = i + 1; p <= t; ++p) s -= LAT(p, i) * xv[(size_t)p * vs];
        const double xi = s / LAT(i, i);
        xv[(size_t)i * vs] = xi;
        a.coef[(size_t)b * a.k + i] = (float)xi;
    }
    a.n_iter[b] = t + 1;
#undef LAT
}

// The batched layout: L[(i*K + p)*B + b], z[i*B + b], x[i*B + b].
__device__ __forceinline__ void chol_update(const IterArgs& a, const int b) {
    chol_update_at(a, b, a.L + b, (size_t)a.B, a.z + b, a.x64 + b, (size_t)a.B);
}

}  // namespace
}  // namespace cs
