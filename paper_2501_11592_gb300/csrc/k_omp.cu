// OMP least squares (Table "s forward block", OMP row: pinv of A(:,Mask)) as
// an incremental float64 Cholesky update, and the residual + stopping test of
// Eq. 2 shared by OMP and CLOMP.  The Cholesky runs one thread per signal so
// that every float64 lane does useful work on a part whose float64 rate is
// low; the residual runs one warp per signal (coalesced column gathers).
#include "k_resid.cuh"

namespace cs {
namespace {

// ---------------------------------------------- OMP: Cholesky update -------
// Row t of L with L L^T = A_S^T A_S:  L[0:t,0:t] l = g,  L_tt = sqrt(d - l.l);
// then z_t = (a_j^T y - l.z)/L_tt and x = L^{-T} z.  float64 throughout.
__global__ void __launch_bounds__(32) k_chol(IterArgs a) {
    pdl_wait();      // no early trigger: the successor launches when this grid completes
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


template <int MCH>
__global__ void __launch_bounds__(256) k_resid(IterArgs a) {
    pdl_wait();
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < a.B; b += nwarps)
        resid_one<MCH>(a, b);
    pdl_trigger();
}

}  // namespace

cudaError_t launch_chol(const IterArgs& a, cudaStream_t s) {
    // one warp per CTA spreads the float64 work over as many SMs as possible
    return launch_pdl(k_chol, dim3(ceil_div(a.B, 32)), dim3(32), 0, s, a);
}


template <int MCH>
void launch_resid_m(const IterArgs& a, cudaStream_t s) {
    const int grid = resident_grid((const void*)k_resid<MCH>, 256, ceil_div(a.B, 8));
    launch_pdl(k_resid<MCH>, dim3(grid), dim3(256), 0, s, a);
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
