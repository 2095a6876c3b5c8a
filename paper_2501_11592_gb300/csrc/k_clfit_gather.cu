// CLOMP coefficient fit in the literal gather form: every Adam step runs the
// forward r = y - A_S s and the adjoint -A_S^T r through the gathered support
// columns (Methods, "Coefficients learning on OMP", structure 1).
#include "k_common.cuh"

namespace cs {
namespace {

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
    pdl_wait();
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
    int tau = c.tau0;
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
            const float2 cc = c.tab[tau - 1];
            const float c1 = cc.x, c2 = cc.y;
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


}  // namespace

cudaError_t launch_clfit_gather(const IterArgs& a, const ClArgs& c, int iter, cudaStream_t s) {
    const int nth = a.m <= 256 ? round_up(a.m, 32) : 256;
    const int rpt = ceil_div(a.m, nth);
    if (a.kmax <= 32) {
        if (rpt == 1) launch_pdl(k_clfit_gather<32, 1>, dim3(a.B), dim3(nth), 0, s, a, c, iter);
        else if (rpt == 2) launch_pdl(k_clfit_gather<32, 2>, dim3(a.B), dim3(nth), 0, s, a, c, iter);
        else launch_pdl(k_clfit_gather<32, 4>, dim3(a.B), dim3(nth), 0, s, a, c, iter);
    } else {
        if (rpt == 1) launch_pdl(k_clfit_gather<64, 1>, dim3(a.B), dim3(nth), 0, s, a, c, iter);
        else if (rpt == 2) launch_pdl(k_clfit_gather<64, 2>, dim3(a.B), dim3(nth), 0, s, a, c, iter);
        else launch_pdl(k_clfit_gather<64, 4>, dim3(a.B), dim3(nth), 0, s, a, c, iter);
    }
    return cudaGetLastError();
}


}  // namespace cs
