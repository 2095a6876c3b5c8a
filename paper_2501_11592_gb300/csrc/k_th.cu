// Threshold selection rule of CLOMP (Methods: the normalised cut-off
// threshold Th of the selection block, with the multi-atom selection of
// stagewise OMP): in one iteration every unselected atom whose correlation
// reaches Th times the largest one joins the support.
//
// One iteration is the float32 correlation C^T = R^T A of the live signals
// (k_corr_fp32, dense output) followed by this kernel, one warp per signal:
//   * M = max |c_j| over the unselected atoms;
//   * the unselected atoms with |c_j| >= Th * M join the support, largest
//     |c_j| first and the lower atom index on ties, until it holds k atoms;
//     each brings its Gram row and column (from A^T A) and a_j^T y;
//   * the Gram-form Adam fit runs its T steps on all t support atoms, with
//     the solve's single Adam state (the new coordinates start at zero);
//   * the residual r = y - A_S s_S, its norm and the stop test of Eq. 2,
//     iterations counted apart from atoms.
// The selection compares float32 correlations, so it decides in the
// precision of the correlation.
#include "k_fit.cuh"
#include "k_resid.cuh"
#include "k_select.cuh"

namespace cs {
namespace {

constexpr int TH_WARPS = 4;   // signals per block

// Largest unselected |c_j| >= floor of one signal, the lower atom on ties;
// (-1, -1) when there is none.  crow: the signal's correlations; mrow: its
// selected-atom bitset (one word per 32 atoms, the same word for the warp).
__device__ __forceinline__ void th_next(int n, const float* __restrict__ crow, const uint32_t* mrow, float floor,
                                        float& bv, int& bj) {
    const int lane = threadIdx.x & 31;
    float lv = -1.f;
    int lj = -1;
    for (int jb = 0; jb < n; jb += 32) {
        const int j = jb + lane;
        const uint32_t w = mrow[jb >> 5];
        if (j < n && !((w >> lane) & 1u)) {
            const float v = fabsf(crow[j]);
            if (v >= floor && cand_better(v, j, lv, lj)) {
                lv = v;
                lj = j;
            }
        }
    }
    bv = lv;
    bj = lj;
    warp_argmax(bv, bj);
}

__device__ __forceinline__ void th_fit(const IterArgs& a, const ClArgs& c, int b, int sz, float* sv,
                                       const float2* tab) {
    switch (round_up(sz, 8)) {
        case 8: fit_grid<8>(a, c, b, c.tau0, sv, tab, nullptr, sz); break;
        case 16: fit_grid<16>(a, c, b, c.tau0, sv, tab, nullptr, sz); break;
        case 24: fit_grid<24>(a, c, b, c.tau0, sv, tab, nullptr, sz); break;
        default: fit_grid<32>(a, c, b, c.tau0, sv, tab, nullptr, sz); break;
    }
}

template <int MCH>
__global__ void __launch_bounds__(32 * TH_WARPS) k_clomp_th(IterArgs a, ClArgs c, const float* __restrict__ C,
                                                            int ldc, int iter) {
    __shared__ __align__(16) float sh_s[TH_WARPS][32];
    __shared__ float2 sh_tab[kAdamStaged];
    const float2* tab = stage_adam(c, sh_tab);
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x * TH_WARPS + w;
    if (b >= a.B || a.status[b] >= 0) return;
    const float* crow = C + (size_t)b * ldc;
    uint32_t* mrow = a.mask + (size_t)b * a.nw;

    // ---- selection and support append
    float M;
    int j;
    th_next(a.n, crow, mrow, 0.f, M, j);
    if (j < 0) {
        // every atom is in the support already
        if (lane == 0) a.status[b] = CS_SIG_MAX_ITER;
        return;
    }
    const float floor = c.th * M;
    int t = a.n_iter[b];
    {
        float4 y[MCH];
        load_row<MCH>(a.Y32 + (size_t)b * a.mp, a.mp, y);
        while (true) {
            if (lane == 0) mrow[j >> 5] |= 1u << (j & 31);
            append_atom<MCH>(a, b, t, j, y);
            ++t;
            __syncwarp();   // mask word and support entry, for the other lanes
            if (t >= a.k) break;
            float v;
            th_next(a.n, crow, mrow, floor, v, j);
            if (j < 0) break;
        }
    }

    // ---- Gram-form Adam fit on the t support atoms
    th_fit(a, c, b, t, sh_s[w], tab);
    __syncwarp();   // coefficients written by their owner lanes

    // ---- residual, stop test
    float4 r[MCH];
    load_row<MCH>(a.Y32 + (size_t)b * a.mp, a.mp, r);
    resid_vector<MCH>(a, b, t, r);
    float ss = 0.f;
    float4* R = reinterpret_cast<float4*>(a.R32 + (size_t)b * a.mp);
#pragma unroll
    for (int q = 0; q < MCH; ++q) {
        const int i4 = q * 32 + lane;
        if (i4 * 4 < a.mp) {
            R[i4] = r[q];
            ss += dot4(r[q], r[q]);
        }
    }
    const float rho = sqrtf(warp_sum(ss));
    if (lane == 0) {
        a.res_norm[b] = rho;
        if ((double)rho <= a.tol) a.status[b] = CS_SIG_REACHED_TOL;
        else if (t >= a.k) a.status[b] = CS_SIG_REACHED_K;
        else if (iter + 1 >= a.iters) a.status[b] = CS_SIG_MAX_ITER;
    }
}

template <int MCH>
void launch_m(const IterArgs& a, const ClArgs& c, const float* C, int ldc, int iter, cudaStream_t s) {
    k_clomp_th<MCH><<<ceil_div(a.B, TH_WARPS), 32 * TH_WARPS, 0, s>>>(a, c, C, ldc, iter);
}

}  // namespace

bool clomp_th_supported(const IterArgs& a) {
    return a.need_gram && a.G != nullptr && a.k <= 32 && a.kmax >= a.k && row_chunks(a.mp) <= kMaxRowChunks;
}

cudaError_t launch_clomp_th(const IterArgs& a, const ClArgs& c, const float* C, int ldc, int iter, cudaStream_t s) {
    if (!clomp_th_supported(a)) return cudaErrorNotSupported;
    const int rc = row_chunks(a.mp);
    if (rc == 1) launch_m<1>(a, c, C, ldc, iter, s);
    else if (rc == 2) launch_m<2>(a, c, C, ldc, iter, s);
    else if (rc <= 4) launch_m<4>(a, c, C, ldc, iter, s);
    else launch_m<8>(a, c, C, ldc, iter, s);
    return cudaGetLastError();
}

}  // namespace cs
