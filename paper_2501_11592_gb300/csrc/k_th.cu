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
//     each brings its Gram row and column (from A^T A) and a_j^T y.  The
//     atoms taken (at most 32) are listed by one scan -- after a bisection
//     of the cut when more than 32 pass -- sorted in registers and appended
//     together;
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

// Number of unselected atoms of one signal with |c_j| >= f; when cv is
// given, the first 32 of them (in atom order) are written to cv / cj.
__device__ __forceinline__ int th_scan(int n, const float* __restrict__ crow, const uint32_t* mrow, float f,
                                       float* cv, int* cj) {
    const int lane = threadIdx.x & 31;
    int cnt = 0;
    for (int jb = 0; jb < n; jb += 32) {
        const int jj = jb + lane;
        const uint32_t mw = mrow[jb >> 5];
        const float v = (jj < n && !((mw >> lane) & 1u)) ? fabsf(crow[jj]) : -1.f;
        const bool hit = v >= f;
        const uint32_t bal = __ballot_sync(FULL, hit);
        if (cv) {
            const int pos = cnt + __popc(bal & ((1u << lane) - 1u));
            if (hit && pos < 32) {
                cv[pos] = v;
                cj[pos] = jj;
            }
        }
        cnt += __popc(bal);
    }
    return cnt;
}

// Bitonic sort of one (|c|, atom) pair per lane across the warp: largest
// |c| first, the lower atom on ties, empty entries (atom -1) last.
__device__ __forceinline__ void warp_sort_best_first(float& v, int& j) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int d = k >> 1; d > 0; d >>= 1) {
            const float ov = __shfl_xor_sync(FULL, v, d);
            const int oj = __shfl_xor_sync(FULL, j, d);
            const bool lower = (lane & d) == 0;
            const bool best_first = (lane & k) == 0;   // this block's direction (k = 32: the whole warp)
            const bool swap = (lower == best_first) ? cand_better(ov, oj, v, j) : cand_better(v, j, ov, oj);
            if (swap) {
                v = ov;
                j = oj;
            }
        }
    }
}

// Append the nnew atoms held by lanes 0..nnew-1 (my_j) as support entries
// t0 .. t0+nnew-1 of signal b, in lane order: bitset, support, a_j^T y (32
// dot products at once), and the new rows / columns of the support's Gram
// matrix, gathered from A^T A.
template <int MCH>
__device__ __forceinline__ void th_append_batch(const IterArgs& a, int b, int t0, int nnew, int my_j,
                                                const float4 (&y)[MCH], uint32_t* mrow) {
    const int lane = threadIdx.x & 31;
    int* sup = a.support + (size_t)b * a.k;
    if (lane < nnew) {
        sup[t0 + lane] = my_j;
        atomicOr(&mrow[my_j >> 5], 1u << (my_j & 31));
    }
    const float by = warp_dots32<MCH>(a.A32, a.mp, lane < nnew ? my_j : -1, y);
    __syncwarp();   // the support entries, for the gathers below
    const int t1 = t0 + nnew;
    const int si = (lane < t1) ? sup[lane] : 0;
    float* G = a.G + (size_t)b * a.kmax * a.kmax;
    for (int q = 0; q < nnew; ++q) {
        const int jq = __shfl_sync(FULL, my_j, q);
        if (lane < t1) {
            const float g = a.GA[(size_t)jq * a.n + si];
            G[(size_t)(t0 + q) * a.kmax + lane] = g;              // row of the new atom (incl. the new block)
            if (lane < t0) G[(size_t)lane * a.kmax + t0 + q] = g;  // mirror into the earlier rows
        }
    }
    if (lane < nnew) a.bvec[(size_t)b * a.kmax + t0 + lane] = by;
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

// Blocks per SM the register budget is sized for: at m <= 256, seven blocks
// (28 signal warps) keep a 4096-signal batch on the GPU in one wave.
template <int MCH>
constexpr int th_min_blocks() { return MCH <= 2 ? 7 : 1; }

template <int MCH>
__global__ void __launch_bounds__(32 * TH_WARPS, th_min_blocks<MCH>()) k_clomp_th(IterArgs a, ClArgs c, const float* __restrict__ C,
                                                            int ldc, int iter) {
    __shared__ __align__(16) float sh_s[TH_WARPS][32];
    __shared__ float2 sh_tab[kAdamStaged];
    __shared__ float sh_cv[TH_WARPS][32];   // the warp's threshold list: |c| and atom
    __shared__ int sh_cj[TH_WARPS][32];
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
        // The atoms at or above the threshold, listed in one scan.  When more
        // than 32 pass, the ones this iteration takes (at most k - t <= 32,
        // largest first) are the largest of all unselected atoms: bisect a
        // higher cut tau (on the float bit pattern, which orders
        // non-negative floats) until between k - t and 32 atoms reach it,
        // and list those.
        const int room = a.k - t;
        float* cv = sh_cv[w];
        int* cj = sh_cj[w];
        int cnt = th_scan(a.n, crow, mrow, floor, cv, cj);
        if (cnt > 32) {
            uint32_t lo = __float_as_uint(floor), hi = __float_as_uint(M);
            int chi = th_scan(a.n, crow, mrow, M, nullptr, nullptr);
            bool found = chi <= 32 && chi >= room;
            while (chi <= 32 && !found && hi - lo > 1u) {
                const uint32_t mid = lo + ((hi - lo) >> 1);
                const int cm = th_scan(a.n, crow, mrow, __uint_as_float(mid), nullptr, nullptr);
                if (cm > 32) {
                    lo = mid;
                } else {
                    hi = mid;
                    chi = cm;
                    found = cm >= room;
                }
            }
            // (no such cut only when more than 32 - room atoms tie exactly:
            // then one warp argmax per atom)
            cnt = found ? th_scan(a.n, crow, mrow, __uint_as_float(hi), cv, cj) : -1;
        }
        __syncwarp();
        if (cnt >= 0) {
            // sort best-first and append the first min(cnt, room) at once
            float v = lane < cnt ? cv[lane] : -1.f;
            int jj = lane < cnt ? cj[lane] : -1;
            warp_sort_best_first(v, jj);
            const int nnew = min(cnt, room);
            th_append_batch<MCH>(a, b, t, nnew, jj, y, mrow);
            t += nnew;
            __syncwarp();
        } else {
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
    return a.need_gram && a.G != nullptr && a.GA != nullptr && a.k <= 32 && a.kmax >= a.k &&
           row_chunks(a.mp) <= kMaxRowChunks;
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
