// IHT (Methods, Table "s forward block", IHT row), the paper's comparison
// method, on the same residual-injection layer: per iteration the float32
// correlation C = A^T R of the live signals (k_corr_fp32), then one warp per
// signal
//   * forms u = s + t c for every atom (s dense, kept per signal) in shared
//     memory;
//   * finds the k-th largest |u| from its float32 bit pattern (non-negative
//     floats order like their bits) by a radix select: four passes of
//     256-bin histograms over 8-bit digits, most significant first, each
//     over the keys that match the digits found so far;
//   * keeps the atoms above it and, of those equal to it, the lowest
//     indices -- H_k with the lowest-index tie rule -- written in ascending
//     index order with their values u_j, and clears the atoms it dropped;
//   * forms the residual r = y - A_S s_S, its norm and the stopping rule
//     (tol, or the iteration limit R).
#include <algorithm>

#include "k_resid.cuh"

namespace cs {
namespace {

constexpr int IH_WARPS = 4;   // warps per CTA, each with n floats and a 256-bin histogram of shared memory
constexpr int IH_BINS = 256;

template <int MCH>
__global__ void __launch_bounds__(32 * IH_WARPS) k_iht_update(IterArgs a, const float* __restrict__ C, int ldc,
                                                             float* __restrict__ sd, float step, int it) {
    extern __shared__ float sh_u[];   // [IH_WARPS][n], then [IH_WARPS][IH_BINS] counts
    pdl_wait();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float* u = sh_u + (size_t)w * a.n;
    unsigned* hist = reinterpret_cast<unsigned*>(sh_u + (size_t)IH_WARPS * a.n) + w * IH_BINS;
    const int nwarps = gridDim.x * IH_WARPS;
    const unsigned lt = (1u << lane) - 1u;
    for (int b = blockIdx.x * IH_WARPS + w; b < a.B; b += nwarps) {
        if (a.status[b] >= 0) continue;
        float* sb = sd + (size_t)b * a.n;
        const float* cb = C + (size_t)b * ldc;
        for (int j = lane; j < a.n; j += 32) u[j] = fmaf(step, cb[j], sb[j]);
        __syncwarp();
        // T = the k-th largest key (the largest value with #{key >= T} >= k),
        // one 8-bit digit per pass: among the keys whose higher digits equal
        // T's, the digit d with #{digit > d} < need <= #{digit >= d}
        unsigned T = 0, hi_mask = 0;
        int rem = a.k;                                     // rank of T among the keys still matching
        for (int shift = 24; shift >= 0; shift -= 8) {
            for (int q = lane; q < IH_BINS; q += 32) hist[q] = 0u;
            __syncwarp();
            for (int j = lane; j < a.n; j += 32) {
                const unsigned key = __float_as_uint(u[j]) & 0x7fffffffu;
                if ((key & hi_mask) == T) atomicAdd(&hist[(key >> shift) & 255u], 1u);
            }
            __syncwarp();
            // lane l holds bins 8l .. 8l + 7; counts above each lane's bins by a suffix scan
            unsigned c[8], sum = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                c[q] = hist[8 * lane + q];
                sum += c[q];
            }
            unsigned incl = sum;                           // keys in this lane's bins and above
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned v = __shfl_down_sync(FULL, incl, o);
                if (lane + o < 32) incl += v;
            }
            const unsigned above = incl - sum;             // keys in the bins of higher lanes
            // the lane whose bins hold the rem-th largest key: above < rem <= above + sum
            const bool mine = above < (unsigned)rem && (unsigned)rem <= above + sum;
            const unsigned owner = __ballot_sync(FULL, mine);
            const int L = __ffs(owner) - 1;
            int d = 0;
            unsigned gt = 0;                               // keys with a larger digit
            if (lane == L) {
                unsigned acc = above;
                for (int q = 7; q >= 0; --q) {
                    if (acc + c[q] >= (unsigned)rem) {
                        d = 8 * lane + q;
                        break;
                    }
                    acc += c[q];
                }
                gt = acc;
            }
            d = __shfl_sync(FULL, d, L);
            gt = __shfl_sync(FULL, gt, L);
            T |= (unsigned)d << shift;
            hi_mask |= 255u << shift;
            rem -= (int)gt;
            __syncwarp();
        }
        int gt = 0;
        for (int j = lane; j < a.n; j += 32) gt += (__float_as_uint(u[j]) & 0x7fffffffu) > T ? 1 : 0;
        const int need = a.k - __reduce_add_sync(FULL, gt);   // ties at T to keep, lowest index first
        // the previous support (k <= 64: two per lane), cleared from s
        int* sup = a.support + (size_t)b * a.k;
        float* cf = a.coef + (size_t)b * a.k;
        const int o0 = lane < a.k ? sup[lane] : -1;
        const int o1 = lane + 32 < a.k ? sup[lane + 32] : -1;
        __syncwarp();
        if (o0 >= 0) sb[o0] = 0.f;
        if (o1 >= 0) sb[o1] = 0.f;
        __syncwarp();
        // the kept atoms in ascending index order
        int pos = 0, ties = 0;
        for (int j0 = 0; j0 < a.n; j0 += 32) {
            const int j = j0 + lane;
            const unsigned key = j < a.n ? (__float_as_uint(u[j]) & 0x7fffffffu) : 0u;
            const bool big = j < a.n && key > T;
            const bool tie = j < a.n && key == T;
            const unsigned eq = __ballot_sync(FULL, tie);
            const bool keep = big || (tie && ties + __popc(eq & lt) < need);
            const unsigned km = __ballot_sync(FULL, keep);
            if (keep) {
                const int q = pos + __popc(km & lt);
                sup[q] = j;
                cf[q] = u[j];
                sb[j] = u[j];
            }
            pos += __popc(km);
            ties += __popc(eq);
        }
        __syncwarp();
        // residual, norm, stopping rule
        float4 r[MCH];
        load_row<MCH>(a.Y32 + (size_t)b * a.mp, a.mp, r);
        resid_vector_from<MCH>(a, a.k, r, sup, cf);
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
        ss = warp_sum(ss);
        if (lane == 0) {
            const float rho = sqrtf(ss);
            a.res_norm[b] = rho;
            a.n_iter[b] = it + 1;
            if ((double)rho <= a.tol) a.status[b] = CS_SIG_REACHED_TOL;
            else if (it + 1 >= a.iters) a.status[b] = CS_SIG_MAX_ITER;
        }
        __syncwarp();
    }
    pdl_trigger();
}

template <int MCH>
cudaError_t launch_m(const IterArgs& a, const float* C, int ldc, float* sd, float step, int it, cudaStream_t s) {
    const size_t smem = sizeof(float) * IH_WARPS * (size_t)a.n + sizeof(unsigned) * IH_WARPS * IH_BINS;
    const cudaError_t attr =
        set_smem_limit((const void*)k_iht_update<MCH>,
                       (int)(sizeof(float) * IH_WARPS * kIhtMaxN + sizeof(unsigned) * IH_WARPS * IH_BINS));
    if (attr != cudaSuccess) return attr;
    const int grid = std::min(ceil_div(a.B, IH_WARPS), 65535);   // warps stride over the signals
    return launch_pdl(k_iht_update<MCH>, dim3(grid), dim3(32 * IH_WARPS), smem, s, a, C, ldc, sd, step, it);
}

}  // namespace

bool iht_supported(const IterArgs& a) {
    return a.n <= kIhtMaxN && a.k <= 64 && row_chunks(a.mp) <= kMaxRowChunks;
}

cudaError_t launch_iht_update(const IterArgs& a, const float* C, int ldc, float* sd, float step, int it,
                              cudaStream_t s) {
    if (!iht_supported(a)) return cudaErrorNotSupported;
    switch (row_chunks(a.mp)) {
        case 1: return launch_m<1>(a, C, ldc, sd, step, it, s);
        case 2: return launch_m<2>(a, C, ldc, sd, step, it, s);
        case 3:
        case 4: return launch_m<4>(a, C, ldc, sd, step, it, s);
        default: return launch_m<8>(a, C, ldc, sd, step, it, s);
    }
}

}  // namespace cs
