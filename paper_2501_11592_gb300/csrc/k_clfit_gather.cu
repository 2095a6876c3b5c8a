// CLOMP coefficient fit in the literal gather form: every Adam step runs the
// forward r = y - A_S s and the adjoint -A_S^T r through the gathered support
// columns (Methods, "Coefficients learning on OMP", structure 1).
#include "k_common.cuh"

namespace cs {
namespace {

constexpr int GF_MAXT = 256;              // threads per signal, at most
constexpr int GF_MAXW = GF_MAXT / 32;

// Transposed sum over the warp of N partials (N = 8, 16 or 32), held in
// lane-permuted slots when N = 32: slot i of lane l holds partial i ^ (l & 16).
// Afterwards lane l holds in v[0] the warp's total of partial l mod N.  With
// that storage the first halving stage (lanes 16 apart) sends the upper half
// of the slots and keeps the lower half in every lane, with no selects; the
// later stages exchange by lane parity; the butterfly stages then add the
// copies held by lanes that differ above bit log2(N).
template <int N>
__device__ __forceinline__ void warp_reduce_scatter_perm(float (&v)[N]) {
    const unsigned lane = threadIdx.x & 31u;
    if constexpr (N == 32) {
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] += __shfl_xor_sync(FULL, v[i + 16], 16);
    }
#pragma unroll
    for (int off = (N == 32 ? 8 : N / 2); off >= 1; off >>= 1) {
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < off; ++i) {
            const float send = upper ? v[i] : v[i + off];
            const float keep = upper ? v[i + off] : v[i];
            v[i] = keep + __shfl_xor_sync(FULL, send, off);
        }
    }
#pragma unroll
    for (int off = N; off < 32; off <<= 1) v[0] += __shfl_xor_sync(FULL, v[0], off);
}

// ------------------------------------------ CLOMP: gather-form Adam fit ----
// One CTA of NTH = 32 * nw threads per signal; thread i holds rows i, i + NTH,
// ... (RPT of them) of the gathered A_S in registers as column pairs, so the
// support columns are read once per fit and every step is on chip:
//   forward   r_i = y_i - sum_q a_iq s_q      (paired fp32 FMAs, s broadcast
//                                              from the warp's shared copy)
//   adjoint   p_q = sum_i a_iq r_i             (paired FMAs over the thread's
//                                              rows, a transposed sum over
//                                              the warp, then over the warps
//                                              in shared memory)
//   Adam      on g_q = -p_q, by every warp for its own copy of s, so a step
//             needs one CTA barrier (the cross-warp partials are double-
//             buffered: a warp can only overwrite a buffer after the next
//             barrier, which every warp reaches after reading it).
// With 32 partials per transposed sum, lane l keeps its columns in the order
// q ^ perm, perm = l & 16, which takes the selects out of the sum's widest
// stage; each warp then keeps two copies of s (the second in the order of
// perm = 16, padded by four floats so that the copies fall in different
// banks), and a lane reads its own copy as float4 at fixed offsets from one
// base.  KT (8, 16, 32 or 64) >= the support size: coordinates beyond the
// support have zero columns and zero state and stay at exactly zero.
template <int KT, int RPT>
__global__ void __launch_bounds__(GF_MAXT) k_clfit_gather(IterArgs a, ClArgs c) {
    constexpr int KP = KT / 2;                 // column pairs
    constexpr int NR = KT < 32 ? KT : 32;      // partials per transposed sum
    constexpr int NQ = KT / NR;                // coordinates held per lane (1, or 2 for KT = 64)
    constexpr int NC = NR == 32 ? 2 : 1;       // permuted copies of s per warp
    constexpr int CS = KT + 4;                 // floats per copy
    __shared__ __align__(16) float sh_s[GF_MAXW][NC * CS];
    __shared__ float red[2][GF_MAXW][KT];
    __shared__ int sh_j[KT];
    pdl_wait();
    const int b = blockIdx.x;
    if (a.status[b] >= 0) return;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int nth = blockDim.x, nwarp = nth >> 5;
    const int sz = a.n_iter[b] + 1;
    const int K = a.kmax;
    const int perm = NR == 32 ? (lane & 16) : 0;   // slot p of this lane holds column p ^ perm (per 32)

    for (int q = tid; q < KT; q += nth) sh_j[q] = (q < sz) ? a.support[(size_t)b * a.k + q] : -1;
    __syncthreads();
    unsigned long long ap[RPT][KP];            // (a_i,2p, a_i,2p+1) of row i = tid + r * NTH
    float yv[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int i = tid + r * nth;
        const bool on = i < a.m;
        yv[r] = on ? a.Y32[(size_t)b * a.mp + i] : 0.f;
#pragma unroll
        for (int p = 0; p < KP; ++p) {
            const int q0 = (2 * p) ^ perm;     // perm is even: q0 + 1 = (2p + 1) ^ perm
            const int j0 = sh_j[q0], j1 = sh_j[q0 + 1];
            const float a0 = (on && j0 >= 0) ? a.A32[(size_t)j0 * a.mp + i] : 0.f;
            const float a1 = (on && j1 >= 0) ? a.A32[(size_t)j1 * a.mp + i] : 0.f;
            ap[r][p] = pack2(a0, a1);
        }
    }
    // coordinate q = (lane mod NR) + NR h of this lane; lanes >= KT (KT < 32)
    // hold copies of lanes below
    float s[NQ], mo[NQ], ve[NQ];
#pragma unroll
    for (int h = 0; h < NQ; ++h) {
        const int q = (lane % NR) + NR * h;
        const bool on = q < sz;
        s[h] = on ? a.coef[(size_t)b * a.k + q] : 0.f;
        mo[h] = (on && !c.reset) ? a.am[(size_t)b * K + q] : 0.f;
        ve[h] = (on && !c.reset) ? a.av[(size_t)b * K + q] : 0.f;
    }
    float* my_s = sh_s[w];
    const float* my_copy = my_s + (perm >> 4) * CS;
    // copy c holds s_q at (q ^ 16c) within each block of NR coordinates
    auto put_s = [&]() {
        if (lane < NR)
#pragma unroll
            for (int cpy = 0; cpy < NC; ++cpy)
#pragma unroll
                for (int h = 0; h < NQ; ++h) my_s[cpy * CS + (lane ^ (16 * cpy)) + NR * h] = s[h];
    };
    put_s();
    __syncwarp();
    const float omb1 = 1.f - c.beta1, omb2 = 1.f - c.beta2;

    for (int step = 0; step < c.steps; ++step) {
        // forward: the residual of this thread's rows (two paired partial
        // sums per row, s read four entries at a time)
        unsigned long long acc[RPT][2];
#pragma unroll
        for (int r = 0; r < RPT; ++r) acc[r][0] = acc[r][1] = 0ull;
#pragma unroll
        for (int p4 = 0; p4 < KT; p4 += 4) {
            const float4 sv = *reinterpret_cast<const float4*>(&my_copy[p4]);
            const unsigned long long s01 = pack2(sv.x, sv.y), s23 = pack2(sv.z, sv.w);
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
                acc[r][0] = ffma2(ap[r][p4 / 2], s01, acc[r][0]);
                acc[r][1] = ffma2(ap[r][p4 / 2 + 1], s23, acc[r][1]);
            }
        }
        float res[RPT];
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            float l0, h0, l1, h1;
            unpack2(acc[r][0], l0, h0);
            unpack2(acc[r][1], l1, h1);
            res[r] = yv[r] - ((l0 + h0) + (l1 + h1));
        }
        // adjoint: this thread's partials of A_S^T r
        unsigned long long pp[KP];
#pragma unroll
        for (int p = 0; p < KP; ++p) pp[p] = 0ull;
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            const unsigned long long rr = pack2(res[r], res[r]);
#pragma unroll
            for (int p = 0; p < KP; ++p) pp[p] = ffma2(ap[r][p], rr, pp[p]);
        }
        float gsum[NQ];
#pragma unroll
        for (int h = 0; h < NQ; ++h) {
            float part[NR];
#pragma unroll
            for (int p = 0; p < NR / 2; ++p) unpack2(pp[h * NR / 2 + p], part[2 * p], part[2 * p + 1]);
            warp_reduce_scatter_perm<NR>(part);
            gsum[h] = part[0];
        }
        if (nwarp > 1) {
            float* rb = &red[step & 1][0][0];
            if (lane < NR)
#pragma unroll
                for (int h = 0; h < NQ; ++h) rb[w * KT + lane + NR * h] = gsum[h];
            __syncthreads();
#pragma unroll
            for (int h = 0; h < NQ; ++h) {
                float g = 0.f;
#pragma unroll
                for (int ww = 0; ww < GF_MAXW; ++ww)
                    if (ww < nwarp) g += rb[ww * KT + (lane % NR) + NR * h];
                gsum[h] = g;
            }
        }
        const float2 cc = c.tab[c.tau0 + step];
        const float c1 = cc.x, c2 = cc.y;
#pragma unroll
        for (int h = 0; h < NQ; ++h) {
            const float g = -gsum[h];
            if ((lane % NR) + NR * h < sz) {
                mo[h] = fmaf(c.beta1, mo[h], omb1 * g);
                ve[h] = fmaf(c.beta2, ve[h], omb2 * g * g);
                // sqrt(v) as v * rsqrt(v) (0 stays 0), approximate reciprocal
                const float rt = ve[h] * rsqrtf(fmaxf(ve[h], 1e-37f));
                s[h] -= c1 * mo[h] * rcp_approx(fmaf(rt, c2, c.eps));
            }
        }
        __syncwarp();                          // every lane has read its copy this step
        put_s();
        __syncwarp();
    }
    if (w == 0 && lane < NR) {
#pragma unroll
        for (int h = 0; h < NQ; ++h) {
            const int q = lane + NR * h;
            if (q < sz) {
                a.coef[(size_t)b * a.k + q] = s[h];
                a.am[(size_t)b * K + q] = mo[h];
                a.av[(size_t)b * K + q] = ve[h];
            }
        }
        if (lane == 0) {
            a.tau[b] = c.tau0 + c.steps;
            a.n_iter[b] = sz;
        }
    }
}


}  // namespace

cudaError_t launch_clfit_gather(const IterArgs& a, const ClArgs& c, int iter, cudaStream_t s) {
    // every live signal holds exactly `iter` atoms before this fit, so the
    // support after it has iter + 1 <= KT atoms
    const int sz = iter + 1;
    const int kt = sz <= 8 ? 8 : sz <= 16 ? 16 : sz <= 32 ? 32 : 64;
    if (kt > a.kmax) return cudaErrorInvalidValue;
    // rows per thread: up to 128 / KT (at most 4; more rows spill A_S out
    // of the registers), fewer for short columns, more when m needs them to
    // stay within GF_MAXT threads
    int rpt = std::min(4, 128 / kt);
    while (rpt > 1 && a.m <= 32 * (rpt / 2)) rpt /= 2;
    while (rpt < 4 && ceil_div(a.m, rpt) > GF_MAXT) rpt *= 2;
    if (ceil_div(a.m, rpt) > GF_MAXT) return cudaErrorInvalidValue;   // m > 4 * GF_MAXT: not an on-chip size
    const int nth = std::min(GF_MAXT, round_up(ceil_div(a.m, rpt), 32));
#define CS_GATHER_LAUNCH(KT_)                                                                     \
    do {                                                                                          \
        if (rpt == 1) launch_pdl(k_clfit_gather<KT_, 1>, dim3(a.B), dim3(nth), 0, s, a, c);       \
        else if (rpt == 2) launch_pdl(k_clfit_gather<KT_, 2>, dim3(a.B), dim3(nth), 0, s, a, c);  \
        else launch_pdl(k_clfit_gather<KT_, 4>, dim3(a.B), dim3(nth), 0, s, a, c);                \
    } while (0)
    switch (kt) {
        case 8: CS_GATHER_LAUNCH(8); break;
        case 16: CS_GATHER_LAUNCH(16); break;
        case 32: CS_GATHER_LAUNCH(32); break;
        default: CS_GATHER_LAUNCH(64); break;
    }
#undef CS_GATHER_LAUNCH
    return cudaGetLastError();
}


}  // namespace cs
