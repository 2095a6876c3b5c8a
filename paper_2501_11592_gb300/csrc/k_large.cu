// OMP and CLOMP for instances beyond the on-chip kernels: supports of up to
// kLargeMaxK atoms and measurements of up to kLargeMaxM rows (the flattened
// images of Results, "Evaluation with synthetic 2D data", solved as one long
// 1-D signal, and the large members of uneven batches).  A batch of signals
// sharing A runs as a sequence of grid-wide kernels per iteration of Eq. 2's
// greedy loop, each signal with its own sparsity k:
//
//   correlation   c~ = A^T r: A's copy (bf16, or float32) streamed from HBM
//                 in 32 KB tiles through a shared-memory ring, r in shared
//                 memory, float32 accumulation (k_lg_corr_tma); or, for
//                 eight or more bf16 signals, one tcgen05 GEMM over bf16
//                 residuals (k_lg_corr_mma); each signal's largest
//                 unselected |c~| is folded into a per-signal maximum;
//   selection     every unselected atom with |c~_j| >= max - 2 delta (delta
//                 bounds |c~_j - c_j| for every atom, see below) is re-scored
//                 in float32 against the caller's A by a whole CTA, and the
//                 largest |c_j| (lowest atom on ties) wins through one 64-bit
//                 atomicMax of (value bits, ~atom) -- the float32 argmax over
//                 all unselected atoms;
//   Gram column   g_i = a_{S_i}^T a_j, ||a_j||^2 and a_j^T y in float32, each
//                 dot product split into 2048-row segments summed in segment
//                 order by the warp that completes the entry;
//   least squares the float64 update of W = L^{-T} of k_chol.cuh -- l = W^T g,
//   (OMP)         pivot, z_t, u = W l, the new column of W, x += z_t w --
//                 both products as partial sums over 32-entry chunks, added
//                 in chunk order by the warp that completes a block
//                 (k_lg_lpiv, k_lg_uupd);
//   CL fit        (CLOMP, Gram form) row t of G = A_S^T A_S and b_t = a_j^T y
//   (CLOMP)       from the same Gram column, then the T Adam steps on
//                 1/2 ||y - A_S s||^2 with gradient G s - b, one cooperative
//                 launch per iteration whose CTAs keep their rows of G in
//                 shared memory (see k_lgc_fit), or one launch per step;
//   residual      r = y - A_S x (x as float32), partial sums over chunks of
//                 32 support atoms added in chunk order, ||r|| from per-block
//                 sums, the stopping rule of Eq. 2 (k_lg_resid).
// The reductions across CTAs are last-arriver reductions: arrival counters
// (reset by the last arriver) and a fixed summation order, no CTA waiting
// for another, so a solve is deterministic.
//
// Certificate.  With bf16 A (unit roundoff 2^-8) and float32 accumulation
// of N1 = m/32 + 13 terms per lane plus the warp tree, and the float32
// re-score summing N2 = m/1024 + 16 terms per thread plus the block tree,
// for every atom |c~_j - c_j^{fp32}| <= delta =
//   (2^-8 (1 + g1) + g1 + g2) max_j ||a_j|| ||r||,  g = N 2^-24 (1.01 margin),
// so the atom whose re-scored |c| is largest has |c~| >= max|c~| - 2 delta.
// The float32 path drops the 2^-8 term; the GEMM form (both operands bf16)
// uses 2^-7 + 2^-16 and m 2^-22 for the tensor core's accumulation.
#include <algorithm>
#include <map>
#include <vector>

#include "k_common.cuh"
#include "k_tc.cuh"

namespace cs {
namespace {

constexpr int LG_SEG = 2048;           // rows per partial Gram dot product
constexpr int LG_LC = 32;              // inner-index chunk of the float64 products
constexpr int LG_RQ = 32;              // support atoms per residual partial sum
constexpr int LG_RESCORE_MIN_CTAS = 16;   // CTAs per signal re-scoring candidates: at least this,
                                          // else two per SM shared by the chunk's signals
// Correlation: A's copy (bf16, or float32) in tiles of 64 atoms x 256 (bf16)
// or 128 (float32) rows, 32 KB each, one bulk copy per tile, streamed through
// a ring of shared-memory stages
constexpr int LG_TA = 64;
constexpr int LG_TILE_BYTES = 32 * 1024;
template <typename T>
__host__ __device__ constexpr int lg_tr() { return LG_TILE_BYTES / (LG_TA * (int)sizeof(T)); }
constexpr int LG_TMA_CONSUMERS = 8;                       // warps, eight atoms each
constexpr int LG_TMA_THREADS = 32 * (LG_TMA_CONSUMERS + 1);
constexpr int LG_TMA_MAX_STAGES = 6;
constexpr unsigned LG_ERR_CORR = 64u;                     // a wait of the correlation's ring gave up
// Many signals sharing A (bf16): the correlation as a tcgen05 GEMM, M = 128
// atoms, N = up to 256 signals, K in chunks of 64 through a TMA ring
constexpr int LG_MMA_MIN_SIGNALS = 8;
constexpr int LG_MMA_MAXN = 256;
constexpr int LG_MMA_KCH = 64;
constexpr int LG_MMA_ATILE = 128 * 128;                   // 128 atoms x 128 bytes
constexpr int LG_MMA_MAX_STAGES = 8;
constexpr int LG_MMA_THREADS = 128;
constexpr int LG_MMA_CFG = 8;                             // its configuration index
constexpr unsigned LG_ERR_MMA = 128u;                     // a wait of the GEMM correlation gave up

// Per-signal state (Bl signals, K = largest k rounded up to 32, mp = m
// rounded up to 8, NSEG = ceil(m / LG_SEG), LCH = ceil(K / LG_LC),
// RCH = ceil(K / LG_RQ)).
struct LgState {
    int m, n, lda, mp, K, nseg, lch, rch, Bl, nb, bf16;
    int mpt, nc, njb;               // tiles: rows padded to the tile height, row chunks, atom blocks of 64
    int nsm, smem_optin;            // the device's SMs and per-CTA shared-memory limit
    int mma, mpk;                   // correlation as a tensor-core GEMM (bf16, many signals); rows to 64
    const __nv_bfloat16* Ak;        // mma: bf16 copy of A in 16 KB tiles [n/128][mpk/64] of 128 atoms x 64
                                    // K values, each the 128-byte-swizzled shared-memory image of the
                                    // tile (rows >= m and atoms >= n zero)
    __nv_bfloat16* R16;             // mma: [Bl][mpk] bf16 copy of the residuals (rows >= m zero)
    double tol;
    const float* A;                 // caller's A (float32, leading dimension lda)
    const void* At;                 // [njb][nc][64][TR] copy of A in tiles (bf16, TR = 256; or float32,
                                    // TR = 128): tile (jb, ic) holds rows TR ic .. TR ic + TR - 1 of
                                    // atoms 64 jb .. 64 jb + 63, atom-major; rows >= m and atoms >= n
                                    // are zero
    int* cblk;                      // [Bl] next atom block per pass of the correlation
    const float* colmax;            // max_j ||a_j||
    const float* const* ys;         // [Bl] caller's measurement vectors
    const LargeOut* outs;           // [Bl] caller's outputs
    const int* kv;                  // [Bl] sparsity
    const int* itv;                 // [Bl] iteration limit min(k, max_iter)
    float* y;                       // [Bl][mp]
    float* r;                       // [Bl][mp]
    float* c;                       // [Bl][n] |c~|
    uint32_t* mask;                 // [Bl][nw]
    int* cand;                      // [Bl][n] candidate atoms
    int* ncand;                     // [Bl]
    unsigned* cmax;                 // [Bl] bits of the largest unselected |c~|
    unsigned long long* best;       // [Bl] (|c| bits << 32) | ~atom of the re-scored winner
    int* sup;                       // [Bl][K]
    float* gpart;                   // [Bl][nseg][K + 2]
    float* gsum;                    // [Bl][K + 2]
    double* W;                      // [Bl][2][K][K] (rows, then columns)
    double* z;                      // [Bl][K]
    double* x;                      // [Bl][K]
    float* xf;                      // [Bl][K]
    double* lpart;                  // [Bl][lch][K]
    double* l;                      // [Bl][K]
    double* upart;                  // [Bl][lch][K]
    double* scal;                   // [Bl][2] 1/L_tt, z_t
    float* rpart;                   // [Bl][rch][mp]
    float* nrm;                     // [Bl][rblk] sums of r_i^2 per 256-row block
    int rblk;                       // ceil(m / 256)
    // Arrival counters of the fused reductions (zero between uses: the last
    // arriver resets its counter), per signal: pbmax = K / 32
    int pbmax;
    unsigned* cntG;                 // [Bl][K + 2] Gram entries: segments done
    unsigned* cntL;                 // [Bl][pbmax] blocks of l: chunks done
    unsigned* cntP;                 // [Bl] blocks of l done
    unsigned* cntU;                 // [Bl][pbmax] blocks of u: chunks done
    unsigned* cntR;                 // [Bl][rblk] residual row blocks: atom chunks done
    unsigned* cntN;                 // [Bl] residual row blocks done
    double* pbpart;                 // [Bl][pbmax][2] sum l_p^2 and sum l_p z_p per block of l
    float* rnorm;                   // [Bl]
    int* nit;                       // [Bl]
    int* st;                        // [Bl] status (-1 running)
    int* live;                      // [1] signals still running after the last check
    // CLOMP (Gram form): G = A_S^T A_S and b = A_S^T y grown by one row per
    // iteration, s double-buffered across the Adam steps, the moments
    int cl, steps, reset;
    float beta1, beta2, eps;
    const float2* tab;              // Adam factor pairs for tau = 1, 2, ...
    float* G;                       // [Bl][K][K]
    float* bv;                      // [Bl][K]
    // s as tagged words (tag << 32 | float bits), two buffers: the value of
    // Adam step number `tag` of the solve sits in buffer tag & 1
    unsigned long long* s0;         // [Bl][K]
    unsigned long long* s1;         // [Bl][K]
    float* am;                      // [Bl][K]
    float* av;                      // [Bl][K]
    unsigned* gbar;                 // [1] the solve's give-up word (a fit's wait ran out)
    unsigned* errflag;              // device error flags
};

__device__ __forceinline__ float lg_delta(const LgState& S, int b) {
    const float g2 = ((float)S.m / 1024.f + 16.f) * 0x1p-24f;
    if (S.mma) {
        // both operands rounded to bf16 (2u + u^2, u = 2^-8) and the tensor
        // core's float32 accumulation, taken as m 2^-22 of sum |a_i r_i|
        const float g1 = (float)S.m * 0x1p-22f;
        return (0x1p-7f + 0x1p-16f + g1 + g2) * 1.01f * (*S.colmax) * S.rnorm[b] * 1.01f;
    }
    const float g1 = ((float)S.m / 32.f + 13.f) * 0x1p-24f;
    const float ua = S.bf16 ? 0x1p-8f * (1.f + g1) : 0.f;
    return (ua + g1 + g2) * 1.01f * (*S.colmax) * S.rnorm[b] * 1.01f;
}

// Block-wide sum (blockDim.x a multiple of 32, <= 1024), fixed order: each
// warp's butterfly, then warp 0 over the warps' sums in warp order.
template <typename T>
__device__ T block_sum(T v, T* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nw ? sh[lane] : T(0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if (lane == 0) sh[32] = w;
    }
    __syncthreads();
    const T out = sh[32];
    __syncthreads();
    return out;
}

// ------------------------------------------------------------- set-up --
// The largest column norm and the tiled copy of A (bf16 or float32; rows
// padded to the tile height, atoms to a multiple of 64, with zeros).  One
// warp per atom of the padded range.
template <typename T>
__global__ void k_lg_prep(const float* __restrict__ A, int lda, int m, int n, int mpt, int njb,
                          T* __restrict__ At, float* colmax) {
    constexpr int TR = lg_tr<T>();
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= njb * LG_TA) return;
    const float* a = A + (size_t)min(j, n - 1) * lda;
    const int nc = mpt / TR;
    float ss = 0.f;
    for (int i = lane; i < mpt; i += 32) {
        const float v = (i < m && j < n) ? a[i] : 0.f;
        ss = fmaf(v, v, ss);
        T* dst = At + (((size_t)(j / LG_TA) * nc + i / TR) * LG_TA + (j % LG_TA)) * TR + (i % TR);
        if constexpr (sizeof(T) == 2) *dst = __float2bfloat16_rn(v);
        else *dst = v;
    }
    ss = warp_sum(ss);
    if (lane == 0 && j < n) atomicMax(reinterpret_cast<unsigned*>(colmax), __float_as_uint(sqrtf(ss)));
}

// Per signal (one CTA): y, r = y, ||y||, the non-finite and tolerance tests.
__global__ void __launch_bounds__(1024) k_lg_setup(LgState S) {
    __shared__ float sh[33];
    const int b = blockIdx.x;
    const float* y = S.ys[b];
    float ss = 0.f;
    int finite = 1;
    for (int i = threadIdx.x; i < S.mp; i += blockDim.x) {
        const float v = i < S.m ? y[i] : 0.f;
        finite &= isfinite(v) ? 1 : 0;
        S.y[(size_t)b * S.mp + i] = v;
        S.r[(size_t)b * S.mp + i] = v;
        if (S.mma) S.R16[(size_t)b * S.mpk + i] = __float2bfloat16_rn(v);
        ss = fmaf(v, v, ss);
    }
    if (S.mma)
        for (int i = S.mp + threadIdx.x; i < S.mpk; i += blockDim.x) S.R16[(size_t)b * S.mpk + i] = __float2bfloat16_rn(0.f);
    const int nw = (S.n + 31) / 32;
    for (int w = threadIdx.x; w < nw; w += blockDim.x) S.mask[(size_t)b * nw + w] = 0u;
    finite = __syncthreads_and(finite);
    ss = block_sum(ss, sh);
    if (threadIdx.x == 0) {
        const float rho = sqrtf(ss);
        S.rnorm[b] = finite ? rho : NAN;
        S.nit[b] = 0;
        S.ncand[b] = 0;
        S.cmax[b] = 0u;
        S.best[b] = 0ull;
        if (!finite) S.st[b] = CS_SIG_NONFINITE;
        else if ((double)rho <= S.tol) S.st[b] = CS_SIG_REACHED_TOL;
        else S.st[b] = -1;
    }
}

// ------------------------------------------------------- correlation --
// Correlation |c~_j| streamed through shared memory: one CTA per SM (per
// pass of NB signals), the pass's residuals in shared memory once, and A's
// tiles (64 atoms x TR rows, 32 KB) brought in by one-dimensional bulk
// copies into a ring of `stages` buffers.  Warp 8's lane 0 takes atom blocks
// from the pass's counter (cblk) and issues their row chunks in order; warp
// w < 8 owns atoms 8w .. 8w + 7 of the block, lane l the 16 bytes at rows
// RPL l .. RPL l + RPL - 1 of every chunk (RPL = 8 bf16 or 4 float32 values),
// summed in ascending row order with float32 fused multiply-adds, and after
// a block's last chunk writes |c~| and folds the per-signal maximum (the
// largest unselected |c~|, atomicMax on the float bits).  Every
// wait is bounded (about 2 s); on time-out the error flags get bit 64 and the
// CTA stops after the copies it issued have landed.
// A's tiles are read once per iteration and are larger than L2: they are
// copied with an evict-first L2 policy, so that what the rest of the
// iteration reuses (W, G, the support's columns, the residuals) stays in L2.
__device__ __forceinline__ uint64_t l2_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ void bulk_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t pol) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
                 : "memory");
}

__host__ __device__ constexpr size_t lg_tma_smem(int stages, int nb, int mpt) {
    return (size_t)stages * LG_TILE_BYTES + sizeof(float) * (size_t)nb * mpt + (size_t)stages * 24;
}

template <typename T, int NB>
__global__ void __launch_bounds__(LG_TMA_THREADS, 1) k_lg_corr_tma(LgState S, int stages) {
    constexpr int TR = lg_tr<T>(), RPL = TR / 32;
    extern __shared__ __align__(1024) unsigned char lsm[];
    unsigned char* tiles = lsm;
    float* rs = reinterpret_cast<float*>(lsm + (size_t)stages * LG_TILE_BYTES);   // [NB][mpt]
    uint64_t* full = reinterpret_cast<uint64_t*>(rs + (size_t)NB * S.mpt);
    uint64_t* empty = full + stages;
    int2* info = reinterpret_cast<int2*>(empty + stages);                       // (block, chunk)
    const int s0 = blockIdx.y * NB;
    bool any = false;
#pragma unroll
    for (int s = 0; s < NB; ++s) any |= (s0 + s < S.Bl) && S.st[s0 + s] < 0;
    if (!any) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        for (int st = 0; st < stages; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], LG_TMA_CONSUMERS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int e = tid; e < NB * S.mpt; e += blockDim.x) {
        const int s = e / S.mpt, i = e - s * S.mpt;
        rs[e] = (s0 + s < S.Bl && i < S.mp) ? S.r[(size_t)(s0 + s) * S.mp + i] : 0.f;
    }
    __syncthreads();

    if (warp == LG_TMA_CONSUMERS) {
        if (lane != 0) return;
        // producer
        const uint64_t pol = l2_evict_first();
        int it = 0;
        bool ok = true;
        for (;;) {
            const int blk = atomicAdd(S.cblk + blockIdx.y, 1);
            if (blk >= S.njb) break;
            const T* src = static_cast<const T*>(S.At) + (size_t)blk * S.nc * LG_TA * TR;
            for (int ic = 0; ic < S.nc; ++ic, ++it) {
                const int st = it % stages;
                if (it >= stages && !mbar_wait(&empty[st], ((it / stages) - 1) & 1)) {
                    ok = false;
                    break;
                }
                info[st] = make_int2(blk, ic);
                mbar_arrive_expect_tx(&full[st], LG_TILE_BYTES);
                bulk_load_1d(tiles + (size_t)st * LG_TILE_BYTES, src + (size_t)ic * LG_TA * TR, LG_TILE_BYTES,
                             &full[st], pol);
            }
            if (!ok) break;
        }
        if (ok) {
            // end of the work: a stage whose block is -1
            const int st = it % stages;
            if (it >= stages && !mbar_wait(&empty[st], ((it / stages) - 1) & 1)) ok = false;
            if (ok) {
                info[st] = make_int2(-1, 0);
                mbar_arrive(&full[st]);
            }
        }
        if (!ok) {
            atomicOr(S.errflag, LG_ERR_CORR);
            // let the copies in flight land before the CTA ends
            for (int q = (it > stages ? it - stages : 0); q < it; ++q) mbar_wait(&full[q % stages], (q / stages) & 1);
        }
        return;
    }

    // consumers
    const int nw = (S.n + 31) / 32;
    float acc[8][NB];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int s = 0; s < NB; ++s) acc[a][s] = 0.f;
    for (int it = 0;; ++it) {
        const int st = it % stages;
        if (!mbar_wait(&full[st], (it / stages) & 1)) {
            if (lane == 0) atomicOr(S.errflag, LG_ERR_CORR);
            break;
        }
        const int2 inf = info[st];
        if (inf.x < 0) break;
        const unsigned char* tile = tiles + (size_t)st * LG_TILE_BYTES;
        uint4 av[8];
#pragma unroll
        for (int a = 0; a < 8; ++a)
            av[a] = *reinterpret_cast<const uint4*>(tile + ((size_t)(warp * 8 + a) * TR + RPL * lane) * sizeof(T));
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[st]);
        const int i = inf.y * TR + RPL * lane;
#pragma unroll
        for (int s = 0; s < NB; ++s) {
            const float4 r0 = *reinterpret_cast<const float4*>(rs + (size_t)s * S.mpt + i);
            if constexpr (sizeof(T) == 2) {
                const float4 r1 = *reinterpret_cast<const float4*>(rs + (size_t)s * S.mpt + i + 4);
                const float rv[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
#pragma unroll
                for (int a = 0; a < 8; ++a) {
                    const unsigned w[4] = {av[a].x, av[a].y, av[a].z, av[a].w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        acc[a][s] = fmaf(__uint_as_float(w[q] << 16), rv[2 * q], acc[a][s]);
                        acc[a][s] = fmaf(__uint_as_float(w[q] & 0xffff0000u), rv[2 * q + 1], acc[a][s]);
                    }
                }
            } else {
#pragma unroll
                for (int a = 0; a < 8; ++a) {
                    acc[a][s] = fmaf(__uint_as_float(av[a].x), r0.x, acc[a][s]);
                    acc[a][s] = fmaf(__uint_as_float(av[a].y), r0.y, acc[a][s]);
                    acc[a][s] = fmaf(__uint_as_float(av[a].z), r0.z, acc[a][s]);
                    acc[a][s] = fmaf(__uint_as_float(av[a].w), r0.w, acc[a][s]);
                }
            }
        }
        if (inf.y == S.nc - 1) {
            const int j0 = inf.x * LG_TA + warp * 8;
#pragma unroll
            for (int s = 0; s < NB; ++s) {
                const int b = s0 + s;
                float mx = 0.f;
#pragma unroll
                for (int a = 0; a < 8; ++a) {
                    const float v = fabsf(warp_sum(acc[a][s]));
                    acc[a][s] = 0.f;
                    const int j = j0 + a;
                    if (b < S.Bl && j < S.n) {
                        if (lane == 0) S.c[(size_t)b * S.n + j] = v;
                        const bool sel = (S.mask[(size_t)b * nw + (j >> 5)] >> (j & 31)) & 1u;
                        if (!sel) mx = fmaxf(mx, v);
                    }
                }
                if (lane == 0 && b < S.Bl && S.st[b] < 0) atomicMax(S.cmax + b, __float_as_uint(mx));
            }
        }
    }
}

// Transposed max-reduction: lane l ends with the maximum over the warp of
// k[l] (in k[0]), 31 shuffles for the 32 values.
__device__ __forceinline__ void lg_max_scatter32(uint32_t (&k)[32]) {
    const unsigned lane = threadIdx.x & 31u;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < off; ++i) {
            const uint32_t send = upper ? k[i] : k[i + off];
            const uint32_t keep = upper ? k[i + off] : k[i];
            k[i] = max(keep, __shfl_xor_sync(0xffffffffu, send, off));
        }
    }
}

// Correlation of a pass of up to 256 signals as one tensor-core GEMM
// (bf16 operands, float32 accumulation in tensor memory): CTA x owns atoms
// 128 x .. 128 x + 127 (UMMA M, the TMEM lanes) and the pass's N signals
// (UMMA N, TMEM columns); the K = m dimension streams by TMA in 64-element
// chunks -- the atom tile (128 rows of A's K-major copy) and the residual
// tile (N rows of the residuals' copy), 128-byte swizzled -- through a ring
// of `stages` buffers.  Thread 0 issues the copies, thread 32 the four
// MMAs of each chunk and a commit that frees the stage; after the last
// chunk a commit signals the epilogue, where thread t reads its atom's N
// accumulators (tcgen05.ld), writes |c~| per signal and folds each signal's
// largest unselected |c~| (a warp maximum, then atomicMax on the float
// bits).  Every wait is bounded (about 2 s); on time-out the error flags
// get bit 128, the epilogue is skipped and the CTA returns after its copies
// and MMAs in flight have finished and its tensor memory is freed.
__global__ void __launch_bounds__(LG_MMA_THREADS, 1)
k_lg_corr_mma(const __grid_constant__ CUtensorMap mapR, LgState S, int stages, int N, int tmem_cols) {
    extern __shared__ uint8_t lmsm[];
    __shared__ __align__(8) uint64_t full[LG_MMA_MAX_STAGES];
    __shared__ __align__(8) uint64_t empty[LG_MMA_MAX_STAGES];
    __shared__ __align__(8) uint64_t done;
    __shared__ uint32_t tmem_slot;
    __shared__ int failed;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int j0 = blockIdx.x * 128;
    const int s0 = blockIdx.y * LG_MMA_MAXN;
    bool any = false;
    for (int s = 0; s < N && s0 + s < S.Bl; ++s) any |= S.st[s0 + s] < 0;
    if (!any) return;
    const int rbytes = N * 128;
    const int stage_bytes = LG_MMA_ATILE + rbytes;
    const uint32_t raw = smem_u32(lmsm);
    uint8_t* base = lmsm + (((raw + 1023u) & ~1023u) - raw);
    if (tid == 0) {
        failed = 0;
        for (int st = 0; st < stages; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], 1);
        }
        mbar_init(&done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const int nk = S.mpk / LG_MMA_KCH;

    if (tid == 0) {
        // producer: the K chunks in order, one stage each
        const uint64_t pol = l2_evict_first();
        int it = 0;
        bool ok = true;
        for (; it < nk; ++it) {
            const int st = it % stages;
            if (it >= stages && !mbar_wait(&empty[st], ((it / stages) - 1) & 1)) {
                ok = false;
                break;
            }
            uint8_t* sa = base + (size_t)st * stage_bytes;
            mbar_arrive_expect_tx(&full[st], (uint32_t)stage_bytes);
            bulk_load_1d(sa, S.Ak + ((size_t)blockIdx.x * nk + it) * (LG_MMA_ATILE / 2), LG_MMA_ATILE, &full[st], pol);
            tma_load_2d(sa + LG_MMA_ATILE, &mapR, &full[st], it * LG_MMA_KCH, s0);
        }
        if (!ok) {
            failed = 1;
            atomicOr(S.errflag, LG_ERR_MMA);
            // let the copies in flight land
            for (int q = (it > stages ? it - stages : 0); q < it; ++q) mbar_wait(&full[q % stages], (q / stages) & 1);
        }
    } else if (tid == 32) {
        // MMA issuer
        const uint32_t idesc = make_idesc(128, N);
        bool ok = true;
        for (int it = 0; it < nk; ++it) {
            const int st = it % stages;
            if (!mbar_wait(&full[st], (it / stages) & 1)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint8_t* sa = base + (size_t)st * stage_bytes;
            const uint64_t da = smem_desc_sw128(smem_u32(sa));
            const uint64_t db = smem_desc_sw128(smem_u32(sa + LG_MMA_ATILE));
#pragma unroll
            for (int k = 0; k < 4; ++k) umma_bf16(tmem, da + (uint64_t)(2 * k), db + (uint64_t)(2 * k), idesc, (it | k) != 0);
            umma_commit(&empty[st]);   // the stage is free once these MMAs have read it
        }
        if (!ok) {
            failed = 1;
            atomicOr(S.errflag, LG_ERR_MMA);
        }
        umma_commit(&done);            // arrives once every issued MMA has completed
    }
    __syncwarp();
    const bool waited = mbar_wait(&done, 0);
    tc_fence_after();
    if (!waited && lane == 0) atomicOr(S.errflag, LG_ERR_MMA);
    const bool ok = __syncthreads_and(waited && !failed) != 0;
    if (ok) {
        // epilogue: thread tid holds atom j0 + tid (TMEM lane tid)
        const int j = j0 + tid;
        const int nw = (S.n + 31) / 32;
        const uint32_t tbase = tmem + ((uint32_t)(warp * 32) << 16);
        const int jw = (j0 + warp * 32) >> 5;        // this warp's mask word (32-aligned atoms)
        for (int c0 = 0; c0 < N; c0 += 32) {
            // lane q fetches signal c0 + q's mask word and status for the whole warp
            const int bq = s0 + c0 + lane;
            const bool vq = c0 + lane < N && bq < S.Bl;
            const uint32_t mword = (vq && jw < nw) ? S.mask[(size_t)bq * nw + jw] : 0u;
            const int stq = vq ? S.st[bq] : 0;
            uint32_t v[32];
            tmem_ld32(tbase + (uint32_t)c0, v);
            tmem_ld_wait();
            // |c~| of the 32 signals for this atom; the unselected ones (as
            // float bits: non-negative floats order like their bits) go to a
            // transposed max-reduction, after which lane q holds the warp's
            // largest for signal c0 + q
            uint32_t key[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                const int b = s0 + c0 + q;
                const uint32_t mw = __shfl_sync(FULL, mword, q);
                const float x = fabsf(__uint_as_float(v[q]));
                const bool valid = c0 + q < N && b < S.Bl && j < S.n;
                if (valid) S.c[(size_t)b * S.n + j] = x;
                key[q] = (valid && !((mw >> lane) & 1u)) ? __float_as_uint(x) : 0u;
            }
            lg_max_scatter32(key);
            if (vq && stq < 0) atomicMax(S.cmax + bq, key[0]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
    }
}

// bf16 copy of A for the GEMM correlation, in 16 KB tiles of 128 atoms x 64
// K values, each stored as the shared-memory image that a TMA copy with the
// 128-byte swizzle would produce -- row r (atom) of 128 bytes, its 16-byte
// chunk c at position c ^ (r mod 8) -- so that one 1-D bulk copy per tile
// lands it ready for the MMA descriptor; and the largest column norm (one
// warp per atom of the padded range).
__global__ void k_lg_prep_k(const float* __restrict__ A, int lda, int m, int n, int mpk,
                            __nv_bfloat16* __restrict__ Ak, float* colmax) {
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= round_up(n, 128)) return;
    const float* a = A + (size_t)min(j, n - 1) * lda;
    const int nkc = mpk / LG_MMA_KCH, r = j % 128;
    __nv_bfloat16* tiles = Ak + (size_t)(j / 128) * nkc * (LG_MMA_ATILE / 2);
    float ss = 0.f;
    for (int i = lane; i < mpk; i += 32) {
        const float v = (i < m && j < n) ? a[i] : 0.f;
        ss = fmaf(v, v, ss);
        const int kc = i / LG_MMA_KCH, e = i % LG_MMA_KCH;
        const int off = r * 64 + (((e >> 3) ^ (r & 7)) << 3) + (e & 7);   // bf16 elements within the tile
        tiles[(size_t)kc * (LG_MMA_ATILE / 2) + off] = __float2bfloat16_rn(v);
    }
    ss = warp_sum(ss);
    if (lane == 0 && j < n) atomicMax(reinterpret_cast<unsigned*>(colmax), __float_as_uint(sqrtf(ss)));
}

// ---------------------------------------------------------- selection --
// Candidates: unselected atoms with |c~| >= max - 2 delta.
__global__ void __launch_bounds__(256) k_lg_scan(LgState S) {
    pdl_wait();      // the previous launch of the iteration is complete
    pdl_trigger();
    const int b = blockIdx.y;
    if (S.st[b] >= 0) return;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= S.n) return;
    const int nw = (S.n + 31) / 32;
    if ((S.mask[(size_t)b * nw + (j >> 5)] >> (j & 31)) & 1u) return;
    const float theta = __uint_as_float(S.cmax[b]) - 2.f * lg_delta(S, b);
    if (S.c[(size_t)b * S.n + j] >= theta) {
        const int q = atomicAdd(S.ncand + b, 1);
        S.cand[(size_t)b * S.n + q] = j;
    }
}

// float32 re-score of the candidates (one CTA per candidate) and the argmax.
__global__ void __launch_bounds__(1024) k_lg_rescore(LgState S) {
    pdl_wait();      // the previous launch of the iteration is complete
    pdl_trigger();
    __shared__ float sh[33];
    const int b = blockIdx.y;
    if (S.st[b] >= 0) return;
    const int nc = S.ncand[b];
    const float* r = S.r + (size_t)b * S.mp;
    for (int q = blockIdx.x; q < nc; q += gridDim.x) {
        const int j = S.cand[(size_t)b * S.n + q];
        const float* a = S.A + (size_t)j * S.lda;
        float acc = 0.f;
#pragma unroll 8
        for (int i = threadIdx.x; i < S.m; i += blockDim.x) acc = fmaf(a[i], r[i], acc);
        const float v = fabsf(block_sum(acc, sh));
        if (threadIdx.x == 0) {
            const unsigned long long key =
                ((unsigned long long)__float_as_uint(v) << 32) | (unsigned long long)(0xffffffffu - (unsigned)j);
            atomicMax(S.best + b, key);
        }
    }
}

// ------------------------------------------------------- Gram column --
// Append the winner (CTA 0) and the partial dot products of a_j with the
// support atoms (i < t), itself (i = t) and y (i = t + 1), one warp per
// (entry, 2048-row segment).
__global__ void __launch_bounds__(256) k_lg_gram(LgState S, int t) {
    pdl_wait();      // the previous launch of the iteration is complete
    pdl_trigger();
    const int b = blockIdx.y;
    if (S.st[b] >= 0) return;
    const unsigned long long key = S.best[b];
    const int lane = threadIdx.x & 31;
    const int nw = (S.n + 31) / 32;
    if (key == 0ull) {                       // no unselected atom left
        if (blockIdx.x == 0 && threadIdx.x == 0) S.st[b] = CS_SIG_MAX_ITER;
        return;
    }
    const int j = (int)(0xffffffffu - (unsigned)(key & 0xffffffffull));
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        S.sup[(size_t)b * S.K + t] = j;
        S.mask[(size_t)b * nw + (j >> 5)] |= 1u << (j & 31);
    }
    const int items = (t + 2) * S.nseg;
    const int item = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (item >= items) return;
    const int i = item % (t + 2), seg = item / (t + 2);
    const float* aj = S.A + (size_t)j * S.lda;
    const float* other = (i < t) ? S.A + (size_t)S.sup[(size_t)b * S.K + i] * S.lda
                                 : (i == t ? aj : S.y + (size_t)b * S.mp);
    const int r0 = seg * LG_SEG, r1 = min(S.m, r0 + LG_SEG);
    float acc = 0.f;
    for (int q0 = r0; q0 < r1; q0 += 256) {     // eight rows per lane in flight, ascending
        float o[8], v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int q = q0 + lane + 32 * u;
            o[u] = q < r1 ? other[q] : 0.f;
            v[u] = q < r1 ? aj[q] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) acc = fmaf(o[u], v[u], acc);
    }
    acc = warp_sum(acc);
    // the warp that completes entry i sums its segments in order
    unsigned prev = 0;
    if (lane == 0) {
        S.gpart[((size_t)b * S.nseg + seg) * (S.K + 2) + i] = acc;
        __threadfence();
        prev = atomicAdd(S.cntG + (size_t)b * (S.K + 2) + i, 1u);
    }
    if (lane == 0 && prev == (unsigned)(S.nseg - 1)) {
        __threadfence();
        float v = 0.f;
        for (int sg = 0; sg < S.nseg; ++sg) v += __ldcg(S.gpart + ((size_t)b * S.nseg + sg) * (S.K + 2) + i);
        S.gsum[(size_t)b * (S.K + 2) + i] = v;
        S.cntG[(size_t)b * (S.K + 2) + i] = 0u;
    }
}

// -------------------------------------------------- float64 Cholesky --
__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// The pivot and the diagonal entries once sum l_p^2 (ssq) and sum l_p z_p (lz)
// are known: 1 / L_tt, z_t, W_tt, x_t (or status 3 for a dependent atom).
__device__ void lg_pivot_finish(const LgState& S, int b, int t, double ssq, double lz) {
    const double d = (double)S.gsum[(size_t)b * (S.K + 2) + t];
    const double bt = (double)S.gsum[(size_t)b * (S.K + 2) + t + 1];
    const double piv = d - ssq;
    if (!(piv > 0x1p-20 * d)) {
        S.st[b] = CS_SIG_DEPENDENT;
        return;
    }
    const double ltt = sqrt(piv);
    const double zt = (bt - lz) / ltt;
    const double rinv = 1.0 / ltt;
    S.scal[2 * b] = rinv;
    S.scal[2 * b + 1] = zt;
    S.z[(size_t)b * S.K + t] = zt;
    double* Wr = S.W + (size_t)b * 2 * S.K * S.K;
    Wr[(size_t)t * S.K + t] = rinv;
    Wr[(size_t)S.K * S.K + (size_t)t * S.K + t] = rinv;
    const double xt = zt * rinv;
    S.x[(size_t)b * S.K + t] = xt;
    S.xf[(size_t)b * S.K + t] = (float)xt;
    S.nit[b] = t + 1;
}

// l = W^T g, l_p = sum_{i <= p} W_ip g_i, and the pivot: one warp per
// (32 entries p, 32-entry chunk of i), lanes over p, partial sums per chunk.
// The warp that completes a block of p sums its chunks in order (l_p) and
// that block's sum l_p^2 and l_p z_p; the last block adds the blocks' sums
// in order and finishes the pivot.  t = 0: one warp, no l.
__global__ void __launch_bounds__(32) k_lg_lpiv(LgState S, int t) {
    pdl_wait();      // the previous launch of the iteration is complete
    pdl_trigger();
    const int b = blockIdx.y;
    if (S.st[b] >= 0) return;
    const int lane = threadIdx.x & 31;
    const int item = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (t == 0) {
        if (item == 0 && lane == 0) lg_pivot_finish(S, b, 0, 0.0, 0.0);
        return;
    }
    const int pblocks = (t + 31) / 32, ich = (t + LG_LC - 1) / LG_LC;
    if (item >= pblocks * ich) return;
    const int pb = item % pblocks, ic = item / pblocks;
    const int p = pb * 32 + lane;
    const int i0 = ic * LG_LC, i1 = min(t, i0 + LG_LC);
    const double* Wr = S.W + (size_t)b * 2 * S.K * S.K;
    const float* g = S.gsum + (size_t)b * (S.K + 2);
    double acc = 0.0;
    for (int ib = i0; ib < i1; ib += 8) {
        double wv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = ib + u;
            wv[u] = (i < i1 && i <= p && p < t) ? Wr[(size_t)i * S.K + p] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = ib + u;
            if (i < i1 && i <= p && p < t) acc = fma(wv[u], (double)g[i], acc);
        }
    }
    if (p < t) S.lpart[((size_t)b * S.lch + ic) * S.K + p] = acc;
    __threadfence();
    unsigned prev = 0;
    if (lane == 0) prev = atomicAdd(S.cntL + (size_t)b * S.pbmax + pb, 1u);
    prev = __shfl_sync(FULL, prev, 0);
    if (prev != (unsigned)(ich - 1)) return;
    // last chunk of this block: l_p over the chunks in order
    __threadfence();
    double lp = 0.0;
    for (int ic0 = 0; ic0 < ich; ic0 += 8) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
            v[u] = (ic0 + u < ich && p < t) ? __ldcg(S.lpart + ((size_t)b * S.lch + ic0 + u) * S.K + p) : 0.0;
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (ic0 + u < ich) lp += v[u];
    }
    double sq = 0.0, lz = 0.0;
    if (p < t) {
        S.l[(size_t)b * S.K + p] = lp;
        sq = lp * lp;
        lz = lp * S.z[(size_t)b * S.K + p];
    }
    sq = warp_sum_f64(sq);
    lz = warp_sum_f64(lz);
    if (lane == 0) {
        S.pbpart[((size_t)b * S.pbmax + pb) * 2] = sq;
        S.pbpart[((size_t)b * S.pbmax + pb) * 2 + 1] = lz;
        S.cntL[(size_t)b * S.pbmax + pb] = 0u;
        __threadfence();
        prev = atomicAdd(S.cntP + b, 1u);
    }
    prev = __shfl_sync(FULL, prev, 0);
    if (prev == (unsigned)(pblocks - 1)) {
        // last block: the blocks' sums (lane q takes blocks q, q + 32, ...,
        // then the warp tree), then the pivot
        __threadfence();
        double ssq = 0.0, lzs = 0.0;
        for (int q = lane; q < pblocks; q += 32) {
            ssq += __ldcg(S.pbpart + ((size_t)b * S.pbmax + q) * 2);
            lzs += __ldcg(S.pbpart + ((size_t)b * S.pbmax + q) * 2 + 1);
        }
        ssq = warp_sum_f64(ssq);
        lzs = warp_sum_f64(lzs);
        if (lane == 0) {
            S.cntP[b] = 0u;
            lg_pivot_finish(S, b, t, ssq, lzs);
        }
    }
}

// u = W l, u_i = sum_{p >= i} W_ip l_p, then the new column of W and
// x += z_t w: one warp per (32 entries i, 32-entry chunk of p), lanes over
// i; the warp that completes a block of i sums its chunks in order (from the
// block's own chunk: earlier chunks hold no p >= i) and updates those
// entries (t >= 1; W_tt and x_t come with the pivot).
__global__ void __launch_bounds__(32) k_lg_uupd(LgState S, int t) {
    pdl_wait();      // the previous launch of the iteration is complete
    pdl_trigger();
    const int b = blockIdx.y;
    if (S.st[b] >= 0) return;
    const int lane = threadIdx.x & 31;
    const int item = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int iblocks = (t + 31) / 32, pch = (t + LG_LC - 1) / LG_LC;
    if (item >= iblocks * pch) return;
    const int ib = item % iblocks, pc = item / iblocks;
    const int i = ib * 32 + lane;
    const int p0 = pc * LG_LC, p1 = min(t, p0 + LG_LC);
    double* Wr = S.W + (size_t)b * 2 * S.K * S.K;
    double* Wc = Wr + (size_t)S.K * S.K;
    const double* l = S.l + (size_t)b * S.K;
    double acc = 0.0;
    for (int pb = p0; pb < p1; pb += 8) {
        double wv[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const int p = pb + v;
            wv[v] = (p < p1 && i <= p) ? Wc[(size_t)p * S.K + i] : 0.0;
        }
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const int p = pb + v;
            if (p < p1 && i <= p) acc = fma(wv[v], l[p], acc);
        }
    }
    if (i < t) S.upart[((size_t)b * S.lch + pc) * S.K + i] = acc;
    __threadfence();
    unsigned prev = 0;
    if (lane == 0) prev = atomicAdd(S.cntU + (size_t)b * S.pbmax + ib, 1u);
    prev = __shfl_sync(FULL, prev, 0);
    if (prev != (unsigned)(pch - 1)) return;
    __threadfence();
    if (lane == 0) S.cntU[(size_t)b * S.pbmax + ib] = 0u;
    if (i >= t) return;
    const int pc0 = (ib * 32) / LG_LC;
    double u = 0.0;
    for (int q0 = pc0; q0 < pch; q0 += 8) {
        double v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q)
            v[q] = q0 + q < pch ? __ldcg(S.upart + ((size_t)b * S.lch + q0 + q) * S.K + i) : 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (q0 + q < pch) u += v[q];
    }
    const double rinv = S.scal[2 * b], zt = S.scal[2 * b + 1];
    const double w = -u * rinv;
    Wr[(size_t)i * S.K + t] = w;
    Wc[(size_t)t * S.K + i] = w;
    const double xi = fma(zt, w, S.x[(size_t)b * S.K + i]);
    S.x[(size_t)b * S.K + i] = xi;
    S.xf[(size_t)b * S.K + i] = (float)xi;
}

// ------------------------------------------------------ CLOMP Gram fit --
__device__ __forceinline__ unsigned long long lg_tagged(unsigned tag, float v) {
    return ((unsigned long long)tag << 32) | __float_as_uint(v);
}

// Append the new atom to the Gram form: row and column t of G from the Gram
// column, G_tt = ||a_j||^2, b_t = a_j^T y; the new coefficient (zero, with
// the fit's first tag) and its moments start at zero (with
// reset_adam_each_iter every moment restarts).
__global__ void __launch_bounds__(256) k_lgc_append(LgState S, int t, unsigned tag0) {
    pdl_wait();      // the previous launch of the iteration is complete
    pdl_trigger();
    const int b = blockIdx.y;
    if (S.st[b] >= 0) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > t) return;
    const float* g = S.gsum + (size_t)b * (S.K + 2);
    float* G = S.G + (size_t)b * S.K * S.K;
    const size_t o = (size_t)b * S.K;
    if (i < t) {
        G[(size_t)t * S.K + i] = g[i];
        G[(size_t)i * S.K + t] = g[i];
        if (S.reset) {
            S.am[o + i] = 0.f;
            S.av[o + i] = 0.f;
        }
    } else {
        G[(size_t)t * S.K + t] = g[t];
        S.bv[o + t] = g[t + 1];
        ((tag0 & 1u) ? S.s1 : S.s0)[o + t] = lg_tagged(tag0, 0.f);
        S.am[o + t] = 0.f;
        S.av[o + t] = 0.f;
        S.xf[o + t] = 0.f;
        S.nit[b] = t + 1;
    }
}

// (G s - b)_q by one warp, lane-strided with eight entries in flight per
// lane, ascending; Gq and sv may sit in global or shared memory.
__device__ __forceinline__ float lg_gram_row_dot(const float* Gq, const float* sv, int t1, int lane) {
    float acc = 0.f;
    for (int p0 = 0; p0 < t1; p0 += 256) {
        float gv[8], xv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int p = p0 + lane + 32 * u;
            gv[u] = p < t1 ? Gq[p] : 0.f;
            xv[u] = p < t1 ? sv[p] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) acc = fmaf(gv[u], xv[u], acc);
    }
    return warp_sum(acc);
}

// Adam on one coordinate (PyTorch's update rule; cc = the step's factors)
__device__ __forceinline__ float lg_adam(const LgState& S, float g, float s_q, float2 cc, float& mo, float& ve) {
    mo = fmaf(S.beta1, mo, (1.f - S.beta1) * g);
    ve = fmaf(S.beta2, ve, (1.f - S.beta2) * g * g);
    return s_q - cc.x * mo / fmaf(sqrtf(ve), cc.y, S.eps);
}

// One Adam step of every live signal on its t1 coordinates (one warp per
// coordinate q): reads s of step `tag` (stream order makes it complete),
// writes step tag + 1.  The last step of a fit also writes the coefficients
// used by the residual.
__global__ void __launch_bounds__(256) k_lgc_step(LgState S, int t1, int tau, unsigned tag, int last) {
    __shared__ float ss[kLargeMaxK];
    const int b = blockIdx.y;
    if (S.st[b] >= 0) return;
    const size_t o = (size_t)b * S.K;
    const unsigned long long* in = ((tag & 1u) ? S.s1 : S.s0) + o;
    unsigned long long* out = (((tag + 1u) & 1u) ? S.s1 : S.s0) + o;
    for (int p = threadIdx.x; p < t1; p += blockDim.x) ss[p] = __uint_as_float((unsigned)in[p]);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (q >= t1) return;
    const float g = lg_gram_row_dot(S.G + (o + q) * S.K, ss, t1, lane) - S.bv[o + q];
    if (lane == 0) {
        float mo = S.am[o + q], ve = S.av[o + q];
        const float sn = lg_adam(S, g, ss[q], S.tab[tau - 1], mo, ve);
        S.am[o + q] = mo;
        S.av[o + q] = ve;
        out[q] = lg_tagged(tag + 1u, sn);
        if (last) S.xf[o + q] = sn;
    }
}

// All T Adam steps of one iteration in one cooperative launch (every CTA
// resident).  CTA (x, b) owns the rows q0 = x R .. q0 + R - 1 of signal b's G,
// copied to shared memory once, with their moments and b_q.  Per step it
// waits for all t1 words of s carrying the step's tag (each written, value
// and tag in one 64-bit store, by the CTA that owns the coordinate), stages
// the values, forms its rows of G s - b in the order of k_lgc_step and
// writes the new values with the next tag into the other buffer.  No CTA can
// overwrite a word another still has to read: writing step j + 2 needs all of
// step j + 1, which each CTA writes only after reading all of step j.  Waits
// are bounded; on time-out the error flags get bit 32, the solve's give-up
// word is set, and every CTA of this and later fits of the solve returns.
constexpr unsigned long long LG_WAIT_CYCLES = 4000000000ull;   // ~2 s at 2 GHz
constexpr unsigned LG_ERR_WAIT = 32u;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Stage s of step `tag` (t1 words from `in`) in ss: every thread polls its
// words (up to eight per round, all re-read together) until each carries the
// tag; false on give-up (time-out here, or another CTA's).
__device__ bool lg_stage_tagged(const LgState& S, const unsigned long long* in, unsigned tag, int t1, float* ss) {
    const unsigned long long t0 = clock64();
    unsigned spins = 0;
    for (int p0 = 0; p0 < t1; p0 += 8 * blockDim.x) {
        unsigned pending = 0;
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (p0 + (int)threadIdx.x + u * (int)blockDim.x < t1) pending |= 1u << u;
        while (pending != 0u) {
            unsigned long long v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                v[u] = (pending >> u) & 1u ? ld_relaxed_u64(in + p0 + threadIdx.x + u * blockDim.x) : 0ull;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (((pending >> u) & 1u) && (unsigned)(v[u] >> 32) == tag) {
                    ss[p0 + threadIdx.x + u * blockDim.x] = __uint_as_float((unsigned)v[u]);
                    pending &= ~(1u << u);
                }
            }
            if (pending != 0u && (++spins & 15u) == 0u) {
                if (ld_acquire_u32(S.gbar) != 0u) return false;
                if (clock64() - t0 > LG_WAIT_CYCLES) {
                    atomicOr(S.errflag, LG_ERR_WAIT);
                    atomicExch(S.gbar, 1u);
                    return false;
                }
            }
        }
    }
    return true;
}

__host__ __device__ constexpr int lg_fit_smem_floats(int t1, int R) {
    return (t1 + 3) / 4 * 4 * (R + 1) + 3 * R;
}

__global__ void __launch_bounds__(256) k_lgc_fit(LgState S, int t1, int R, int tau0, unsigned tag0) {
    extern __shared__ __align__(16) float fsh[];
    __shared__ int go;
    const int t1p = (t1 + 3) / 4 * 4;
    float* ss = fsh;                 // [t1p] s of the step
    float* ams = ss + t1p;           // [R] moments and b of the CTA's rows
    float* avs = ams + R;
    float* bvs = avs + R;
    float* Gs = bvs + R;             // [R][t1p] (16-byte aligned: t1p and 3 R are multiples of 4)
    const int b = blockIdx.y;
    if (S.st[b] >= 0) return;        // no CTA of a finished signal is waited for
    const int q0 = blockIdx.x * R, nr = min(R, t1 - q0);
    if (nr <= 0) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t o = (size_t)b * S.K;
    if (threadIdx.x == 0) go = ld_acquire_u32(S.gbar) == 0u;
    __syncthreads();
    if (!go) return;
    // the rows (16-byte copies, eight in flight per lane; G's rows are K
    // floats apart, K a multiple of 32, and t1p <= K)
    for (int r = warp; r < nr; r += blockDim.x >> 5) {
        const float4* src = reinterpret_cast<const float4*>(S.G + (o + q0 + r) * S.K);
        float4* dst = reinterpret_cast<float4*>(Gs + (size_t)r * t1p);
        const int n4 = t1p / 4;
        for (int c0 = 0; c0 < n4; c0 += 256) {
            float4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int c = c0 + lane + 32 * u;
                if (c < n4) v[u] = src[c];
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int c = c0 + lane + 32 * u;
                if (c < n4) dst[c] = v[u];
            }
        }
    }
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
        ams[r] = S.am[o + q0 + r];
        avs[r] = S.av[o + q0 + r];
        bvs[r] = S.bv[o + q0 + r];
    }
    for (int step = 0; step < S.steps; ++step) {
        const unsigned tag = tag0 + (unsigned)step;
        const unsigned long long* in = ((tag & 1u) ? S.s1 : S.s0) + o;
        unsigned long long* out = (((tag + 1u) & 1u) ? S.s1 : S.s0) + o;
        const bool ok = lg_stage_tagged(S, in, tag, t1, ss);
        if (__syncthreads_or(!ok)) return;
        const float2 cc = S.tab[tau0 + step];
        for (int r = warp; r < nr; r += blockDim.x >> 5) {
            const int q = q0 + r;
            const float g = lg_gram_row_dot(Gs + (size_t)r * t1p, ss, t1, lane) - bvs[r];
            if (lane == 0) {
                float mo = ams[r], ve = avs[r];
                const float sn = lg_adam(S, g, ss[q], cc, mo, ve);
                ams[r] = mo;
                avs[r] = ve;
                st_relaxed_u64(out + q, lg_tagged(tag + 1u, sn));
                if (step + 1 == S.steps) S.xf[o + q] = sn;
            }
        }
        __syncthreads();
    }
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
        S.am[o + q0 + r] = ams[r];
        S.av[o + q0 + r] = avs[r];
    }
}

// ----------------------------------------------------------- residual --
// r = y - A_S x (x as float32): CTA (row block x of 256 rows, chunk qc of
// 32 support atoms) forms the chunk's partial sums for its rows; the CTA
// that completes a row block adds the chunks in order, writes r (and its
// bf16 copy) and the block's sum of r_i^2; the last row block adds those in
// order and applies the stopping rule of Eq. 2, resetting the selection
// state for the next iteration.
__global__ void __launch_bounds__(256) k_lg_resid(LgState S, int t1) {
    pdl_wait();      // the previous launch of the iteration is complete
    pdl_trigger();
    __shared__ int sj[LG_RQ];
    __shared__ float sx[LG_RQ];
    __shared__ float sh[33];
    __shared__ unsigned last;
    const int b = blockIdx.z;
    if (S.st[b] >= 0) return;
    const int qc = blockIdx.y, rb = blockIdx.x;
    const int q0 = qc * LG_RQ, q1 = min(t1, q0 + LG_RQ);
    const int nq = q1 - q0;
    for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
        sj[q - q0] = S.sup[(size_t)b * S.K + q];
        sx[q - q0] = S.xf[(size_t)b * S.K + q];
    }
    __syncthreads();
    const int i = rb * 256 + threadIdx.x;
    if (i < S.m) {
        float acc = 0.f;
        int q = 0;
        for (; q + 8 <= nq; q += 8) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = S.A[(size_t)sj[q + u] * S.lda + i];
#pragma unroll
            for (int u = 0; u < 8; ++u) acc = fmaf(v[u], sx[q + u], acc);
        }
        for (; q < nq; ++q) acc = fmaf(S.A[(size_t)sj[q] * S.lda + i], sx[q], acc);
        S.rpart[((size_t)b * S.rch + qc) * S.mp + i] = acc;
    }
    __threadfence();
    __syncthreads();
    const int qch = gridDim.y;
    if (threadIdx.x == 0) last = atomicAdd(S.cntR + (size_t)b * S.rblk + rb, 1u) == (unsigned)(qch - 1) ? 1u : 0u;
    __syncthreads();
    if (!last) return;
    // this row block's chunks are all in: r over the chunks in order
    __threadfence();
    float ri = 0.f;
    if (i < S.m) {
        float acc = 0.f;
        for (int c = 0; c < qch; ++c) acc += __ldcg(S.rpart + ((size_t)b * S.rch + c) * S.mp + i);
        ri = S.y[(size_t)b * S.mp + i] - acc;
        S.r[(size_t)b * S.mp + i] = ri;
        if (S.mma) S.R16[(size_t)b * S.mpk + i] = __float2bfloat16_rn(ri);
    }
    const float ss = block_sum(ri * ri, sh);
    if (threadIdx.x == 0) {
        S.nrm[(size_t)b * S.rblk + rb] = ss;
        S.cntR[(size_t)b * S.rblk + rb] = 0u;
        __threadfence();
        last = atomicAdd(S.cntN + b, 1u) == (unsigned)(S.rblk - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (!last) return;
    // the last row block: ||r||^2 over the blocks (thread q takes blocks
    // q, q + 256, ..., then the block tree), the stopping rule
    __threadfence();
    float part = 0.f;
    for (int q = threadIdx.x; q < S.rblk; q += blockDim.x) part += __ldcg(S.nrm + (size_t)b * S.rblk + q);
    const float tot = block_sum(part, sh);
    if (threadIdx.x == 0) {
        S.cntN[b] = 0u;
        const float rho = sqrtf(tot);
        S.rnorm[b] = rho;
        S.ncand[b] = 0;
        S.cmax[b] = 0u;
        S.best[b] = 0ull;
        if ((double)rho <= S.tol) S.st[b] = CS_SIG_REACHED_TOL;
        else if (t1 >= S.kv[b]) S.st[b] = CS_SIG_REACHED_K;
        else if (t1 >= S.itv[b]) S.st[b] = CS_SIG_MAX_ITER;
    }
}

// Signals still running (for the host's early end of the iteration loop).
__global__ void k_lg_count(LgState S) {
    int c = 0;
    for (int b = threadIdx.x; b < S.Bl; b += blockDim.x) c += S.st[b] < 0 ? 1 : 0;
    c = __reduce_add_sync(0xffffffffu, c);
    if (threadIdx.x == 0) *S.live = c;
}

// Outputs: support and coefficients (-1 / 0 past n_iter), n_iter, ||r||, status.
__global__ void k_lg_out(LgState S) {
    const int b = blockIdx.x;
    const LargeOut o = S.outs[b];
    const int t = S.nit[b];
    for (int q = threadIdx.x; q < o.k; q += blockDim.x) {
        o.support[q] = q < t ? S.sup[(size_t)b * S.K + q] : -1;
        o.coef[q] = q < t ? S.xf[(size_t)b * S.K + q] : 0.f;
    }
    if (threadIdx.x == 0) {
        *o.n_iter = t;
        *o.res_norm = S.rnorm[b];
        *o.status = S.st[b] < 0 ? CS_SIG_MAX_ITER : S.st[b];
    }
}

struct LgLayout {
    size_t At, Ak, R16, cblk, cnt, pbpart, colmax, ys, outs, kv, itv, y, r, c, mask, cand, ncand, cmax, best, sup, gpart, gsum, W, z, x,
        xf, lpart, l, upart, scal, rpart, nrm, rnorm, nit, st, live, G, bv, s0, s1, am, av, gbar, total;
};

// The correlation runs as a tensor-core GEMM for bf16 and at least
// LG_MMA_MIN_SIGNALS signals sharing A (one pass over A per iteration instead
// of one per pass of up to four signals).
bool lg_uses_mma(int bf16, int Bl) { return bf16 && Bl >= LG_MMA_MIN_SIGNALS; }

// cl: CLOMP's Gram-form state instead of OMP's float64 W = L^{-T}.
LgLayout lg_layout(int m, int n, int Bl, int kmax, int bf16, int cl) {
    const size_t B = (size_t)Bl, K = (size_t)round_up(kmax, 32), mp = (size_t)round_up(m, 8);
    const size_t nseg = (size_t)ceil_div(m, LG_SEG), lch = (size_t)ceil_div((int)K, LG_LC),
                 rch = (size_t)ceil_div((int)K, LG_RQ), nw = (size_t)ceil_div(n, 32);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = (off + 255) & ~(size_t)255;
        const size_t o = off;
        off += bytes;
        return o;
    };
    LgLayout L{};
    if (lg_uses_mma(bf16, Bl)) {
        const size_t mpk = (size_t)round_up(m, LG_MMA_KCH);
        L.Ak = take(sizeof(__nv_bfloat16) * (size_t)round_up(n, 128) * mpk);
        L.R16 = take(sizeof(__nv_bfloat16) * B * mpk);
    } else {
        L.At = bf16 ? take(sizeof(__nv_bfloat16) * (size_t)round_up(n, LG_TA) * (size_t)round_up(m, lg_tr<__nv_bfloat16>()))
                    : take(sizeof(float) * (size_t)round_up(n, LG_TA) * (size_t)round_up(m, lg_tr<float>()));
    }
    L.cblk = take(sizeof(int) * B);
    L.colmax = take(sizeof(float));
    L.ys = take(sizeof(const float*) * B);
    L.outs = take(sizeof(LargeOut) * B);
    L.kv = take(sizeof(int) * B);
    L.itv = take(sizeof(int) * B);
    L.y = take(sizeof(float) * B * mp);
    L.r = take(sizeof(float) * B * mp);
    L.c = take(sizeof(float) * B * n);
    L.mask = take(sizeof(uint32_t) * B * nw);
    L.cand = take(sizeof(int) * B * n);
    L.ncand = take(sizeof(int) * B);
    L.cmax = take(sizeof(unsigned) * B);
    L.best = take(sizeof(unsigned long long) * B);
    L.sup = take(sizeof(int) * B * K);
    L.gpart = take(sizeof(float) * B * nseg * (K + 2));
    L.gsum = take(sizeof(float) * B * (K + 2));
    L.W = cl ? 0 : take(sizeof(double) * B * 2 * K * K);
    L.z = take(sizeof(double) * B * K);
    L.x = take(sizeof(double) * B * K);
    L.xf = take(sizeof(float) * B * K);
    L.lpart = take(sizeof(double) * B * lch * K);
    L.l = take(sizeof(double) * B * K);
    L.upart = take(sizeof(double) * B * lch * K);
    L.scal = take(sizeof(double) * B * 2);
    L.rpart = take(sizeof(float) * B * rch * mp);
    L.nrm = take(sizeof(float) * B * (size_t)ceil_div(m, 256));
    {
        const size_t pbmax = K / 32, rbl = (size_t)ceil_div(m, 256);
        L.cnt = take(sizeof(unsigned) * B * ((K + 2) + 2 * pbmax + rbl + 2));
        L.pbpart = take(sizeof(double) * B * pbmax * 2);
    }
    L.rnorm = take(sizeof(float) * B);
    L.nit = take(sizeof(int) * B);
    L.st = take(sizeof(int) * B);
    L.live = take(sizeof(int));
    if (cl) {
        L.G = take(sizeof(float) * B * K * K);
        L.bv = take(sizeof(float) * B * K);
        L.s0 = take(sizeof(unsigned long long) * B * K);
        L.s1 = take(sizeof(unsigned long long) * B * K);
        L.am = take(sizeof(float) * B * K);
        L.av = take(sizeof(float) * B * K);
        L.gbar = take(sizeof(unsigned));
    }
    L.total = off;
    return L;
}

// Ring stages of the correlation with NB residuals in shared memory (0: it
// does not fit).
int lg_tma_stages(const LgState& S, int nb) {
    const size_t fixed = lg_tma_smem(0, nb, S.mpt);
    if (fixed >= (size_t)S.smem_optin) return 0;
    const int st = (int)(((size_t)S.smem_optin - fixed) / (LG_TILE_BYTES + 24));
    return st >= 2 ? std::min(st, LG_TMA_MAX_STAGES) : 0;
}

template <typename T, int NB>
cudaError_t launch_corr_tma(const LgState& S, cudaStream_t s) {
    const int stages = lg_tma_stages(S, NB);
    if (stages == 0) return cudaErrorInvalidValue;
    const size_t smem = lg_tma_smem(stages, NB, S.mpt);
    const cudaError_t attr = set_smem_limit((const void*)k_lg_corr_tma<T, NB>, S.smem_optin);
    if (attr != cudaSuccess) return attr;
    const int npass = ceil_div(S.Bl, NB);
    cudaError_t e = cudaMemsetAsync(S.cblk, 0, sizeof(int) * npass, s);
    if (e != cudaSuccess) return e;
    const dim3 grid(std::max(1, std::min(S.njb, S.nsm / npass)), npass);
    k_lg_corr_tma<T, NB><<<grid, LG_TMA_THREADS, smem, s>>>(S, stages);
    return cudaGetLastError();
}

// The GEMM correlation: N = the signals per pass rounded up to 16 (at most
// 256), as many ring stages as shared memory holds.
struct LgMma {
    CUtensorMap mapR;
    int N, stages, tmem_cols;
    size_t smem;
};

cudaError_t setup_corr_mma(const LgState& S, LgMma& M) {
    M.N = round_up(std::min(S.Bl, LG_MMA_MAXN), 16);
    M.tmem_cols = 32;
    while (M.tmem_cols < M.N) M.tmem_cols *= 2;
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, k_lg_corr_mma);
    if (e != cudaSuccess) return e;
    const int dyn_max = S.smem_optin - (int)fa.sharedSizeBytes;   // the dynamic part's limit
    const int stage_bytes = LG_MMA_ATILE + M.N * 128;
    M.stages = std::min(LG_MMA_MAX_STAGES, (dyn_max - 1024) / stage_bytes);   // 1024: alignment slack
    if (M.stages < 2) return cudaErrorInvalidValue;
    M.smem = (size_t)M.stages * stage_bytes + 1024;
    if (!make_tma_map_bf16(&M.mapR, S.R16, S.mpk, S.Bl, (size_t)S.mpk * 2, M.N))
        return cudaErrorInvalidValue;
    return set_smem_limit((const void*)k_lg_corr_mma, dyn_max);
}

cudaError_t launch_corr_mma(const LgState& S, const LgMma& M, cudaStream_t s) {
    const dim3 grid(ceil_div(S.n, 128), ceil_div(S.Bl, LG_MMA_MAXN));
    k_lg_corr_mma<<<grid, LG_MMA_THREADS, M.smem, s>>>(M.mapR, S, M.stages, M.N, M.tmem_cols);
    return cudaGetLastError();
}

// Correlation configuration cfg = 2 log2(NB): NB signals per pass.
cudaError_t launch_corr(const LgState& S, int cfg, cudaStream_t s) {
    const int nbl = cfg >> 1;
    if (S.bf16) {
        switch (nbl) {
            case 0: return launch_corr_tma<__nv_bfloat16, 1>(S, s);
            case 1: return launch_corr_tma<__nv_bfloat16, 2>(S, s);
            default: return launch_corr_tma<__nv_bfloat16, 4>(S, s);
        }
    }
    switch (nbl) {
        case 0: return launch_corr_tma<float, 1>(S, s);
        case 1: return launch_corr_tma<float, 2>(S, s);
        default: return launch_corr_tma<float, 4>(S, s);
    }
}

// The configurations that fit: NB residuals in shared memory beside at least
// two ring stages, no more signal slots than signals.
std::vector<int> corr_configs(const LgState& S) {
    std::vector<int> out;
    if (S.mma) return {LG_MMA_CFG};
    for (int nbl = 0; nbl <= 2; ++nbl) {
        const int nb = 1 << nbl;
        if (lg_tma_stages(S, nb) == 0) break;
        if (nb > 1 && nb / 2 >= S.Bl) break;
        out.push_back(2 * nbl);
    }
    return out;
}

}  // namespace

bool large_supported(int m, int n, int k) {
    return m >= 1 && m <= kLargeMaxM && n >= 1 && k >= 1 && k <= kLargeMaxK;
}

size_t large_ws_bytes(int m, int n, int Bl, int kmax, int bf16, int cl) {
    return lg_layout(m, n, Bl, kmax, bf16, cl).total;
}

cudaError_t large_solve(const LargeCall& call, void* ws, size_t ws_bytes, cudaStream_t s) {
    const int Bl = (int)call.ys.size();
    if (Bl == 0) return cudaSuccess;
    const int kmax = *std::max_element(call.ks.begin(), call.ks.end());
    const int cl = call.cl != nullptr ? 1 : 0;
    const LgLayout L = lg_layout(call.m, call.n, Bl, kmax, call.bf16, cl);
    if (L.total > ws_bytes) return cudaErrorInvalidValue;
    char* w = static_cast<char*>(ws);
    LgState S{};
    S.m = call.m;
    S.n = call.n;
    S.lda = call.lda;
    S.mp = round_up(call.m, 8);
    S.K = round_up(kmax, 32);
    S.nseg = ceil_div(call.m, LG_SEG);
    S.lch = ceil_div(S.K, LG_LC);
    S.rch = ceil_div(S.K, LG_RQ);
    S.Bl = Bl;
    S.bf16 = call.bf16;
    S.tol = call.tol;
    S.nb = 1;   // set from the chosen correlation configuration below
    S.A = call.A;
    S.mma = lg_uses_mma(call.bf16, Bl) ? 1 : 0;
    S.At = S.mma ? nullptr : w + L.At;
    S.mpt = round_up(call.m, call.bf16 ? lg_tr<__nv_bfloat16>() : lg_tr<float>());
    S.nc = S.mpt / (call.bf16 ? lg_tr<__nv_bfloat16>() : lg_tr<float>());
    S.njb = ceil_div(call.n, LG_TA);
    S.mpk = round_up(call.m, LG_MMA_KCH);
    S.Ak = S.mma ? reinterpret_cast<__nv_bfloat16*>(w + L.Ak) : nullptr;
    S.R16 = S.mma ? reinterpret_cast<__nv_bfloat16*>(w + L.R16) : nullptr;
    S.cblk = reinterpret_cast<int*>(w + L.cblk);
    {
        int dev = 0;
        cudaError_t e0 = cudaGetDevice(&dev);
        if (e0 == cudaSuccess) e0 = cudaDeviceGetAttribute(&S.nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e0 == cudaSuccess) e0 = cudaDeviceGetAttribute(&S.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e0 != cudaSuccess) return e0;
    }
    S.colmax = reinterpret_cast<float*>(w + L.colmax);
    S.ys = reinterpret_cast<const float* const*>(w + L.ys);
    S.outs = reinterpret_cast<const LargeOut*>(w + L.outs);
    S.kv = reinterpret_cast<const int*>(w + L.kv);
    S.itv = reinterpret_cast<const int*>(w + L.itv);
    S.y = reinterpret_cast<float*>(w + L.y);
    S.r = reinterpret_cast<float*>(w + L.r);
    S.c = reinterpret_cast<float*>(w + L.c);
    S.mask = reinterpret_cast<uint32_t*>(w + L.mask);
    S.cand = reinterpret_cast<int*>(w + L.cand);
    S.ncand = reinterpret_cast<int*>(w + L.ncand);
    S.cmax = reinterpret_cast<unsigned*>(w + L.cmax);
    S.best = reinterpret_cast<unsigned long long*>(w + L.best);
    S.sup = reinterpret_cast<int*>(w + L.sup);
    S.gpart = reinterpret_cast<float*>(w + L.gpart);
    S.gsum = reinterpret_cast<float*>(w + L.gsum);
    S.W = cl ? nullptr : reinterpret_cast<double*>(w + L.W);
    S.cl = cl;
    if (cl) {
        S.steps = call.cl->steps;
        S.reset = call.cl->reset;
        S.beta1 = call.cl->beta1;
        S.beta2 = call.cl->beta2;
        S.eps = call.cl->eps;
        S.tab = call.cl->tab;
        S.G = reinterpret_cast<float*>(w + L.G);
        S.bv = reinterpret_cast<float*>(w + L.bv);
        S.s0 = reinterpret_cast<unsigned long long*>(w + L.s0);
        S.s1 = reinterpret_cast<unsigned long long*>(w + L.s1);
        S.am = reinterpret_cast<float*>(w + L.am);
        S.av = reinterpret_cast<float*>(w + L.av);
        S.gbar = reinterpret_cast<unsigned*>(w + L.gbar);
    }
    S.errflag = call.errflag;
    S.z = reinterpret_cast<double*>(w + L.z);
    S.x = reinterpret_cast<double*>(w + L.x);
    S.xf = reinterpret_cast<float*>(w + L.xf);
    S.lpart = reinterpret_cast<double*>(w + L.lpart);
    S.l = reinterpret_cast<double*>(w + L.l);
    S.upart = reinterpret_cast<double*>(w + L.upart);
    S.scal = reinterpret_cast<double*>(w + L.scal);
    S.rpart = reinterpret_cast<float*>(w + L.rpart);
    S.nrm = reinterpret_cast<float*>(w + L.nrm);
    S.rblk = ceil_div(call.m, 256);
    S.pbmax = S.K / 32;
    {
        unsigned* c = reinterpret_cast<unsigned*>(w + L.cnt);
        S.cntG = c;
        S.cntL = S.cntG + (size_t)Bl * (S.K + 2);
        S.cntU = S.cntL + (size_t)Bl * S.pbmax;
        S.cntR = S.cntU + (size_t)Bl * S.pbmax;
        S.cntP = S.cntR + (size_t)Bl * S.rblk;
        S.cntN = S.cntP + Bl;
    }
    S.pbpart = reinterpret_cast<double*>(w + L.pbpart);
    S.rnorm = reinterpret_cast<float*>(w + L.rnorm);
    S.nit = reinterpret_cast<int*>(w + L.nit);
    S.st = reinterpret_cast<int*>(w + L.st);
    S.live = reinterpret_cast<int*>(w + L.live);

    // the per-signal tables (pageable host vectors: staged before the calls return)
    std::vector<int> itv(Bl);
    int iters = 0;
    for (int b = 0; b < Bl; ++b) {
        itv[b] = call.max_iter > 0 ? std::min(call.ks[b], call.max_iter) : call.ks[b];
        iters = std::max(iters, itv[b]);
    }
    cudaError_t e;
#define LG_TRY(x)                          \
    do {                                   \
        e = (x);                           \
        if (e != cudaSuccess) return e;    \
    } while (0)
    LG_TRY(cudaMemcpyAsync(w + L.ys, call.ys.data(), sizeof(const float*) * Bl, cudaMemcpyHostToDevice, s));
    LG_TRY(cudaMemcpyAsync(w + L.outs, call.outs.data(), sizeof(LargeOut) * Bl, cudaMemcpyHostToDevice, s));
    LG_TRY(cudaMemcpyAsync(w + L.kv, call.ks.data(), sizeof(int) * Bl, cudaMemcpyHostToDevice, s));
    LG_TRY(cudaMemcpyAsync(w + L.itv, itv.data(), sizeof(int) * Bl, cudaMemcpyHostToDevice, s));
    LG_TRY(cudaMemsetAsync(w + L.colmax, 0, sizeof(float), s));
    auto mark = [&](int phase, int after) {
        if (call.mark) call.mark(call.mark_ctx, phase, after);
    };
    LgMma mm{};
    if (S.mma) LG_TRY(setup_corr_mma(S, mm));
    LG_TRY(cudaMemsetAsync(S.cntG, 0, sizeof(unsigned) * (size_t)Bl * ((S.K + 2) + 2 * S.pbmax + S.rblk + 2), s));
    mark(CS_PHASE_SETUP, 0);
    if (S.mma)
        k_lg_prep_k<<<ceil_div(round_up(S.n, 128), 8), 256, 0, s>>>(S.A, S.lda, S.m, S.n, S.mpk, const_cast<__nv_bfloat16*>(S.Ak),
                                                     const_cast<float*>(S.colmax));
    else if (S.bf16)
        k_lg_prep<__nv_bfloat16><<<ceil_div(S.njb * LG_TA, 8), 256, 0, s>>>(
            S.A, S.lda, S.m, S.n, S.mpt, S.njb, static_cast<__nv_bfloat16*>(const_cast<void*>(S.At)),
            const_cast<float*>(S.colmax));
    else
        k_lg_prep<float><<<ceil_div(S.njb * LG_TA, 8), 256, 0, s>>>(
            S.A, S.lda, S.m, S.n, S.mpt, S.njb, static_cast<float*>(const_cast<void*>(S.At)),
            const_cast<float*>(S.colmax));
    LG_TRY(cudaGetLastError());
    k_lg_setup<<<Bl, 1024, 0, s>>>(S);
    LG_TRY(cudaGetLastError());
    mark(CS_PHASE_SETUP, 1);
    // correlation configuration: given, or tuned here on the first
    // iteration's data (the kernel is idempotent), or the widest that fits
    const std::vector<int> cfgs = corr_configs(S);
    int cfg = call.corr_cfg;
    if (cfg < 0 || std::find(cfgs.begin(), cfgs.end(), cfg) == cfgs.end()) {
        cfg = cfgs.back();
        if (call.tune && cfgs.size() > 1) {
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            LG_TRY(cudaEventCreate(&e0));
            LG_TRY(cudaEventCreate(&e1));
            float best_ms = 0.f;
            int best = -1;
            for (int cand : cfgs) {
                LgState T = S;
                T.nb = 1 << (cand >> 1);
                LG_TRY(launch_corr(T, cand, s));
                LG_TRY(cudaEventRecord(e0, s));
                for (int r = 0; r < 3; ++r) LG_TRY(launch_corr(T, cand, s));
                LG_TRY(cudaEventRecord(e1, s));
                float ms = 0.f;
                LG_TRY(cudaEventSynchronize(e1));
                LG_TRY(cudaEventElapsedTime(&ms, e0, e1));
                if (best < 0 || ms < best_ms) {
                    best_ms = ms;
                    best = cand;
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            cfg = best;
        }
    }
    if (call.chosen_cfg) *call.chosen_cfg = cfg;
    S.nb = 1 << (cfg >> 1);
    int* live_h = call.live_host;
    // CLOMP: the device's limits for the cooperative fit, the CTAs of it that
    // fit an SM per shared-memory size (cached), and the tag of the next step
    int coop = 0, nsm = 0, smem_optin = 0;
    std::map<int, int> per_sm;
    unsigned tag = 0;
    if (cl) {
        int dev = 0;
        LG_TRY(cudaGetDevice(&dev));
        LG_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
        if (call.no_coop) coop = 0;
        LG_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        LG_TRY(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        cudaFuncAttributes fa{};
        LG_TRY(cudaFuncGetAttributes(&fa, k_lgc_fit));
        smem_optin -= (int)fa.sharedSizeBytes;   // the dynamic part's limit
        LG_TRY(cudaFuncSetAttribute(k_lgc_fit, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin));
        LG_TRY(cudaMemsetAsync(S.s0, 0, sizeof(unsigned long long) * Bl * S.K, s));
        LG_TRY(cudaMemsetAsync(S.s1, 0, sizeof(unsigned long long) * Bl * S.K, s));
        LG_TRY(cudaMemsetAsync(S.gbar, 0, sizeof(unsigned), s));
    }
    // rows per CTA of the cooperative fit at t1 coordinates (0: it does not fit)
    auto fit_rows = [&](int t1, int& gx, int& smem) -> int {
        if (!coop || S.steps <= 0) return 0;
        // from 16 rows per CTA (two per warp; measured at n = 65536, m = 19661,
        // k = 2000: 16 rows 257 ms of fit per solve, 8 rows 307, 32 rows 422)
        for (int R = 16; R <= std::max(16, round_up(t1, 8)); R *= 2) {
            smem = (int)sizeof(float) * lg_fit_smem_floats(t1, R);
            if (smem > smem_optin) return 0;
            const int key = round_up(smem, 1024);
            auto f = per_sm.find(key);
            if (f == per_sm.end()) {
                int v = 0;
                if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_lgc_fit, 256, key) != cudaSuccess) v = 0;
                f = per_sm.emplace(key, v).first;
            }
            gx = ceil_div(t1, R);
            if ((long long)gx * Bl <= (long long)nsm * f->second) return R;
        }
        return 0;
    };
    for (int it = 0; it < iters; ++it) {
        const int t = it;
        mark(CS_PHASE_CORR, 0);
        if (S.mma) LG_TRY(launch_corr_mma(S, mm, s));
        else LG_TRY(launch_corr(S, cfg, s));
        mark(CS_PHASE_CORR, 1);
        mark(CS_PHASE_SELECT, 0);
        LG_TRY(launch_pdl(k_lg_scan, dim3(ceil_div(S.n, 256), Bl), dim3(256), 0, s, S));
        LG_TRY(launch_pdl(k_lg_rescore, dim3(std::max(LG_RESCORE_MIN_CTAS, 2 * S.nsm / Bl), Bl), dim3(1024), 0, s, S));
        LG_TRY(launch_pdl(k_lg_gram, dim3(ceil_div((t + 2) * S.nseg, 8), Bl), dim3(256), 0, s, S, t));
        mark(CS_PHASE_SELECT, 1);
        mark(CS_PHASE_FIT, 0);
        if (cl) {
            // Gram form: grow G and b, then the T Adam steps on t + 1 coordinates,
            // in one cooperative launch where the grid fits, else one launch per step
            LG_TRY(launch_pdl(k_lgc_append, dim3(ceil_div(t + 1, 256), Bl), dim3(256), 0, s, S, t, tag));
            const int tau0 = S.reset ? 0 : t * S.steps;
            int gx = 0, smem = 0;
            const int R = fit_rows(t + 1, gx, smem);
            if (R > 0) {
                int t1 = t + 1, r = R, tz = tau0;
                unsigned tg = tag;
                void* args[] = {&S, &t1, &r, &tz, &tg};
                LG_TRY(cudaLaunchCooperativeKernel((const void*)k_lgc_fit, dim3(gx, Bl), dim3(256), args,
                                                   (size_t)smem, s));
            } else {
                for (int step = 0; step < S.steps; ++step)
                    k_lgc_step<<<dim3(ceil_div(t + 1, 8), Bl), 256, 0, s>>>(S, t + 1, tau0 + step + 1,
                                                                           tag + (unsigned)step,
                                                                           step + 1 == S.steps ? 1 : 0);
            }
            tag += (unsigned)S.steps;
        } else {
            // one warp per CTA: the items spread over every SM (the float64
            // unit of one SM is narrow; eight warps on one SM queue on it)
            const int nl = t > 0 ? ceil_div(t, 32) * ceil_div(t, LG_LC) : 1;
            LG_TRY(launch_pdl(k_lg_lpiv, dim3(nl, Bl), dim3(32), 0, s, S, t));
            if (t > 0) LG_TRY(launch_pdl(k_lg_uupd, dim3(nl, Bl), dim3(32), 0, s, S, t));
        }
        mark(CS_PHASE_FIT, 1);
        mark(CS_PHASE_RESID, 0);
        LG_TRY(launch_pdl(k_lg_resid, dim3(S.rblk, ceil_div(t + 1, LG_RQ), Bl), dim3(256), 0, s, S, t + 1));
        mark(CS_PHASE_RESID, 1);
        LG_TRY(cudaGetLastError());
        // every 64 iterations: stop once no signal is running
        if (live_h && (it % 64) == 63 && it + 1 < iters) {
            k_lg_count<<<1, 32, 0, s>>>(S);
            LG_TRY(cudaMemcpyAsync(live_h, S.live, sizeof(int), cudaMemcpyDeviceToHost, s));
            LG_TRY(cudaStreamSynchronize(s));
            if (*live_h == 0) break;
        }
    }
    k_lg_out<<<Bl, 256, 0, s>>>(S);
    LG_TRY(cudaGetLastError());
#undef LG_TRY
    return cudaSuccess;
}

}  // namespace cs
