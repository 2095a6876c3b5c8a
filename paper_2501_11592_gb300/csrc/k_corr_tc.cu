// K1: bf16 or FP8 (E4M3) tensor-core correlation C^T = R^T A on sm_103a
// (tcgen05 + TMA), fp32 accumulation in tensor memory, fused masked top-c
// epilogue.  In FP8 mode the operands carry per-atom and per-signal scales
// (a_j ~ sa_j A8_j, r_b ~ sr_b R8_b) applied in the epilogue; a 128-element
// E4M3 row is the same 128-byte swizzled row as 64 bf16 elements, so the
// staging, the descriptors and the four MMAs per chunk are the same.
//
// The residual-injection branch (Methods, "Coefficients learning on OMP")
// applies the fixed layer A to r^T for all signals at once -- a GEMM with
// M = signals, N = atoms, K = m.  Both operands are K-major (one residual /
// one column of A is contiguous), which is the native operand layout of
// tcgen05.mma:
//   * one CTA owns 128 signals x 256 atoms; the residual tile (128 x m) and
//     the atom tile (256 x m) are staged by TMA in 64-element K chunks with
//     the 128-byte swizzle, one mbarrier per chunk, so the MMAs of chunk 0
//     start while later chunks are still in flight;
//   * one thread issues 4 x tcgen05.mma (M=128, N=256, K=16) per chunk into a
//     256-column fp32 accumulator in tensor memory;
//   * 16 warps (four per TMEM lane quadrant, 64 columns each) read their
//     32 lanes (= 32 signals) with tcgen05.ld, mask already-selected atoms,
//     take |c|, and keep for every 16-atom group its two best atoms and the
//     third value (a bound on the rest of the group) -- C itself never
//     reaches global memory.
// Every wait is bounded; on time-out the kernel raises a device error flag,
// skips the epilogue, frees its tensor memory and returns.
#include <algorithm>
#include <cstdio>
#include <mutex>

#include "k_tc.cuh"

namespace cs {
namespace {

constexpr int TM = 128;              // signals per CTA (UMMA M, TMEM lanes)
constexpr int KCH = 64;              // bf16 elements per 128-byte swizzled row
constexpr int KCH8 = 128;            // E4M3 elements per 128-byte swizzled row
constexpr int R_CHUNK_BYTES = TM * 128;   // 16 KiB
constexpr int MAX_KC = 4;            // m <= 256 staged at once
// The tile width TN (atoms per CTA: UMMA N, TMEM columns) is a template
// parameter, 128 or 256, chosen per problem size by the autotuner; the
// candidates are the same two per 16-atom group either way.
constexpr int a_chunk_bytes(int TN) { return TN * 128; }
struct TcArgs {
    int B, n, kc, nch, topc, nw;
    const uint32_t* mask;
    const int* status;
    float* cand_val;
    int* cand_idx;
    float* cand_bound;
    float* dense;       // optional dense output C^T (B x n, row stride ldd); nullptr = top-c only
    int ldd;
    unsigned* errflag;
    const float* sa;    // FP8: per-atom scales
    const float* sr;    // FP8: per-signal scales
};

constexpr int NTHREADS = 512;          // 16 warps: four per TMEM lane quadrant
constexpr int NPART = NTHREADS / 128;  // column parts per quadrant

template <bool FP8, int TN>
__global__ void __launch_bounds__(NTHREADS, 1)
k_corr_tc(const __grid_constant__ CUtensorMap mapR, const __grid_constant__ CUtensorMap mapA, TcArgs p) {
    static_assert(TN == 128 || TN == 256, "UMMA N for M=128");
    constexpr int KEL = FP8 ? KCH8 : KCH;   // elements per chunk row
    constexpr int HALF = TN / NPART;        // columns per epilogue warp (32 or 64)
    constexpr int CPT = 2 * TN / kTcGroup;  // candidates per tile
    constexpr int A_CHUNK_BYTES = a_chunk_bytes(TN);
    extern __shared__ uint8_t smem_raw[];
    __shared__ float sSa[FP8 ? TN : 1];     // FP8: the tile's atom scales
    __shared__ __align__(8) uint64_t full_bar[MAX_KC];
    __shared__ __align__(8) uint64_t done_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int failed;
    __shared__ uint32_t sMask[TM][TN / 32];     // selected-atom bits of the tile (past n: set)

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3;           // TMEM lanes 32*quad .. 32*quad+31
    const int half = warp >> 2;          // column part: half*HALF .. +HALF-1
    const int b0 = blockIdx.x * TM;
    const int j0 = blockIdx.y * TN;

    if (tid == 0) failed = 0;

    // 1024-byte aligned operand tiles (128-byte swizzle atoms)
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t pad = ((raw + 1023u) & ~1023u) - raw;
    uint8_t* sR = smem_raw + pad;                       // kc x 16 KiB
    uint8_t* sA = sR + (size_t)p.kc * R_CHUNK_BYTES;    // kc x 32 KiB

    // Prologue that reads nothing earlier kernels wrote: it overlaps the
    // tail of the previous kernel (programmatic dependent launch).
    if (tid == 0) {
        for (int c = 0; c < p.kc; ++c) mbar_init(&full_bar[c], 1);
        mbar_init(&done_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(TN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    pdl_wait();

    // Skip tiles whose signals have all stopped.
    int live_here = 0;
    if (tid < TM) {
        const int b = b0 + tid;
        live_here = (p.dense != nullptr || (b < p.B && p.status[b] < 0)) ? 1 : 0;
    }
    if (!__syncthreads_or(live_here)) {
        if (warp == 1) {
            tc_fence_after();
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN) : "memory");
        }
        return;
    }

    // Bitset words of the tile's 128 signals x 256 atoms, loaded coalesced
    // while TMA and the MMAs run (read by the epilogue after the barrier).
    if (!p.dense) {
        for (int e = tid; e < TM * (TN / 32); e += NTHREADS) {
            const int sl = e / (TN / 32), w = e % (TN / 32);
            const int sg = b0 + sl, wb = j0 + 32 * w;
            uint32_t bits = 0xffffffffu;
            if (sg < p.B && wb < p.n) {
                bits = p.mask[(size_t)sg * p.nw + (wb >> 5)];
                if (p.n - wb < 32) bits |= ~0u << (p.n - wb);
            }
            sMask[sl][w] = bits;
        }
    }
    if constexpr (FP8) {
        for (int e = tid; e < TN; e += NTHREADS) sSa[e] = (j0 + e < p.n) ? p.sa[j0 + e] : 0.f;
    }

    if (tid == 0) {
        // producer: all K chunks of both operands, one barrier per chunk
        for (int c = 0; c < p.kc; ++c) {
            mbar_arrive_expect_tx(&full_bar[c], R_CHUNK_BYTES + A_CHUNK_BYTES);
            tma_load_2d(sR + (size_t)c * R_CHUNK_BYTES, &mapR, &full_bar[c], c * KEL, b0);
            tma_load_2d(sA + (size_t)c * A_CHUNK_BYTES, &mapA, &full_bar[c], c * KEL, j0);
        }
    } else if (tid == 32) {
        // MMA issuer
        constexpr uint32_t idesc = FP8 ? make_idesc_e4m3(TM, TN) : make_idesc(TM, TN);
        bool ok = true;
        for (int c = 0; c < p.kc && ok; ++c) {
            if (!mbar_wait(&full_bar[c], 0)) { ok = false; break; }
            tc_fence_after();
            const uint64_t da = smem_desc_sw128(smem_u32(sR + (size_t)c * R_CHUNK_BYTES));
            const uint64_t db = smem_desc_sw128(smem_u32(sA + (size_t)c * A_CHUNK_BYTES));
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                // advance 32 bytes along K inside the swizzled row (16 bf16 / 32 E4M3 elements)
                if constexpr (FP8)
                    umma_e4m3(tmem, da + (uint64_t)(2 * k), db + (uint64_t)(2 * k), idesc, (c | k) != 0);
                else
                    umma_bf16(tmem, da + (uint64_t)(2 * k), db + (uint64_t)(2 * k), idesc, (c | k) != 0);
            }
        }
        if (!ok) {
            failed = 1;
            atomicOr(p.errflag, 1u);
        }
        umma_commit(&done_bar);   // arrives once every issued MMA has completed
    }

    const bool waited = mbar_wait(&done_bar, 0);
    tc_fence_after();
    if (!waited && lane == 0) atomicOr(p.errflag, 2u);
    // block-uniform verdict (also the barrier after which the operand tiles,
    // no longer read by any MMA, are reused as epilogue scratch)
    const bool ok = __syncthreads_and(waited && !failed) != 0;
    const int sig = b0 + quad * 32 + lane;
    const bool live = sig < p.B;
    const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(half * HALF);
    const int a0 = j0 + half * HALF;     // first atom of this warp's half
    // FP8: c = sr_b sa_j acc (the signal's scale here, the atom's per value)
    const float srow = (FP8 && live) ? p.sr[sig] : 1.f;

    if (ok && p.dense) {
        for (int c0 = 0; c0 < HALF; c0 += 32) {
            uint32_t v[32];
            tmem_ld32(tbase + (uint32_t)c0, v);
            tmem_ld_wait();
            if (!live) continue;
            for (int q = 0; q < 32; ++q) {
                const int atom = a0 + c0 + q;
                float x = __uint_as_float(v[q]);
                if constexpr (FP8) x = x * sSa[half * HALF + c0 + q] * srow;
                if (atom < p.n) p.dense[(size_t)sig * p.ldd + atom] = x;
            }
        }
    } else if (ok) {
        // Per 16-atom group: the two largest masked |c| (lower atom first on
        // ties) become candidates, the third largest bounds every other atom
        // of the group.  Branch-free, ~11 instructions per value.  Results go
        // to shared memory first (the operand tiles are free now) and leave
        // the CTA in contiguous 128-byte rows per signal.
        constexpr int SV = CPT + 1;                             // padded row strides
        constexpr int SB = TN / kTcGroup + 1;
        float* sVal = reinterpret_cast<float*>(sR);             // [TM][SV]
        int* sIdx = reinterpret_cast<int*>(sVal + TM * SV);     // [TM][SV]
        float* sBnd = reinterpret_cast<float*>(sIdx + TM * SV); // [TM][SB]
        const int sl = quad * 32 + lane;
        constexpr int PER_HALF = 2 * HALF / kTcGroup;          // candidates per part
#pragma unroll
        for (int c = 0; c < HALF / 32; ++c) {
            const uint32_t mw = sMask[sl][half * (HALF / 32) + c];
            uint32_t v[32];
            tmem_ld32(tbase + (uint32_t)(32 * c), v);
            tmem_ld_wait();
#pragma unroll
            for (int g = 0; g < 32 / kTcGroup; ++g) {
                float m1 = -1.f, m2 = -1.f, m3 = -1.f;
                int i1 = 0, i2 = 0;
#pragma unroll
                for (int q = 0; q < kTcGroup; ++q) {
                    const int qq = kTcGroup * g + q;
                    float cv = __uint_as_float(v[qq]);
                    if constexpr (FP8) cv = cv * sSa[half * HALF + 32 * c + qq] * srow;
                    const float x = ((mw >> qq) & 1u) ? -1.f : fabsf(cv);
                    const bool gt1 = x > m1, gt2 = x > m2;
                    m3 = gt2 ? m2 : fmaxf(m3, x);
                    m2 = gt1 ? m1 : (gt2 ? x : m2);
                    i2 = gt1 ? i1 : (gt2 ? qq : i2);
                    m1 = gt1 ? x : m1;
                    i1 = gt1 ? qq : i1;
                }
                const int e = half * PER_HALF + 4 * c + 2 * g;
                sVal[sl * SV + e] = m1;
                sIdx[sl * SV + e] = (m1 >= 0.f) ? a0 + 32 * c + i1 : -1;
                sVal[sl * SV + e + 1] = m2;
                sIdx[sl * SV + e + 1] = (m2 >= 0.f) ? a0 + 32 * c + i2 : -1;
                sBnd[sl * SB + half * (HALF / kTcGroup) + 2 * c + g] = m3;
            }
        }
        __syncthreads();
        for (int e = tid; e < TM * CPT; e += NTHREADS) {
            const int r = e / CPT, q = e % CPT;
            const int sg = b0 + r;
            if (sg < p.B) {
                const size_t o = ((size_t)sg * p.nch + blockIdx.y) * CPT + q;
                p.cand_val[o] = sVal[r * SV + q];
                p.cand_idx[o] = sIdx[r * SV + q];
            }
        }
        constexpr int G = TN / kTcGroup;
        for (int e = tid; e < TM * G; e += NTHREADS) {
            const int r = e / G, q = e % G;
            const int sg = b0 + r;
            if (sg < p.B) p.cand_bound[((size_t)sg * p.nch + blockIdx.y) * G + q] = sBnd[r * SB + q];
        }
    }
    pdl_trigger();   // after the epilogue: the successor only overlaps our teardown
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN) : "memory");
    }
}

// ---- host side: tensor maps through the driver entry point (no libcuda link)
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn get_encode() {
    static EncodeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(f);
    });
    return fn;
}

// 2-D map over rows of `row_elems` elements (bf16: a multiple of 64; fp8: of
// 128) with byte stride `row_bytes`; box = one 128-byte row x box_rows,
// 128-byte swizzle, zero fill outside.
bool make_map(CUtensorMap* map, const void* base, int row_elems, int rows, size_t row_bytes, int box_rows,
              bool fp8 = false) {
    EncodeFn enc = get_encode();
    if (!enc) return false;
    cuuint64_t gdim[2] = {(cuuint64_t)row_elems, (cuuint64_t)rows};
    cuuint64_t gstride[1] = {(cuuint64_t)row_bytes};
    cuuint32_t box[2] = {(cuuint32_t)(fp8 ? KCH8 : KCH), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                     const_cast<void*>(base), gdim, gstride, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

size_t smem_bytes(int kc, int TN) { return (size_t)kc * (R_CHUNK_BYTES + a_chunk_bytes(TN)) + 1024; }

// R and A operand rows of `rowlen` elements (bf16: 2 bytes, fp8: 1 byte).
// At most two CTAs share an SM (tensor memory: 2 x 256 columns), or four
// with TN = 128.
template <bool FP8, int TN>
cudaError_t launch_tc(const void* R, const void* A, int rowlen, int B, int n, TcArgs p, cudaStream_t s) {
    CUtensorMap mR, mA;
    const size_t rb = (size_t)rowlen * (FP8 ? 1 : 2);
    if (!make_map(&mR, R, rowlen, B, rb, TM, FP8) || !make_map(&mA, A, rowlen, n, rb, TN, FP8))
        return cudaErrorInvalidValue;
    const size_t smem = std::max(smem_bytes(p.kc, TN), (size_t)(TN == 256 ? 100 : 50) * 1024);
    const cudaError_t e = set_smem_limit((const void*)k_corr_tc<FP8, TN>, (int)smem_bytes(MAX_KC, TN));
    if (e != cudaSuccess) return e;
    dim3 grid(ceil_div(B, TM), ceil_div(n, TN));
    return launch_pdl(k_corr_tc<FP8, TN>, grid, dim3(NTHREADS), smem, s, mR, mA, p);
}

template <bool FP8>
cudaError_t launch_tc_w(const void* R, const void* A, int rowlen, int B, int n, TcArgs p, int tn, cudaStream_t s) {
    return tn == 128 ? launch_tc<FP8, 128>(R, A, rowlen, B, n, p, s) : launch_tc<FP8, 256>(R, A, rowlen, B, n, p, s);
}

}  // namespace

bool make_tma_map_bf16(CUtensorMap* map, const void* base, int row_elems, int rows, size_t row_bytes,
                       int box_rows) {
    return make_map(map, base, row_elems, rows, row_bytes, box_rows);
}

bool corr_tc_supported(int m, int n) {
    return m >= 1 && m <= MAX_KC * KCH && n >= 1 && n <= kCorrTcMaxN && get_encode() != nullptr;
}

cudaError_t launch_corr_tc(const IterArgs& a, cudaStream_t s) {
    const bool fp8 = a.prec == CS_CORR_FP8;
    TcArgs p{};
    p.B = a.B;
    p.n = a.n;
    p.kc = fp8 ? a.mq / KCH8 : a.mh / KCH;
    p.nch = a.nch;
    p.topc = a.topc;
    p.nw = a.nw;
    p.mask = a.mask;
    p.status = a.status;
    p.cand_val = a.cand_val;
    p.cand_idx = a.cand_idx;
    p.cand_bound = a.cand_bound;
    p.dense = nullptr;
    p.errflag = a.counters + 1;
    const int tn = a.tc_tile == 128 ? 128 : 256;
    if (fp8) {
        p.sa = a.sa;
        p.sr = a.sr;
        return launch_tc_w<true>(a.R8, a.A8, a.mq, a.B, a.n, p, tn, s);
    }
    return launch_tc_w<false>(a.R16, a.A16, a.mh, a.B, a.n, p, tn, s);
}

cudaError_t launch_corr_tc_dense(const __nv_bfloat16* R16, const __nv_bfloat16* A16, int mh, int B, int n,
                                 float* C, int ldc, unsigned* errflag, cudaStream_t s) {
    TcArgs p{};
    p.B = B;
    p.n = n;
    p.kc = mh / KCH;
    p.nch = 1;
    p.topc = 1;
    p.nw = 1;
    p.dense = C;
    p.ldd = ldc;
    p.errflag = errflag;
    return launch_tc<false, 256>(R16, A16, mh, B, n, p, s);
}

cudaError_t launch_corr_tc8_dense(const uint8_t* R8, const uint8_t* A8, const float* sr, const float* sa, int mq,
                                  int B, int n, float* C, int ldc, unsigned* errflag, cudaStream_t s) {
    TcArgs p{};
    p.B = B;
    p.n = n;
    p.kc = mq / KCH8;
    p.nch = 1;
    p.topc = 1;
    p.nw = 1;
    p.dense = C;
    p.ldd = ldc;
    p.errflag = errflag;
    p.sa = sa;
    p.sr = sr;
    return launch_tc<true, 256>(R8, A8, mq, B, n, p, s);
}

}  // namespace cs
