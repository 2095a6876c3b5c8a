// Persistent batched CLOMP (Methods, "Coefficients learning on OMP"; Gram-form
// fit) with the bf16 tensor-core correlation: the whole solve in one launch.
//
// One CTA per SM owns a block of up to 27 signals and runs every iteration of
// them on chip, so no iteration boundary costs a launch, a ramp-up or a tail:
//   * the bf16 atom tiles A16[128 atoms][64] stream by TMA through an 8-deep
//     ring, two stages for each of signal warps 1..4 (the copy rate of this
//     machine grows with the number of issuing warps, not with the ring
//     depth); A is the same in every iteration, so each pass's first tiles
//     are prefetched while the previous pass ends;
//   * one thread of warp 0 issues tcgen05.mma with M = 128 atoms, N = 32
//     signal columns, K = 16: the correlation c = A^T r of the block's
//     signals lands in tensor memory, 32 fp32 columns per atom tile, each
//     tile committed to its own mbarrier so that the epilogue starts on the
//     first tiles while the later ones are still streaming;
//   * warps 1..27 (one per signal) read the accumulators in two passes:
//     pass 1 finds each signal's largest masked bf16 |c| (a packed
//     value/index key, transposed max-reduction per 32 atoms), pass 2 lists
//     every atom within 2 delta of it (delta bounds |c_bf16 - c_fp32| as in
//     the per-iteration path).  Re-scoring that short list in float32 yields
//     the float32 argmax over all atoms.  The signal's warp then appends the
//     atom (Gram row from A^T A), runs the T Adam steps of the Gram-form fit,
//     forms the residual and stop test, and writes the residual as bf16
//     straight into the swizzled shared-memory B operand of the next MMAs.
// Every CTA runs a fixed schedule: k correlation passes per block of signals
// (rounds without a live signal skip the epilogue).
// Every wait is bounded: on time-out the CTA raises a device error flag,
// stops all roles, lets copies and MMAs in flight finish and frees its
// tensor memory.
#include "k_fit.cuh"
#include "k_resid.cuh"
#include "k_select.cuh"
#include "k_tc.cuh"

#include <algorithm>

namespace cs {
namespace {

constexpr int PS_NS = 27;                    // signals per block = signal warps
constexpr int PS_WARPS = PS_NS + 1;          // + one control warp (TMA producer, MMA issuer)
constexpr int PS_THREADS = 32 * PS_WARPS;
constexpr int PS_SIGTHREADS = 32 * PS_NS;
constexpr int PS_N = 32;                     // UMMA N: the block's signals, padded
constexpr int PS_TM = 128;                   // atoms per UMMA M tile (TMEM lanes)
constexpr int PS_KCH = 64;                   // bf16 per 128-byte swizzled row
constexpr int PS_TILE = PS_TM * PS_KCH * 2;  // 16 KiB atom tile
constexpr int PS_ST = 8;                     // atom-tile ring depth
constexpr int PS_PROD = 4;                   // producer warps (PS_ST / PS_PROD stages each)
constexpr int PS_BSTRIDE = PS_N * 128;       // bytes per 64-element K block of the B operand
constexpr int PS_MAXKB = 4;                  // m <= 256
constexpr int PS_CAP = 32;                   // candidates held per signal
constexpr int PS_KT = 32;                    // largest support
constexpr int PS_IDXB = 11;                  // atom-index bits of the packed key
constexpr int PS_MAXN = 1 << PS_IDXB;        // n <= 2048 (also: 16 tiles x 32 TMEM columns)
constexpr int PS_MAXCH = PS_MAXN / PS_TM;
constexpr int PS_TAB = 2048;                 // Adam factor pairs staged

// shared-memory carve-up (from a 1024-byte aligned base)
constexpr int PS_OFF_B = PS_ST * PS_TILE;
constexpr int PS_OFF_MASK = PS_OFF_B + PS_MAXKB * PS_BSTRIDE;
constexpr int PS_OFF_PART = PS_OFF_MASK + PS_MAXN * 4;
constexpr int PS_OFF_THETA = PS_OFF_PART + PS_MAXCH * 4 * 32 * 4;
constexpr int PS_OFF_CCOUNT = PS_OFF_THETA + 32 * 4;
constexpr int PS_OFF_CLIST = PS_OFF_CCOUNT + 32 * 4;
constexpr int PS_OFF_SVEC = PS_OFF_CLIST + 32 * PS_CAP * 4;
constexpr int PS_OFF_SUP = PS_OFF_SVEC + PS_NS * PS_KT * 4;     // support of each signal
constexpr int PS_OFF_CF = PS_OFF_SUP + PS_NS * PS_KT * 4;       // its coefficients
constexpr int PS_OFF_TAB = PS_OFF_CF + PS_NS * PS_KT * 4;
constexpr int PS_SMEM = PS_OFF_TAB + PS_TAB * 8 + 1024;

struct PsArgs {
    IterArgs a;
    ClArgs c;        // tau0 is derived per iteration
    int ns;          // signals per block
    int nblk;        // number of blocks
    int nslots;      // blocks per CTA (the last slot may be empty for some CTAs)
    int kb;          // K blocks of 64 (mh / 64)
    int nchunk;      // atom tiles, ceil(n / 128)
    int nres;        // leading atom tiles kept in tensor memory as the MMA A operand
    int tmem_cols;   // tensor-memory columns allocated (512)
    int staged;      // Adam table staged in shared memory
    int stall;       // test hook: withhold the last tile's completion signal in the first pass
};

__device__ __forceinline__ void named_sync() {
    asm volatile("barrier.sync 1, %0;" ::"n"(PS_SIGTHREADS) : "memory");
}

// Barrier over the signal warps that also ORs a predicate across them.
__device__ __forceinline__ bool named_sync_or(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "barrier.red.or.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(PS_SIGTHREADS)
        : "memory");
    return r != 0;
}

// Bounded wait that also gives up when *flag becomes non-zero:
// 1 = phase complete, 0 = flag raised, -1 = timed out.
__device__ __forceinline__ int wait_or_flag(uint64_t* bar, uint32_t parity, const volatile int* flag) {
    const unsigned long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*flag) return 0;
        if (clock64() - t0 > WAIT_CYCLES) return -1;
    }
    return 1;
}

// Transposed max-reduction: lane l ends with the maximum over the warp of
// k[l] (in k[0]).  31 shuffles.
__device__ __forceinline__ void warp_max_scatter32(uint32_t (&k)[32]) {
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

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15])
        : "r"(taddr));
}

// The four K = 16 MMAs of one 64-element K block (descriptors advance 32
// bytes per step inside the 128-byte swizzled rows); `first` clears the
// accumulator.
__device__ __forceinline__ void umma_kblock(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                           uint32_t first) {
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.eq.u32 p, %4, 0;\n\t"
        "setp.eq.u32 q, %4, %4;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %5, %6, %3, q;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %7, %8, %3, q;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %9, %10, %3, q;\n\t}\n"
        ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(first), "l"(adesc + 2), "l"(bdesc + 2),
          "l"(adesc + 4), "l"(bdesc + 4), "l"(adesc + 6), "l"(bdesc + 6)
        : "memory");
}

// Same with the A operand in tensor memory (8 columns per K = 16 step).
__device__ __forceinline__ void umma_kblock_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                              uint32_t first) {
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.eq.u32 p, %4, 0;\n\t"
        "setp.eq.u32 q, %4, %4;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%5], %6, %3, q;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%7], %8, %3, q;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%9], %10, %3, q;\n\t}\n"
        ::"r"(d_tmem), "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(first), "r"(a_tmem + 8), "l"(bdesc + 2),
          "r"(a_tmem + 16), "l"(bdesc + 4), "r"(a_tmem + 24), "l"(bdesc + 6)
        : "memory");
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, "
        "%17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};"
        ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
          "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]),
          "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]),
          "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}

// Residual row of signal s (row-sliced like load_row) as bf16 into the
// K-major, 128-byte-swizzled B operand: element k of row s sits in K block
// k/64, 8-row group s/8, row s%8, 16-byte chunk ((k%64)/8) ^ (s%8).
template <int MCH>
__device__ __forceinline__ void put_b_row(uint8_t* sB, int s, int mp, const float4 (&r)[MCH], bool zero) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < MCH; ++c) {
        const int k = (c * 32 + lane) * 4;
        if (k < mp) {
            const int kb = k >> 6, ch = (k & 63) >> 3, hf = (k >> 2) & 1;
            uint8_t* dst = sB + kb * PS_BSTRIDE + (s >> 3) * 1024 + (s & 7) * 128 + ((ch ^ (s & 7)) << 4) + hf * 8;
            __nv_bfloat162 lo = __floats2bfloat162_rn(zero ? 0.f : r[c].x, zero ? 0.f : r[c].y);
            __nv_bfloat162 hi = __floats2bfloat162_rn(zero ? 0.f : r[c].z, zero ? 0.f : r[c].w);
            uint2 v;
            v.x = *reinterpret_cast<uint32_t*>(&lo);
            v.y = *reinterpret_cast<uint32_t*>(&hi);
            *reinterpret_cast<uint2*>(dst) = v;
        }
    }
}

__device__ __forceinline__ void fit_dispatch(const IterArgs& a, const ClArgs& c, int b, int t, int tau0,
                                             float* sv, const float2* tab, float* coef_copy) {
    switch (round_up(t + 1, 8)) {
        case 8: fit_grid<8>(a, c, b, tau0, sv, tab, coef_copy); break;
        case 16: fit_grid<16>(a, c, b, tau0, sv, tab, coef_copy); break;
        case 24: fit_grid<24>(a, c, b, tau0, sv, tab, coef_copy); break;
        default: fit_grid<32>(a, c, b, tau0, sv, tab, coef_copy); break;
    }
}

// Support append of atom bj as the (t+1)-th atom of signal b (one warp; the
// same arithmetic as the per-iteration append_atom): support entry, Gram row
// and column from A^T A, A_S^T y entry.  The support sits in shared memory,
// so the Gram-row gathers leave together with the new column's loads.
template <int MCH>
__device__ __forceinline__ void append_ps(const IterArgs& a, const int b, const int t, const int bj,
                                          const float4 (&y)[MCH], const int* sup) {
    const int lane = threadIdx.x & 31;
    const float* garow = a.GA + (size_t)bj * a.n;
    const float g = (lane < t) ? garow[sup[lane]] : 0.f;
    const float gdd = garow[bj];
    float4 aj[MCH];
    load_row<MCH>(a.A32 + (size_t)bj * a.mp, a.mp, aj);
    float by = 0.f;
#pragma unroll
    for (int c = 0; c < MCH; ++c) by += dot4(aj[c], y[c]);
    by = warp_sum(by);
    float* G = a.G + (size_t)b * a.kmax * a.kmax;
    if (lane < t) {
        G[(size_t)t * a.kmax + lane] = g;
        G[(size_t)lane * a.kmax + t] = g;
    }
    if (lane == 0) {
        a.support[(size_t)b * a.k + t] = bj;
        G[(size_t)t * a.kmax + t] = gdd;
        a.bvec[(size_t)b * a.kmax + t] = by;
    }
}

template <int KB>
__global__ void __launch_bounds__(PS_THREADS, 1)
k_clomp_persist(const __grid_constant__ CUtensorMap mapA, const PsArgs p) {
    constexpr int MCH = (KB + 1) / 2;   // 128-row chunks of the fp32 vectors (m <= 64 KB)
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[PS_ST], empty_bar[PS_ST], chunk_bar[PS_MAXCH], rready_bar, fin_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ uint32_t live_bits[2];
    __shared__ volatile int abort_flag;

    const IterArgs& a = p.a;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t* base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    uint8_t* ring = base;
    uint8_t* sB = base + PS_OFF_B;
    uint32_t* mask_t = reinterpret_cast<uint32_t*>(base + PS_OFF_MASK);   // bit s: signal s holds the atom
    uint32_t* part = reinterpret_cast<uint32_t*>(base + PS_OFF_PART);     // [tile*4 + quadrant][32]
    float* theta = reinterpret_cast<float*>(base + PS_OFF_THETA);
    int* ccount = reinterpret_cast<int*>(base + PS_OFF_CCOUNT);
    int* clist = reinterpret_cast<int*>(base + PS_OFF_CLIST);
    float* svec = reinterpret_cast<float*>(base + PS_OFF_SVEC);
    float2* tabs = reinterpret_cast<float2*>(base + PS_OFF_TAB);
    int* sup_s = reinterpret_cast<int*>(base + PS_OFF_SUP);
    float* cf_s = reinterpret_cast<float*>(base + PS_OFF_CF);
    unsigned* errflag = a.counters + 1;

    if (tid == 0) {
        for (int i = 0; i < PS_ST; ++i) {
            mbar_init(&full_bar[i], 1);
            mbar_init(&empty_bar[i], 1);
        }
        mbar_init(&rready_bar, PS_NS);
        for (int i = 0; i < PS_MAXCH; ++i) mbar_init(&chunk_bar[i], 1);
        mbar_init(&fin_bar, 1);
        abort_flag = 0;
        live_bits[0] = live_bits[1] = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(p.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int i = tid; i < PS_MAXKB * PS_BSTRIDE / 16; i += PS_THREADS)
        reinterpret_cast<uint4*>(sB)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (tid < 32) {
        theta[tid] = __int_as_float(0x7f800000);
        ccount[tid] = 0;
    }
    if (p.staged)
        for (int i = tid; i < p.c.tab_len; i += PS_THREADS) tabs[i] = p.c.tab[i];
    tc_fence_before();
    __syncthreads();   // the allocation is visible
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    // Leading atom tiles, resident for the whole solve: tile (c, kk) of row
    // 128c + lane-of-quadrant sits in columns 32 (nchunk + c kb + kk) ...,
    // its 64 bf16 packed in pairs.  Work units (tile, lane quadrant) go to
    // the warps of that quadrant.
    {
        const int q = warp & 3;
        const int wq = warp >> 2, nwq = (PS_WARPS - q + 3) >> 2;   // warps of quadrant q
        const int row = 32 * q + lane;
        for (int u = wq; u < p.nres * KB; u += nwq) {
            const int c = u / KB, kk = u % KB;
            const int atom = c * PS_TM + row;
            uint32_t v[32];
            if (atom < a.n) {
                const uint4* src = reinterpret_cast<const uint4*>(a.A16 + (size_t)atom * a.mh + kk * PS_KCH);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const uint4 w4 = src[i];
                    v[4 * i] = w4.x;
                    v[4 * i + 1] = w4.y;
                    v[4 * i + 2] = w4.z;
                    v[4 * i + 3] = w4.w;
                }
            } else {
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = 0u;
            }
            tmem_st32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * (p.nchunk + u)), v);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const int passes = p.nslots * a.iters;
    const int per_pass = (p.nchunk - p.nres) * KB;            // streamed atom tiles per pass
    const uint32_t total = (uint32_t)passes * (uint32_t)per_pass;

    if (warp == 0) {
        // ------------------------------------------------ MMA issuer ------
        if (lane == 0) {
            constexpr uint32_t idesc = make_idesc(PS_TM, PS_N);
            uint64_t db[KB];   // B operand (the block's residuals), one descriptor per K block
#pragma unroll
            for (int kk = 0; kk < KB; ++kk) db[kk] = smem_desc_sw128(smem_u32(sB + kk * PS_BSTRIDE));
            const uint64_t da0 = smem_desc_sw128(smem_u32(ring));   // ring slot st: + st * PS_TILE / 16
            uint32_t gc = 0;   // tiles consumed
            bool ok = true;
            for (int pass = 0; pass < passes && ok; ++pass) {
                const int w = wait_or_flag(&rready_bar, (uint32_t)pass & 1u, &abort_flag);
                if (w <= 0) {
                    if (w < 0) atomicOr(errflag, 8u);
                    ok = false;
                    break;
                }
                tc_fence_after();
                for (int c = 0; c < p.nres; ++c) {
                    // resident tiles: A from tensor memory, no wait
                    const uint32_t ta = tmem + (uint32_t)(32 * (p.nchunk + c * KB));
#pragma unroll
                    for (int kk = 0; kk < KB; ++kk)
                        umma_kblock_ta(tmem + (uint32_t)(c * PS_N), ta + (uint32_t)(32 * kk), db[kk], idesc,
                                       kk == 0 ? 1u : 0u);
                    if (!(p.stall && pass == 0 && c == p.nchunk - 1)) umma_commit(&chunk_bar[c]);
                }
                for (int c = p.nres; c < p.nchunk && ok; ++c) {
#pragma unroll
                    for (int kk = 0; kk < KB; ++kk) {
                        const int st = gc % PS_ST;
                        if (!mbar_try_wait(&full_bar[st], (gc / PS_ST) & 1u)) {
                            const int w2 = wait_or_flag(&full_bar[st], (gc / PS_ST) & 1u, &abort_flag);
                            if (w2 <= 0) {
                                if (w2 < 0) atomicOr(errflag, 8u);
                                ok = false;
                                break;
                            }
                        }
                        tc_fence_after();
                        umma_kblock(tmem + (uint32_t)(c * PS_N), da0 + (uint64_t)(st * (PS_TILE >> 4)), db[kk], idesc,
                                    kk == 0 ? 1u : 0u);
                        umma_commit(&empty_bar[st]);   // frees the ring slot once these MMAs are done
                        ++gc;
                    }
                    // this atom tile's accumulators are complete (the test hook
                    // withholds the signal once, so that the readers time out)
                    if (ok && !(p.stall && pass == 0 && c == p.nchunk - 1)) umma_commit(&chunk_bar[c]);
                }
            }
            if (!ok) abort_flag = 1;
            // every MMA issued so far completes before teardown
            umma_commit(&fin_bar);
            if (!mbar_wait(&fin_bar, 0)) atomicOr(errflag, 8u);
        }
    } else {
        // ------------------------------------------------ signal warps ----
        const int s = warp - 1;
        const int q = warp & 3;                       // TMEM lane quadrant this warp may read
        const int qfirst = (q >= 1) ? q : 4;          // first signal warp of the quadrant
        const int qidx = (warp - qfirst) >> 2;
        const int qcnt = (PS_WARPS - qfirst + 3) >> 2;   // signal warps of the quadrant
        const float cert = (0x1p-7f + 0x1p-16f + (float)a.m * (0x1p-22f + 0x1p-23f)) * (*a.colnorm_max) * 1.01f;
        uint32_t rnd = 0;
        bool aborted = false;
        // producer s (signal warps 1..PS_PROD): tiles s, s + PS_PROD, ...
        const bool producer = (s < PS_PROD) && lane == 0;
        uint32_t pg = (uint32_t)s;   // next tile this producer issues
        for (int slot = 0; slot < p.nslots && !aborted; ++slot) {
            const int blk = blockIdx.x + slot * gridDim.x;
            const bool have = blk < p.nblk;
            const int b = blk * p.ns + s;
            const bool mine = have && s < p.ns && b < a.B;
            bool live = false;
            int t = 0;
            float rho = 0.f;
            float4 r[MCH];   // the residual, kept in registers from one iteration to the next
            named_sync();   // every warp is done with the previous block's selected-atom bits
            for (int i = tid - 32; i < p.nchunk * PS_TM; i += PS_SIGTHREADS) mask_t[i] = 0u;
            {
                float4 y[MCH];
#pragma unroll
                for (int c2 = 0; c2 < MCH; ++c2) y[c2] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (mine) {
                    load_row<MCH>(a.Y32 + (size_t)b * a.mp, a.mp, y);
                    live = a.status[b] < 0;
                    rho = a.res_norm[b];
                }
                put_b_row<MCH>(sB, s, a.mp, y, !live);
#pragma unroll
                for (int c2 = 0; c2 < MCH; ++c2) r[c2] = y[c2];
            }
            // k rounds per block whatever the signals do (a fixed schedule);
            // rounds without a live signal skip the epilogue
            for (int it = 0; it < a.iters; ++it, ++rnd) {
                if (lane == 0 && live) atomicOr(&live_bits[rnd & 1u], 1u << s);
                const bool any = named_sync_or(live);
                if (warp == 1 && lane == 0) live_bits[(rnd + 1) & 1u] = 0u;
                fence_proxy_async_smem();   // the B rows written above, for the tensor core
                __syncwarp();
                if (lane == 0) mbar_arrive(&rready_bar);
                if (producer) {
                    // this pass's tiles of my stage, then the next pass's first
                    // ones: tile g reuses the slot of tile g - ST, which this
                    // or the previous pass consumes (g < (pass+1) per_pass + ST)
                    const uint32_t lim = min(total, (rnd + 1u) * (uint32_t)per_pass + (uint32_t)PS_ST);
                    for (; pg < lim; pg += PS_PROD) {
                        const int st = pg % PS_ST;
                        if (pg >= (uint32_t)PS_ST) {
                            const int we = wait_or_flag(&empty_bar[st], ((pg / PS_ST) & 1u) ^ 1u, &abort_flag);
                            if (we <= 0) {
                                if (we < 0) {
                                    abort_flag = 1;
                                    atomicOr(errflag, 4u);
                                }
                                break;
                            }
                        }
                        const int tile = (int)(pg % (uint32_t)per_pass) + p.nres * KB;
                        mbar_arrive_expect_tx(&full_bar[st], PS_TILE);
                        tma_load_2d(ring + st * PS_TILE, &mapA, &full_bar[st], (tile % KB) * PS_KCH,
                                    (tile / KB) * PS_TM);
                    }
                }
                __syncwarp();
                if (!any) {
                    // nothing to read this pass; still wait for it (its last
                    // tile's commit covers every MMA of the pass), so that no
                    // warp arrives for the next pass before the MMA issuer has
                    // seen this one
                    const int w = wait_or_flag(&chunk_bar[p.nchunk - 1], rnd & 1u, &abort_flag);
                    if (w < 0 && lane == 0) {
                        abort_flag = 1;
                        atomicOr(errflag, 16u);
                    }
                    if (named_sync_or(w <= 0)) {
                        aborted = true;
                        break;
                    }
                    continue;
                }
                const uint32_t lb = live_bits[rnd & 1u];

                // pass 1: per 32 atoms x 32 signals, the largest masked key per
                // signal, each atom tile as soon as its MMAs have completed
                bool failed = false;
                for (int c = qidx; c < p.nchunk && !failed; c += qcnt) {
                    const int w = wait_or_flag(&chunk_bar[c], rnd & 1u, &abort_flag);
                    if (w <= 0) {
                        if (w < 0 && lane == 0) {
                            abort_flag = 1;
                            atomicOr(errflag, 16u);
                        }
                        failed = true;
                        break;
                    }
                    tc_fence_after();
                    uint32_t k[32];
                    tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(c * PS_N), k);
                    tmem_ld_wait();
                    const int atom = c * PS_TM + 32 * q + lane;
                    const uint32_t mw = ((atom < a.n) ? mask_t[atom] : 0xffffffffu) | ~lb;
                    const uint32_t ilo = (uint32_t)((PS_MAXN - 1) - atom);
#pragma unroll
                    for (int i = 0; i < 32; ++i)
                        k[i] = ((mw >> i) & 1u) ? 0u : (((k[i] & 0x7fffffffu) & ~(uint32_t)(PS_MAXN - 1)) | ilo);
                    warp_max_scatter32(k);
                    part[(c * 4 + q) * 32 + lane] = k[0];
                }
                if (named_sync_or(failed)) {
                    aborted = true;
                    break;
                }
                // threshold of my signal: largest bf16 |c| minus 2 delta
                {
                    uint32_t km = 0u;
                    if (live)
                        for (int e = lane; e < p.nchunk * 4; e += 32) km = max(km, part[e * 32 + s]);
                    km = __reduce_max_sync(0xffffffffu, km);
                    // (no usable key: every unselected atom becomes a candidate)
                    float th = __int_as_float(0x7f800000);
                    if (live)
                        th = (km == 0u) ? __int_as_float(0xff800000)
                                        : __uint_as_float(km & ~(uint32_t)(PS_MAXN - 1)) - 2.f * cert * rho;
                    if (lane == 0) theta[s] = th;
                }
                named_sync();
                // pass 2: list the atoms at or above the threshold.  A block of
                // 32 atoms whose pass-1 key bounds every |c| of a signal below
                // its threshold (value bits with the truncated low bits set)
                // cannot hold a candidate of that signal; blocks with no such
                // signal are skipped.
                for (int c = qidx; c < p.nchunk; c += qcnt) {
                    const uint32_t kb_ = part[(c * 4 + q) * 32 + lane];   // this block's key for signal `lane`
                    const float th_l = theta[lane];
                    const bool hot = !(th_l > 0.f) ||
                                     __uint_as_float((kb_ & ~(uint32_t)(PS_MAXN - 1)) | (uint32_t)(PS_MAXN - 1)) >= th_l;
                    const uint32_t hotmask = __ballot_sync(0xffffffffu, hot);
                    if (hotmask == 0u) continue;
                    const int atom = c * PS_TM + 32 * q + lane;
                    const uint32_t mw = ((atom < a.n) ? mask_t[atom] : 0xffffffffu) | ~lb | ~hotmask;
                    uint32_t hit = 0u;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        uint32_t v[16];
                        tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(c * PS_N + 16 * h), v);
                        tmem_ld_wait();
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            hit |= (fabsf(__uint_as_float(v[i])) >= theta[16 * h + i] ? 1u : 0u) << (16 * h + i);
                    }
                    hit &= ~mw;
                    while (hit) {
                        const int i = __ffs(hit) - 1;
                        hit &= hit - 1u;
                        const int pos = atomicAdd(&ccount[i], 1);
                        if (pos < PS_CAP) clist[i * PS_CAP + pos] = atom;
                    }
                }
                tc_fence_before();
                named_sync();

                if (live) {
                    // ---- selection: float32 re-score of the listed atoms
                    const int cnt = ccount[s];
                    float bv = -1.f;
                    int bj = -1;
                    if (cnt <= PS_CAP) {
                        const int my = (lane < cnt) ? clist[s * PS_CAP + lane] : -1;
                        for (int u0 = 0; u0 < cnt; u0 += 4) {
                            float pr[4];
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                const int j = __shfl_sync(0xffffffffu, my, (u0 + u) & 31);
                                pr[u] = 0.f;
                                if (u0 + u < cnt) {
                                    const float4* col = reinterpret_cast<const float4*>(a.A32 + (size_t)j * a.mp);
#pragma unroll
                                    for (int cc = 0; cc < MCH; ++cc) {
                                        const int i4 = cc * 32 + lane;
                                        if (i4 * 4 < a.mp) pr[u] += dot4(col[i4], r[cc]);
                                    }
                                }
                            }
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                const float v = fabsf(warp_sum(pr[u]));
                                const int j = __shfl_sync(0xffffffffu, my, (u0 + u) & 31);
                                if (u0 + u < cnt && cand_better(v, j, bv, bj)) {
                                    bv = v;
                                    bj = j;
                                }
                            }
                        }
                    } else {
                        // list overflow: float32 scan of every unselected atom
                        for (int j0 = 0; j0 < a.n; j0 += 32) {
                            const int j = j0 + lane;
                            const bool ok = j < a.n && !((mask_t[j] >> s) & 1u);
                            float v = fabsf(warp_dots32<MCH>(a.A32, a.mp, ok ? j : -1, r));
                            int jj = ok ? j : -1;
                            warp_argmax(v, jj);
                            if (cand_better(v, jj, bv, bj)) {
                                bv = v;
                                bj = jj;
                            }
                        }
                        if (lane == 0) atomicAdd(&a.counters[0], 1u);
                    }
                    if (lane == 0) ccount[s] = 0;
                    if (bj < 0) {
                        // nothing left to select
                        live = false;
                        if (lane == 0) a.status[b] = CS_SIG_MAX_ITER;
                    } else {
                        if (lane == 0) {
                            atomicOr(&mask_t[bj], 1u << s);
                            sup_s[s * PS_KT + t] = bj;
                        }
                        float4 y[MCH];
                        load_row<MCH>(a.Y32 + (size_t)b * a.mp, a.mp, y);
                        append_ps<MCH>(a, b, t, bj, y, sup_s + s * PS_KT);
                        __syncwarp();
                        // ---- Gram-form Adam fit on the t+1 support atoms
                        const int tau0 = p.c.reset ? 0 : t * p.c.steps;
                        fit_dispatch(a, p.c, b, t, tau0, svec + s * PS_KT, (p.staged ? tabs : p.c.tab) + tau0,
                                     cf_s + s * PS_KT);
                        __syncwarp();
                        ++t;
                        // ---- residual, stop test, next B operand row
                        r[0] = y[0];
#pragma unroll
                        for (int c2 = 1; c2 < MCH; ++c2) r[c2] = y[c2];
                        resid_vector_from<MCH>(a, t, r, sup_s + s * PS_KT, cf_s + s * PS_KT);
                        float ss = 0.f;
#pragma unroll
                        for (int c2 = 0; c2 < MCH; ++c2) {
                            const int i4 = c2 * 32 + lane;
                            if (i4 * 4 < a.mp) ss += dot4(r[c2], r[c2]);
                        }
                        rho = sqrtf(warp_sum(ss));
                        if (lane == 0) stop_test(a, b, t, rho);
                        live = !((double)rho <= a.tol || t >= a.k || t >= a.iters);
                        if (live) put_b_row<MCH>(sB, s, a.mp, r, false);
                    }
                }
            }
        }
        // the last copies of my stages (the only ones that can still be in
        // flight after an abort) land before the CTA exits
        if (producer)
            for (uint32_t g2 = (pg >= (uint32_t)PS_ST) ? pg - PS_ST : (uint32_t)s; g2 < pg; g2 += PS_PROD)
                if (!mbar_wait(&full_bar[g2 % PS_ST], (g2 / PS_ST) & 1u)) atomicOr(errflag, 4u);
    }

    // ---------------------------------------------------------- teardown --
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tmem_cols)
                     : "memory");
    }
}

int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

}  // namespace

bool clomp_persist_supported(const IterArgs& a, const ClArgs& c) {
    return a.R16 != nullptr && a.need_gram && a.GA != nullptr && a.mh <= PS_MAXKB * PS_KCH &&
           a.n <= PS_MAXN && a.k <= PS_KT && c.steps >= 0;
}

namespace {

template <int KB>
cudaError_t configure_smem() {
    return set_smem_limit((const void*)k_clomp_persist<KB>, PS_SMEM);
}

template <int KB>
cudaError_t launch_kb(const IterArgs& a, const ClArgs& c, int stall, cudaStream_t s) {
    cudaError_t e = configure_smem<KB>();
    if (e != cudaSuccess) return e;
    PsArgs p{};
    p.a = a;
    p.c = c;
    p.kb = a.mh / PS_KCH;
    p.nchunk = ceil_div(a.n, PS_TM);
    // tensor memory: the accumulators (32 columns per atom tile), and as many
    // whole leading atom tiles as fit in the rest of the 512 columns
    p.tmem_cols = 512;
    p.nres = std::min(p.nchunk, (512 - p.nchunk * PS_N) / (32 * p.kb));
    p.staged = c.tab_len <= PS_TAB ? 1 : 0;
    p.stall = stall;
    // one CTA per SM, blocks of <= PS_NS signals
    const int nsm = sm_count();
    const int grid0 = std::min(nsm, a.B);
    p.ns = std::min(PS_NS, ceil_div(a.B, grid0));
    p.nblk = ceil_div(a.B, p.ns);
    const int grid = std::min(grid0, p.nblk);
    p.nslots = ceil_div(p.nblk, grid);
    CUtensorMap mA;
    if (!make_tma_map_bf16(&mA, a.A16, a.mh, a.n, (size_t)a.mh * 2, PS_TM)) return cudaErrorInvalidValue;
    k_clomp_persist<KB><<<grid, PS_THREADS, PS_SMEM, s>>>(mA, p);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_clomp_persist(const IterArgs& a, const ClArgs& c, int stall, cudaStream_t s) {
    if (!clomp_persist_supported(a, c)) return cudaErrorNotSupported;
    switch (a.mh / PS_KCH) {
        case 1: return launch_kb<1>(a, c, stall, s);
        case 2: return launch_kb<2>(a, c, stall, s);
        case 3: return launch_kb<3>(a, c, stall, s);
        default: return launch_kb<4>(a, c, stall, s);
    }
}

}  // namespace cs
