// Internal declarations shared by the CUDA translation units of the library.
// Nothing here is part of the public C ABI (include/cs_omp.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include <vector>

#include "cs_omp.h"

namespace cs {

constexpr int kKmaxLimit = 64;     // largest support size the per-signal kernels hold on chip
constexpr int kMaxRowChunks = 8;   // m <= 8 * 128 = 1024 for the warp-per-signal kernels
constexpr int kCorrFp32TileN = 128;   // atoms per CTA of the fp32 correlation
constexpr int kCorrTcTileN = 256;     // atoms per CTA of the tensor-core correlation
constexpr int kTopcMax = 8;          // candidates re-scored in float32 per signal (bf16 mode)
constexpr int kTcGroup = 16;         // bf16 mode keeps the two largest |c| of every 16-atom group
constexpr int kTcCandPerTile = 2 * kCorrTcTileN / kTcGroup;   // 32 candidates per 256-atom tile
constexpr int kGramAMax = 4096;      // n up to which A^T A is precomputed per solve
constexpr int kCorrTcMaxN = 4096;    // candidate merge holds <= 512 per signal
constexpr int kIhtMaxN = 4096;       // IHT: u = s + t c of a signal in shared memory
constexpr int kLargeMaxM = 32768;    // large-instance solves: rows (residual staged in shared memory)
constexpr int kLargeMaxK = 4096;     // large-instance solves: support size (OMP float64 W = L^{-T}, CLOMP G in HBM)

// Candidate slots per signal, enough for either correlation kernel.
__host__ __device__ inline int cand_slots(int n) {
    const int a = (n + kCorrFp32TileN - 1) / kCorrFp32TileN;
    const int b = ((n + kCorrTcTileN - 1) / kCorrTcTileN) * kTcCandPerTile;
    return a > b ? a : b;
}

__host__ __device__ inline int round_up(int x, int a) { return (x + a - 1) / a * a; }
__host__ __device__ inline int ceil_div(int x, int a) { return (x + a - 1) / a; }

// State of one batched solve, passed by value to every per-iteration kernel.
// Layouts (B = batch, K = kmax of the plan):
//   A32   [n][mp]  float, column j of A at A32 + j*mp, zero-padded rows
//   A16   [n][mh]  bf16 copy of A32 (tensor-core operand), mh = m rounded up to 64
//   Y32   [B][mp]  float, measurements, zero-padded
//   R32   [B][mp]  float residual;  R16 [B][mh] bf16 residual (tensor-core operand)
//   mask  [B][nw]  selected-atom bitset
//   cand  [B][nch][topc]  candidate |c| and atom index per atom tile (fp32: best of
//                   each 128-atom tile; bf16: two best of each 16-atom group, unsorted)
//   cbound [B][n/16]     bf16: third largest |c| of each 16-atom group (bounds the
//                   group's atoms that are not candidates)
//   GA    [n][n]   Gram matrix of A (n <= kGramAMax), row j = a_j^T A
//   gcol  [B][K]   Gram column A_S^T a_j of the new atom (float)
//   L     [B][2][K][K] W = L^{-T} of the Cholesky factor L (double), by rows then
//                   by columns; z, x64 [B][K] (double)
//   G     [B][K][K] Gram matrix of the support (float, CLOMP Gram form), bvec [B][K]
//   am, av [B][K]  Adam moments; tau [B] Adam step counter
//   support, coef [B][k] (caller outputs, k = params.k)
struct IterArgs {
    int m, n, B, k, kmax, iters, mp, mh, nw, nch, topc, prec;
    double tol;
    const float* A32;
    const __nv_bfloat16* A16;
    float* Y32;
    float* R32;
    __nv_bfloat16* R16;
    // FP8 (E4M3) correlation: A8 [n][mq] with per-column scales sa (a_j ~ sa_j
    // A8_j), ea_max = max_j ||a_j - sa_j A8_j||; R8 [B][mq] with per-signal
    // scales sr and quantisation-error norms er; mq = m rounded up to 128
    const uint8_t* A8;
    const float* sa;
    const float* ea_max;
    uint8_t* R8;
    float* sr;
    float* er;
    int mq;
    uint32_t* mask;
    float* cand_val;
    int* cand_idx;
    float* cand_bound;
    float* gcol;
    float* dnorm;
    float* bt;
    double* L;
    double* z;
    double* x64;
    float* G;
    float* bvec;
    float* am;
    float* av;
    int* tau;
    const float* GA;            // n x n Gram matrix A^T A (nullptr: gather the columns instead)
    const float* colnorm_max;   // max_j ||a_j||_2 (for the bf16 certificate)
    unsigned* counters;         // [0] bf16 certificate fallbacks, [1] device error flags
    int* support;
    float* coef;
    int* n_iter;
    float* res_norm;
    int* status;
    int tc_tile;     // atoms per CTA of the tensor-core correlation (128 or 256; nch, topc follow)
    int need_gcol;   // OMP: write gcol/dnorm/bt for the Cholesky update
    int need_gram;   // CLOMP Gram form: maintain G and bvec
};

struct ClArgs {
    int steps;
    float th;            // selection threshold Th (0 < th < 1: threshold rule; else one atom)
    int tau0;            // Adam step counter before this fit (the same for every live signal)
    float beta1, beta2, eps;
    int reset;
    const float2* tab;   // [tab_len] pairs (lr/(1-b1^tau), 1/sqrt(1-b2^tau)) for tau = 1..tab_len
    int tab_len;
};

// Output pointers of one uneven-batch instance.
struct VarlenOut {
    int* support;
    float* coef;
    int* n_iter;
    float* res_norm;
    int* status;
};

// An uneven-batch instance that is not solved (CS_SIG_UNSUPPORTED): its
// outputs, measurement vector, length m and sparsity k.
struct VarlenRefuse {
    VarlenOut o;
    const float* y;
    int m, k;
};

// Large OMP solves (k_large.cu): signals sharing the caller's A (m x n,
// leading dimension lda), each with its own measurement vector, sparsity and
// outputs (device pointers; support and coef hold k entries).
struct LargeOut {
    int* support;
    float* coef;
    int* n_iter;
    float* res_norm;
    int* status;
    int k;
};
struct LargeCall {
    const float* A;
    int m, n, lda;
    std::vector<const float*> ys;
    std::vector<LargeOut> outs;
    std::vector<int> ks;
    int max_iter;          // <= 0: k
    double tol;
    int bf16;              // 1: correlate with a bf16 copy of A (certified, re-scored in float32)
    int* live_host;        // host int for the early end of the iteration loop (NULL: none)
    // measurement hook: called around each launch with (ctx, CS_PHASE_*, 0 before / 1 after)
    void (*mark)(void* ctx, int phase, int after);
    void* mark_ctx;
    // correlation configuration (2 log2(signals per pass) of the streamed form):
    // corr_cfg >= 0 uses it; otherwise tune != 0 times the candidates on the
    // first iteration, else the widest that fits; the choice goes to *chosen_cfg
    int corr_cfg;
    int tune;
    int* chosen_cfg;
    // CLOMP in Gram form (NULL: plain OMP): steps, betas, eps, reset and the
    // Adam factor table (tab) of the solve
    const struct ClArgs* cl;
    // 1: no cooperative launch (the solve runs beside others on the device:
    // a cooperative grid's CTAs could not all be resident)
    int no_coop;
    // device error flags (bit 32: a grid-wide barrier of the CLOMP fit gave up)
    unsigned* errflag;
};
bool large_supported(int m, int n, int k);
size_t large_ws_bytes(int m, int n, int Bl, int kmax, int bf16, int cl);
// Runs a whole solve on `s` (synchronising `s` every 64 iterations to end
// early once every signal has stopped, when live_host is set).
cudaError_t large_solve(const LargeCall& call, void* ws, size_t ws_bytes, cudaStream_t s);

// ---- launchers (defined in the .cu files) --------------------------------
// Outputs of refused instances: support -1, coef 0, n_iter 0, res_norm ||y||,
// status CS_SIG_UNSUPPORTED (one warp each).
cudaError_t launch_varlen_refuse(const VarlenRefuse* items, int count, cudaStream_t s);
cudaError_t launch_varlen_gather(const float* const* ys, int m, int B, float* Y, cudaStream_t s);
cudaError_t launch_varlen_scatter(const VarlenOut* outs, int k, int B, const int* support, const float* coef,
                                  const int* n_iter, const float* res_norm, const int* status, cudaStream_t s);
cudaError_t launch_prep_A(const float* A, int lda, int m, int n, int mp, int mh, float* A32,
                          __nv_bfloat16* A16, float* colnorm_max, cudaStream_t s);
// FP8 copy of A: A8 [n][mq] (E4M3, zero padded), per-column scales sa and
// the largest quantisation-error norm (ea_max, zeroed by the caller first).
cudaError_t launch_prep_A8(const float* A, int lda, int m, int n, int mq, uint8_t* A8, float* sa, float* ea_max,
                           cudaStream_t s);
cudaError_t launch_setup(const IterArgs& a, const float* Y, int ldy, int clomp, cudaStream_t s);
cudaError_t launch_adam_table(float2* tab, int len, float lr, float beta1, float beta2,
                              cudaStream_t s);
cudaError_t launch_corr_fp32(const IterArgs& a, cudaStream_t s);
cudaError_t launch_corr_fp32_dense(const float* R32, const float* A32, int mp, int B, int n, float* C,
                                   int ldc, cudaStream_t s);
// C^T = R^T A (B x n, row stride ldc) in float32 for the live signals' tiles
cudaError_t launch_corr_fp32_dense_live(const IterArgs& a, float* C, int ldc, cudaStream_t s);
cudaError_t launch_corr_tc(const IterArgs& a, cudaStream_t s);
cudaError_t launch_corr_tc_dense(const __nv_bfloat16* R16, const __nv_bfloat16* A16, int mh, int B, int n,
                                 float* C, int ldc, unsigned* errflag, cudaStream_t s);
// FP8 tensor-core correlation, dense output C^T[b][j] = sr_b sa_j (R8_b . A8_j).
cudaError_t launch_corr_tc8_dense(const uint8_t* R8, const uint8_t* A8, const float* sr, const float* sa, int mq,
                                  int B, int n, float* C, int ldc, unsigned* errflag, cudaStream_t s);
// GA = A^T A from the padded float32 copy (mp <= kMaxRowChunks * 128), each
// entry bit-identical to the selection's on-the-fly Gram entry
cudaError_t launch_gram_A(const float* A32, int mp, int n, float* GA, cudaStream_t s);
// T = E^T E of a [n][ep] matrix (any ep that is a multiple of 4)
cudaError_t launch_gram_tiled(const float* E, int ep, int n, float* T, cudaStream_t s);
// Total-variation prior (Eq. 5): GA += lambda (Delta D)^T (Delta D), D N x n
// (ld ldd; nullptr: the identity, N = n); E [n][Ep] and T [n][n] are scratch.
cudaError_t launch_tv_prior(const float* D, int N, int ldd, int n, float lambda, float* E, int Ep, float* T,
                            float* GA, cudaStream_t s);
cudaError_t launch_prep_R(const float* R, int ldr, int m, int B, int mp, int mh, float* R32,
                          __nv_bfloat16* R16, cudaStream_t s);
cudaError_t launch_prep_R8(const float* R, int ldr, int m, int B, int mq, uint8_t* R8, float* sr, float* er,
                           cudaStream_t s);
bool corr_tc_supported(int m, int n);
// 2-D bf16 TMA map over `rows` rows of `row_elems` elements (a multiple of 64,
// byte stride row_bytes): box 64 x box_rows, 128-byte swizzle, zero fill.
bool make_tma_map_bf16(CUtensorMap* map, const void* base, int row_elems, int rows, size_t row_bytes,
                       int box_rows);
bool clomp_persist_supported(const IterArgs& a, const ClArgs& c);
// stall: test hook, withhold one completion signal of the first pass (see CS_OPT_STALL_TEST)
cudaError_t launch_clomp_persist(const IterArgs& a, const ClArgs& c, int stall, cudaStream_t s);
cudaError_t launch_select(const IterArgs& a, cudaStream_t s);
cudaError_t launch_chol(const IterArgs& a, cudaStream_t s);
// Whole plain-OMP solves (float32 correlation), one CTA per signal, one launch.
bool omp_fused_supported(const IterArgs& a);
// A fits the kernel's shared memory: then it may read the caller's A and Y
// (A != nullptr) and do the set-up itself, needing no other launch.
bool omp_fused_self_contained(const IterArgs& a);
cudaError_t launch_omp_fused(const IterArgs& a, const float* A, int lda, const float* Y, int ldy, cudaStream_t s);
cudaError_t launch_resid(const IterArgs& a, cudaStream_t s);
cudaError_t launch_clfit_gram(const IterArgs& a, const ClArgs& c, int iter, cudaStream_t s);
// CL fit with the image priors of Eq. 6 and 7 (k_image_prior.cu): images of
// W consecutive columns, one thread-block cluster per image; lam_h = 2 w_tv / W,
// lv_scale = w_lv / ((H-2)(W-2)) (0: no local variation), lv_eps: the window
// deviation's smoothing, D: H x n (nullptr: x = s).
bool clfit_image_supported(const IterArgs& a, int W, bool lv, int H);
cudaError_t clfit_image_prepare(int W, bool lv, int H, int* ok);
cudaError_t launch_clfit_image(const IterArgs& a, const ClArgs& c, int iter, int W, float lam_h, float lv_scale,
                               float lv_eps, const float* D, int H, int ldd, cudaStream_t s);
cudaError_t launch_clfit_gather(const IterArgs& a, const ClArgs& c, int iter, cudaStream_t s);

// Raises `kernel`'s dynamic shared-memory limit to `bytes` on the current
// device, once per (device, kernel, bytes): a kernel attribute belongs to the
// device's context, so every device that launches the kernel needs its own.
// Thread-safe.
cudaError_t set_smem_limit(const void* kernel, int bytes);
bool update_clomp_fused_supported(const IterArgs& a);
cudaError_t launch_update_clomp(const IterArgs& a, const ClArgs& c, int iter, cudaStream_t s);
// Threshold rule (0 < c.th < 1): one iteration's selection, Gram-form fit,
// residual and stop test from the float32 correlation C (B x n, stride ldc).
// Column-wise 2D output: X[:, b] = D[:, support] coef (one warp per signal), and
// per-image PSNR / SSIM of H x W column-major images against references.
cudaError_t launch_synthesize(const float* D, int N, int n, int ldd, const int* support, const float* coef,
                              const int* n_iter, int k, int B, float* X, int ldx, cudaStream_t s);
cudaError_t launch_image_quality(const float* X, const float* R, int H, int W, int count, float peak,
                                 float* psnr, float* ssim, cudaStream_t s);
// IHT (k_iht.cu): one iteration's H_k(s + step c) from the float32
// correlation C (B x n, row stride ldc), the dense s (sd, B x n), the
// residual and the stopping rule (iteration `it` of a.iters).
bool iht_supported(const IterArgs& a);
cudaError_t launch_iht_update(const IterArgs& a, const float* C, int ldc, float* sd, float step, int it,
                              cudaStream_t s);
bool clomp_th_supported(const IterArgs& a);
cudaError_t launch_clomp_th(const IterArgs& a, const ClArgs& c, const float* C, int ldc, int iter, cudaStream_t s);

cudaError_t launch_clfit_forward(const float* A, int m, int lda, const int32_t* S, const float* Sv,
                                 int t, int lds, const float* Y, int ldy, int batch, float* R,
                                 int ldr, float* loss, cudaStream_t s);
cudaError_t launch_clfit_adjoint(const float* A, int m, int lda, const int32_t* S, float* Sv,
                                 int t, int lds, const float* R, int ldr, int batch, float* grad,
                                 float* mom, float* vel, int tau, float lr, float beta1,
                                 float beta2, float eps, int adam, cudaStream_t s);

// Programmatic dependent launch: the kernel may start (and run its prologue)
// while its predecessor in the stream finishes.  Such a kernel must call
// pdl_wait() before it touches anything written by earlier kernels; it calls
// pdl_trigger() to let its own successor launch early.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ---- device helpers -------------------------------------------------------
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float dot4(float4 a, float4 b) {
    return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, a.x * b.x)));
}

// Candidate order: larger |c| first, lower atom index on equal |c|; j < 0 is empty.
__device__ __forceinline__ bool cand_better(float v, int j, float bv, int bj) {
    if (j < 0) return false;
    if (bj < 0) return true;
    return v > bv || (v == bv && j < bj);
}

// Warp-wide (max |c|, lowest atom on ties) with two redux.sync instructions.
// Valid entries have j >= 0 and v >= 0 (non-negative floats order like their
// bit patterns); the result is (-1, -1) when no lane holds a valid entry.
__device__ __forceinline__ void warp_argmax(float& v, int& j) {
    const unsigned key = (j >= 0) ? __float_as_uint(v) : 0u;
    const unsigned mx = __reduce_max_sync(0xffffffffu, key);
    const int cand = (j >= 0 && key == mx) ? j : 0x7fffffff;
    const int jmin = __reduce_min_sync(0xffffffffu, cand);
    j = (jmin == 0x7fffffff) ? -1 : jmin;
    v = (j >= 0) ? __uint_as_float(mx) : -1.f;
}

// Transposing reduction: every lane holds v[0..31]; afterwards v[0] of lane l
// holds the sum over the warp of v[l].  31 shuffles.
__device__ __forceinline__ void warp_reduce_scatter32(float (&v)[32]) {
    const unsigned lane = threadIdx.x & 31u;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < off; ++i) {
            float send = upper ? v[i] : v[i + off];
            float keep = upper ? v[i + off] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
}
#endif

}  // namespace cs
