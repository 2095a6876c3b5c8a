// Host runtime of the library: plan/workspace management, argument
// validation, the per-iteration launch sequence and the C ABI declared in
// include/cs_omp.h.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "cs_internal.cuh"

using namespace cs;

namespace {

thread_local std::string g_last_error;

cs_status fail(cs_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

cs_status cuda_fail(cudaError_t e, const char* where) {
    return fail(CS_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CS_TRY_LAUNCH(expr, what)                         \
    do {                                                  \
        cudaError_t e_ = (expr);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    cudaError_t err = cudaSuccess;
    explicit DeviceGuard(int dev) {
        err = cudaGetDevice(&prev);
        if (err == cudaSuccess && prev != dev) {
            err = cudaSetDevice(dev);
            changed = (err == cudaSuccess);
        }
    }
    ~DeviceGuard() {
        if (changed) cudaSetDevice(prev);
    }
};

}  // namespace

struct cs_plan {
    int device = 0;
    int m_max = 0, n_max = 0, B_max = 0, k_max = 0;
    int k_user = 0;            // the plan's k_max as created (k_max: the on-chip kernels' 32 or 64)
    int no_large = 0;          // 1: never run the large-instance path (it allocates)
    char* lg = nullptr;        // workspace of the large-instance path, on first use
    size_t lg_bytes = 0;
    // workers that run an uneven batch's large OMP groups side by side: a
    // stream, a workspace and a completion event each (made on first use)
    struct LgWorker {
        cudaStream_t s = nullptr;
        char* ws = nullptr;
        size_t bytes = 0;
        cudaEvent_t done = nullptr;
    };
    std::vector<LgWorker> lgw;
    int mp_max = 0, mh_max = 0, nw_max = 0, nch_max = 0;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    float* A32 = nullptr;
    __nv_bfloat16* A16 = nullptr;
    uint8_t* A8 = nullptr;     // FP8 copy of A, its per-column scales and largest error norm
    float* sa = nullptr;
    float* ea = nullptr;
    uint8_t* R8 = nullptr;     // FP8 residuals, per-signal scales and error norms
    float* sr = nullptr;
    float* er = nullptr;
    float* Y32 = nullptr;
    float* R32 = nullptr;
    __nv_bfloat16* R16 = nullptr;
    uint32_t* mask = nullptr;
    float* cand_val = nullptr;
    int* cand_idx = nullptr;
    float* cand_bound = nullptr;
    float* gcol = nullptr;
    float* dnorm = nullptr;
    float* bt = nullptr;
    double* L = nullptr;
    double* z = nullptr;
    double* x64 = nullptr;
    float* G = nullptr;
    float* bvec = nullptr;
    float* am = nullptr;
    float* av = nullptr;
    int* tau = nullptr;
    float* colnorm_max = nullptr;
    float* GA = nullptr;       // n_max x n_max when n_max <= kGramAMax
    unsigned* counters = nullptr;
    float2* tab = nullptr;     // Adam bias-correction table, grown on demand
    int tab_cap = 0;
    float* cbuf = nullptr;     // B_max x n_max float32 correlations (threshold rule, IHT), on first use
    float* ihts = nullptr;     // B_max x n_max dense IHT coefficients, on first use
    float* tvE = nullptr;      // TV prior: differenced basis [n][Ep] (grown on demand)
    size_t tvE_cap = 0;
    float* tvT = nullptr;      // TV prior: (Delta D)^T (Delta D), n_max x n_max, on first use
    char* io = nullptr;        // device staging for the host-buffer entry points
    size_t io_bytes = 0;
    char* vl = nullptr;        // device staging for uneven batches
    size_t vl_bytes = 0;
    // measurement: launch counts per phase (always) and, when profiling is
    // enabled, CUDA event pairs around every launch
    int64_t launches[CS_PHASES] = {};
    int profiling = 0;
    struct Mark { int phase; cudaEvent_t a, b; };
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> pool;
    // CUDA graphs of whole solves, keyed by every argument the launches bake
    // in: the first call of a configuration runs eagerly, the second is
    // captured on a private stream, later ones replay the graph.
    struct GraphEntry {
        cudaGraphExec_t exec = nullptr;
        int seen = 0;
        int64_t launches[CS_PHASES] = {};
    };
    int use_graphs = 1;
    int fuse_update = 1;       // CLOMP Gram form: one fused kernel per iteration
    int persist = 1;           // CLOMP Gram form, bf16: one persistent kernel per solve
    int stall_test = 0;        // test hook: the next persistent solve lets a bounded wait run out
    int fused_omp = 1;         // plain OMP (fp32), at most one signal per SM: one kernel per solve
    int autotune = 1;          // time candidate tile shapes on the first solve of a size class
    int force_tile = 0;        // 128 / 256: tensor-core correlation tile width (0: tuned or 256)
    std::map<std::string, int> tuned;   // size class -> chosen configuration
    // A's preparation (fp32 / bf16 copies, largest column norm, A^T A) kept
    // for later solves with the same A and generation (generation 0: never)
    uint64_t a_gen = 0;
    struct Prep {
        const void* A = nullptr;   // the caller's A (device, or host for the host-buffer calls)
        int m = 0, n = 0, lda = 0;
        uint64_t gen = 0;
        int bf16 = 0, fp8 = 0, gram = 0;
    } prep;
    const void* a_host = nullptr;   // set by the host-buffer solve around its call of solve()
    int img_ready = 0, img_ready_h = 0;   // image shape whose cluster launch was checked
    cudaStream_t cap_stream = nullptr;
    std::map<std::string, GraphEntry> graphs;
};

namespace {

struct Carver {
    size_t off = 0;
    template <class T>
    size_t take(size_t count) {
        off = (off + 255) & ~size_t(255);
        size_t o = off;
        off += count * sizeof(T);
        return o;
    }
};

// Device workspace layout of a solve, shared by plans and the allocation-free
// entry point.  clomp: CLOMP state (G, bvec, Adam moments); gram_a: the
// n x n Gram matrix of A.
struct WsLayout {
    size_t A32, A16, A8, sa, ea, Y32, R32, R16, R8, sr, er, mask, cval, cidx, cbound, gcol, dnorm, bt, L, z, x64,
        G, bvec, am, av, tau, colnorm, counters, GA, total;
};

WsLayout ws_layout(int m, int n, int B, int K, bool clomp, bool gram_a) {
    const size_t Bm = (size_t)B, Kk = (size_t)K;
    const size_t mp = round_up(m, 4), mh = round_up(m, 64), mq = round_up(m, 128), nw = ceil_div(n, 32);
    const size_t slots = cand_slots(n), tiles = ceil_div(n, kCorrTcTileN);
    Carver cv;
    WsLayout L{};
    L.A32 = cv.take<float>((size_t)n * mp);
    L.A16 = cv.take<__nv_bfloat16>((size_t)n * mh);
    L.A8 = cv.take<uint8_t>((size_t)n * mq);
    L.sa = cv.take<float>(n);
    L.ea = cv.take<float>(1);
    L.Y32 = cv.take<float>(Bm * mp);
    L.R32 = cv.take<float>(Bm * mp);
    L.R16 = cv.take<__nv_bfloat16>(Bm * mh);
    L.R8 = cv.take<uint8_t>(Bm * mq);
    L.sr = cv.take<float>(Bm);
    L.er = cv.take<float>(Bm);
    L.mask = cv.take<uint32_t>(Bm * nw);
    L.cval = cv.take<float>(Bm * slots);
    L.cidx = cv.take<int>(Bm * slots);
    L.cbound = cv.take<float>(Bm * tiles * (kCorrTcTileN / kTcGroup));
    L.gcol = cv.take<float>(Kk * Bm);
    L.dnorm = cv.take<float>(Bm);
    L.bt = cv.take<float>(Bm);
    L.L = cv.take<double>(2 * Kk * Kk * Bm);
    L.z = cv.take<double>(Kk * Bm);
    L.x64 = cv.take<double>(Kk * Bm);
    if (clomp) {
        L.G = cv.take<float>(Bm * Kk * Kk);
        L.bvec = cv.take<float>(Bm * Kk);
        L.am = cv.take<float>(Bm * Kk);
        L.av = cv.take<float>(Bm * Kk);
    }
    L.tau = cv.take<int>(Bm);
    L.colnorm = cv.take<float>(1);
    L.counters = cv.take<unsigned>(16);
    if (gram_a) L.GA = cv.take<float>((size_t)n * n);
    L.total = cv.off;
    return L;
}

void bind_workspace(cs_plan* P, char* w, const WsLayout& L) {
    P->A32 = reinterpret_cast<float*>(w + L.A32);
    P->A16 = reinterpret_cast<__nv_bfloat16*>(w + L.A16);
    P->A8 = reinterpret_cast<uint8_t*>(w + L.A8);
    P->sa = reinterpret_cast<float*>(w + L.sa);
    P->ea = reinterpret_cast<float*>(w + L.ea);
    P->Y32 = reinterpret_cast<float*>(w + L.Y32);
    P->R32 = reinterpret_cast<float*>(w + L.R32);
    P->R16 = reinterpret_cast<__nv_bfloat16*>(w + L.R16);
    P->R8 = reinterpret_cast<uint8_t*>(w + L.R8);
    P->sr = reinterpret_cast<float*>(w + L.sr);
    P->er = reinterpret_cast<float*>(w + L.er);
    P->mask = reinterpret_cast<uint32_t*>(w + L.mask);
    P->cand_val = reinterpret_cast<float*>(w + L.cval);
    P->cand_idx = reinterpret_cast<int*>(w + L.cidx);
    P->cand_bound = reinterpret_cast<float*>(w + L.cbound);
    P->gcol = reinterpret_cast<float*>(w + L.gcol);
    P->dnorm = reinterpret_cast<float*>(w + L.dnorm);
    P->bt = reinterpret_cast<float*>(w + L.bt);
    P->L = reinterpret_cast<double*>(w + L.L);
    P->z = reinterpret_cast<double*>(w + L.z);
    P->x64 = reinterpret_cast<double*>(w + L.x64);
    P->G = L.G ? reinterpret_cast<float*>(w + L.G) : nullptr;
    P->bvec = L.bvec ? reinterpret_cast<float*>(w + L.bvec) : nullptr;
    P->am = L.am ? reinterpret_cast<float*>(w + L.am) : nullptr;
    P->av = L.av ? reinterpret_cast<float*>(w + L.av) : nullptr;
    P->tau = reinterpret_cast<int*>(w + L.tau);
    P->colnorm_max = reinterpret_cast<float*>(w + L.colnorm);
    P->counters = reinterpret_cast<unsigned*>(w + L.counters);
    P->GA = L.GA ? reinterpret_cast<float*>(w + L.GA) : nullptr;
}

cs_status ensure_tab(cs_plan* P, int len) {
    if (len <= P->tab_cap) return CS_OK;
    if (P->tab) {
        cudaError_t e = cudaFree(P->tab);
        P->tab = nullptr;
        P->tab_cap = 0;
        if (e != cudaSuccess) return cuda_fail(e, "cudaFree");
    }
    int cap = std::max(len, 2048);
    cudaError_t e = cudaMalloc(&P->tab, sizeof(float2) * (size_t)cap);
    if (e != cudaSuccess) return fail(CS_ENOMEM, "cudaMalloc(adam table): %s", cudaGetErrorString(e));
    P->tab_cap = cap;
    return CS_OK;
}

// Scratch of the total-variation prior: the differenced basis (n x Ep floats,
// grown when a longer signal needs it) and its n_max x n_max Gram matrix.
cs_status ensure_tv(cs_plan* P, size_t e_floats) {
    if (!P->tvT) {
        cudaError_t e = cudaMalloc(&P->tvT, sizeof(float) * (size_t)P->n_max * (size_t)P->n_max);
        if (e != cudaSuccess) {
            P->tvT = nullptr;
            return fail(CS_ENOMEM, "cudaMalloc(TV Gram matrix): %s", cudaGetErrorString(e));
        }
    }
    if (e_floats > P->tvE_cap) {
        if (P->tvE) {
            cudaError_t e = cudaFree(P->tvE);
            P->tvE = nullptr;
            P->tvE_cap = 0;
            if (e != cudaSuccess) return cuda_fail(e, "cudaFree");
        }
        cudaError_t e = cudaMalloc(&P->tvE, sizeof(float) * e_floats);
        if (e != cudaSuccess) {
            P->tvE = nullptr;
            return fail(CS_ENOMEM, "cudaMalloc(TV differences): %s", cudaGetErrorString(e));
        }
        P->tvE_cap = e_floats;
    }
    return CS_OK;
}

// Multiprocessors of the current device (cached per device).
int device_sm_count() {
    static std::mutex mu;
    static std::map<int, int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    cache[dev] = n;
    return n;
}

// The dense correlation buffer of the threshold rule, sized for the plan once.
cs_status ensure_cbuf(cs_plan* P) {
    if (P->cbuf) return CS_OK;
    cudaError_t e = cudaMalloc(&P->cbuf, sizeof(float) * (size_t)P->B_max * (size_t)P->n_max);
    if (e != cudaSuccess) {
        P->cbuf = nullptr;
        return fail(CS_ENOMEM, "cudaMalloc(correlation buffer): %s", cudaGetErrorString(e));
    }
    return CS_OK;
}

cs_status validate(const cs_plan* P, const float* A, int m, int n, int lda, const float* Y,
                   int ldy, int B, const int32_t* support, const float* coef, const int32_t* n_iter,
                   const float* res_norm, const int32_t* sig_status, const cs_omp_params* op) {
    if (!P) return fail(CS_EINVAL, "plan is NULL");
    if (!op) return fail(CS_EINVAL, "params is NULL");
    if (m < 1 || n < 1) return fail(CS_EINVAL, "m=%d, n=%d must be >= 1", m, n);
    if (B < 0) return fail(CS_EINVAL, "batch=%d must be >= 0", B);
    if (lda < m) return fail(CS_EINVAL, "lda=%d < m=%d", lda, m);
    if (ldy < m) return fail(CS_EINVAL, "ldy=%d < m=%d", ldy, m);
    if (op->k < 1 || op->k > m || op->k > n)
        return fail(CS_EINVAL, "k=%d must satisfy 1 <= k <= min(m=%d, n=%d)", op->k, m, n);
    if (!(op->tol >= 0.0)) return fail(CS_EINVAL, "tol must be >= 0");
    if (op->prec != CS_CORR_FP32 && op->prec != CS_CORR_BF16 && op->prec != CS_CORR_FP8)
        return fail(CS_EINVAL, "prec=%d is not a cs_corr_prec", op->prec);
    if (op->topc < 0 || op->topc > kTopcMax) return fail(CS_EINVAL, "topc=%d not in [0, 8]", op->topc);
    if (m > P->m_max || n > P->n_max || B > P->B_max)
        return fail(CS_EINVAL, "problem m=%d n=%d batch=%d exceeds the plan (%d, %d, %d)", m, n, B,
                    P->m_max, P->n_max, P->B_max);
    if (op->k > P->k_user) return fail(CS_ENOTSUP, "k=%d exceeds the plan k_max=%d", op->k, P->k_user);
    if (B > 0 && (!A || !Y || !support || !coef || !n_iter || !res_norm || !sig_status))
        return fail(CS_EINVAL, "a required array pointer is NULL");
    return CS_OK;
}

// Instances the on-chip batched kernels do not take: more rows than a warp
// holds, a support beyond the plan's on-chip K, or the bf16 correlation
// outside the tensor-core kernel's sizes.  OMP and Gram-form CLOMP run them
// on the large-instance path.
bool needs_large(const cs_plan* P, int m, int n, int k, int prec) {
    return m > kMaxRowChunks * 128 || k > P->k_max || (prec == CS_CORR_BF16 && !corr_tc_supported(m, n));
}

cs_status ensure_lg(char** buf, size_t* have, size_t bytes) {
    if (bytes <= *have) return CS_OK;
    if (*buf) {
        cudaError_t e = cudaFree(*buf);
        *buf = nullptr;
        *have = 0;
        if (e != cudaSuccess) return cuda_fail(e, "cudaFree");
    }
    cudaError_t e = cudaMalloc(buf, bytes);
    if (e != cudaSuccess) {
        *buf = nullptr;
        return fail(CS_ENOMEM, "cudaMalloc(large-instance workspace, %zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    *have = bytes;
    return CS_OK;
}

cudaEvent_t pool_event(cs_plan* P);

// Key of an autotuned size class.
std::string size_key(const char* kind, int prec, int m, int n, int B) {
    char buf[96];
    snprintf(buf, sizeof(buf), "%s prec=%d m=%d n=%d B=%d", kind, prec, m, n, B);
    return buf;
}

// Measurement hook of the large-instance path: every group of launches of
// one phase is counted and, when profiling, bracketed by CUDA events.
struct LargeMarkCtx {
    cs_plan* P;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
};
void large_mark(void* vctx, int phase, int after) {
    LargeMarkCtx* c = static_cast<LargeMarkCtx*>(vctx);
    cs_plan* P = c->P;
    if (!after) {
        P->launches[phase] += 1;
        if (P->profiling) {
            c->a = pool_event(P);
            if (c->a) cudaEventRecord(c->a, c->s);
        }
        return;
    }
    if (P->profiling && c->a) {
        cudaEvent_t b = pool_event(P);
        if (b) {
            cudaEventRecord(b, c->s);
            P->marks.push_back({phase, c->a, b});
        } else {
            P->pool.push_back(c->a);
        }
        c->a = nullptr;
    }
}

// OMP or Gram-form CLOMP of signals sharing A on the large-instance path, in
// chunks whose workspace stays within a few GB.
constexpr size_t kLargeChunkBytes = (size_t)8 << 30;
// Large OMP groups of an uneven batch run at once, at most this many.
constexpr int kVarlenWorkers = 4;

// CLOMP configurations the large-instance path runs: the Gram form, one atom
// per iteration, no prior.
bool large_clomp_ok(const cs_clomp_params* cp) {
    const bool th = cp->select_threshold > 0.f && cp->select_threshold < 1.f;
    return cp->form == CS_CL_GRAM && !th && cp->tv_weight == 0.f && cp->lv_weight == 0.f;
}

template <class F>
cudaError_t timed(cs_plan* P, int phase, cudaStream_t s, F&& launch);

// The large-instance solve on stream s with the workspace *ws (grown as
// needed).  marks: count and time the phases in the plan (one thread at a
// time only); tune_mu (non-null: the solve runs beside others on the device)
// guards the plan's tuned configurations, and then CLOMP finds its Adam
// table already made and runs no cooperative launch.
cs_status solve_large_on(cs_plan* P, const float* A, int m, int n, int lda, const std::vector<const float*>& ys,
                         const std::vector<LargeOut>& outs, const cs_omp_params* op, const cs_clomp_params* cp,
                         cudaStream_t s, char** ws, size_t* ws_bytes, bool marks, std::mutex* tune_mu) {
    if (P->no_large) return fail(CS_ENOTSUP, "this entry point runs only the on-chip kernels (m <= 1024, k <= 64, "
                                             "bf16: m <= 256, n <= 4096)");
    if (cp && !large_clomp_ok(cp))
        return fail(CS_ENOTSUP, "CLOMP beyond the on-chip sizes runs the Gram form with one atom per iteration "
                                "and no prior");
    const size_t count = ys.size();
    int kmax = 1;
    for (const LargeOut& o : outs) kmax = std::max(kmax, o.k);
    if (!large_supported(m, n, kmax))
        return fail(CS_ENOTSUP, "the large-instance path supports m <= %d and k <= %d (m=%d k=%d)", kLargeMaxM, kLargeMaxK, m, kmax);
    const int bf16 = op->prec == CS_CORR_BF16 ? 1 : 0;
    const int clf = cp ? 1 : 0;
    ClArgs cl{};
    if (cp) {
        // Adam factors for every step of the longest signal (one state for the solve)
        const int iters = op->max_iter > 0 ? std::min(kmax, op->max_iter) : kmax;
        const int len = (cp->reset_adam_each_iter ? 1 : iters) * std::max(cp->steps, 1);
        if (!tune_mu) {
            cs_status st = ensure_tab(P, len);
            if (st != CS_OK) return st;
            CS_TRY_LAUNCH(timed(P, CS_PHASE_SETUP, s, [&] {
                              return launch_adam_table(P->tab, len, cp->lr, cp->beta1, cp->beta2, s);
                          }), "adam table");
        } else if (len > P->tab_cap) {
            return fail(CS_EINVAL, "internal: the Adam table was not made for this group");
        }
        cl.steps = cp->steps;
        cl.beta1 = cp->beta1;
        cl.beta2 = cp->beta2;
        cl.eps = cp->eps;
        cl.reset = cp->reset_adam_each_iter ? 1 : 0;
        cl.tab = P->tab;
        cl.tab_len = len;
    }
    // signals per chunk: the fixed part (bf16 A) plus as many signals as fit the budget
    const size_t one = large_ws_bytes(m, n, 1, kmax, bf16, clf), two = large_ws_bytes(m, n, 2, kmax, bf16, clf);
    const size_t per = two > one ? two - one : one;
    size_t cap = one >= kLargeChunkBytes ? 1 : 1 + (kLargeChunkBytes - one) / per;
    cap = std::min(cap, (size_t)std::max(P->B_max, 1));
    DeviceGuard dg(P->device);
    if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
    int live = 0;
    for (size_t b0 = 0; b0 < count; b0 += cap) {
        const size_t nb = std::min(cap, count - b0);
        LargeCall call;
        call.A = A;
        call.m = m;
        call.n = n;
        call.lda = lda;
        call.ys.assign(ys.begin() + b0, ys.begin() + b0 + nb);
        call.outs.assign(outs.begin() + b0, outs.begin() + b0 + nb);
        call.ks.resize(nb);
        for (size_t b = 0; b < nb; ++b) call.ks[b] = call.outs[b].k;
        call.max_iter = op->max_iter;
        call.tol = op->tol;
        call.bf16 = bf16;
        call.live_host = &live;
        LargeMarkCtx mc{P, s};
        call.mark = marks ? large_mark : nullptr;
        call.mark_ctx = &mc;
        // the correlation's configuration for this size class (tuned once)
        const std::string key = size_key("large correlation", op->prec, m, n, (int)nb);
        int chosen = -1;
        bool known;
        {
            std::unique_lock<std::mutex> lk;
            if (tune_mu) lk = std::unique_lock<std::mutex>(*tune_mu);
            auto tk = P->tuned.find(key);
            known = tk != P->tuned.end();
            call.corr_cfg = known ? tk->second : -1;
        }
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        call.tune = P->autotune && cudaStreamIsCapturing(s, &cap) == cudaSuccess && cap == cudaStreamCaptureStatusNone;
        call.chosen_cfg = &chosen;
        const size_t need = large_ws_bytes(m, n, (int)nb, kmax, bf16, clf);
        call.cl = cp ? &cl : nullptr;
        call.no_coop = tune_mu ? 1 : 0;
        call.errflag = P->counters + 1;
        cs_status st = ensure_lg(ws, ws_bytes, need);
        if (st != CS_OK) return st;
        cudaError_t e = large_solve(call, *ws, *ws_bytes, s);
        if (e != cudaSuccess) return cuda_fail(e, "large-instance solve");
        if (call.tune && !known && chosen >= 0) {
            std::unique_lock<std::mutex> lk;
            if (tune_mu) lk = std::unique_lock<std::mutex>(*tune_mu);
            P->tuned[key] = chosen;
        }
    }
    return CS_OK;
}

cs_status solve_large(cs_plan* P, const float* A, int m, int n, int lda, const std::vector<const float*>& ys,
                      const std::vector<LargeOut>& outs, const cs_omp_params* op, const cs_clomp_params* cp,
                      cudaStream_t s) {
    return solve_large_on(P, A, m, n, lda, ys, outs, op, cp, s, &P->lg, &P->lg_bytes, true, nullptr);
}

IterArgs make_args(cs_plan* P, int m, int n, int B, const cs_omp_params* op, int32_t* support,
                   float* coef, int32_t* n_iter, float* res_norm, int32_t* sig_status) {
    IterArgs a{};
    a.m = m;
    a.n = n;
    a.B = B;
    a.k = op->k;
    a.kmax = P->k_max;
    a.iters = (op->max_iter > 0) ? std::min(op->k, op->max_iter) : op->k;
    a.mp = round_up(m, 4);
    a.mh = round_up(m, 64);   // bf16 rows: whole 128-byte swizzle rows for TMA
    a.mq = round_up(m, 128);  // fp8 rows: the same
    a.nw = ceil_div(n, 32);
    a.prec = op->prec;
    if (op->prec == CS_CORR_FP32) {
        a.nch = ceil_div(n, kCorrFp32TileN);
        a.topc = 1;
    } else {
        a.tc_tile = kCorrTcTileN;
        a.nch = ceil_div(n, kCorrTcTileN);
        a.topc = kTcCandPerTile;
    }
    a.tol = op->tol;
    a.A32 = P->A32;
    a.A16 = P->A16;
    a.Y32 = P->Y32;
    a.R32 = P->R32;
    a.R16 = (op->prec == CS_CORR_BF16) ? P->R16 : nullptr;
    const bool fp8 = op->prec == CS_CORR_FP8;
    a.R8 = fp8 ? P->R8 : nullptr;
    a.A8 = P->A8;
    a.sa = P->sa;
    a.ea_max = P->ea;
    a.sr = P->sr;
    a.er = P->er;
    a.mask = P->mask;
    a.cand_val = P->cand_val;
    a.cand_idx = P->cand_idx;
    a.cand_bound = P->cand_bound;
    a.gcol = P->gcol;
    a.dnorm = P->dnorm;
    a.bt = P->bt;
    a.L = P->L;
    a.z = P->z;
    a.x64 = P->x64;
    a.G = P->G;
    a.bvec = P->bvec;
    a.am = P->am;
    a.av = P->av;
    a.tau = P->tau;
    a.colnorm_max = P->colnorm_max;
    a.GA = (P->GA && n <= kGramAMax) ? P->GA : nullptr;
    a.counters = P->counters;
    a.support = support;
    a.coef = coef;
    a.n_iter = n_iter;
    a.res_norm = res_norm;
    a.status = sig_status;
    return a;
}


cudaEvent_t pool_event(cs_plan* P) {
    if (!P->pool.empty()) {
        cudaEvent_t e = P->pool.back();
        P->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Run one launch of `phase`, counting it and (when profiling) timing it.
template <class F>
cudaError_t timed(cs_plan* P, int phase, cudaStream_t s, F&& launch) {
    P->launches[phase] += 1;
    if (!P->profiling) return launch();
    cudaEvent_t a = pool_event(P), b = pool_event(P);
    if (!(a && b)) {            // no pair: untimed (the one event made goes back)
        if (a) P->pool.push_back(a);
        if (b) P->pool.push_back(b);
        a = b = nullptr;
    }
    if (a && b) cudaEventRecord(a, s);
    cudaError_t e = launch();
    if (a && b) {
        cudaEventRecord(b, s);
        P->marks.push_back({phase, a, b});
    }
    return e;
}

// Autotuner: on the first solve of a size class (outside stream capture),
// launch each of `ncand` configurations of one kernel on the solve's own data
// (once to warm up, then three times between CUDA events), keep the fastest
// in the plan and return it; later solves of the class reuse the choice.
// The tuned kernels are idempotent -- a repeated launch rewrites the same
// outputs -- and every configuration computes the same bits, so tuning
// changes timing only.  Returns `fallback` when tuning is off or the stream
// is being captured.
template <class L>
int autotune(cs_plan* P, const std::string& key, int ncand, L&& launch, cudaStream_t s, int fallback) {
    auto it = P->tuned.find(key);
    if (it != P->tuned.end()) return it->second;
    if (!P->autotune || ncand <= 1) return fallback;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return fallback;
    cudaEvent_t e0 = pool_event(P), e1 = pool_event(P);
    if (!e0 || !e1) {
        if (e0) P->pool.push_back(e0);
        if (e1) P->pool.push_back(e1);
        return fallback;
    }
    int best = -1;
    float best_ms = 0.f;
    for (int c = 0; c < ncand; ++c) {
        if (launch(c) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        cudaEventRecord(e0, s);
        for (int r = 0; r < 3; ++r) launch(c);
        cudaEventRecord(e1, s);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) continue;
        if (best < 0 || ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    if (best < 0) best = fallback;
    P->pool.push_back(e0);
    P->pool.push_back(e1);
    P->tuned[key] = best;
    return best;
}

template <class E, class K>
cs_status run_solve(cs_plan* P, cudaStream_t s, E& enqueue, K&& make_key, bool graphs);

// The solve: set-up, then per iteration correlation -> select -> fit -> residual.
cs_status solve(cs_plan* P, const float* A, int m, int n, int lda, const float* Y, int ldy, int B,
                int32_t* support, float* coef, int32_t* n_iter, float* res_norm,
                int32_t* sig_status, const cs_omp_params* op, const cs_clomp_params* cp,
                cudaStream_t s) {
    cs_status st = validate(P, A, m, n, lda, Y, ldy, B, support, coef, n_iter, res_norm,
                            sig_status, op);
    if (st != CS_OK) return st;
    if (cp) {
        if (cp->steps < 0) return fail(CS_EINVAL, "steps=%d must be >= 0", cp->steps);
        if (cp->form != CS_CL_GATHER && cp->form != CS_CL_GRAM)
            return fail(CS_EINVAL, "form=%d is not a cs_cl_form", cp->form);
        if (!(cp->beta1 >= 0.f && cp->beta1 < 1.f && cp->beta2 >= 0.f && cp->beta2 < 1.f))
            return fail(CS_EINVAL, "Adam betas must lie in [0, 1)");
        if (!(cp->eps >= 0.f) || !std::isfinite(cp->lr)) return fail(CS_EINVAL, "bad lr/eps");
        if (!(cp->select_threshold >= 0.f) || !std::isfinite(cp->select_threshold))
            return fail(CS_EINVAL, "select_threshold must be finite and >= 0");
        if (!(cp->tv_weight >= 0.f) || !std::isfinite(cp->tv_weight))
            return fail(CS_EINVAL, "tv_weight must be finite and >= 0");
        if (cp->tv_weight > 0.f && cp->tv_D && (cp->tv_N < 2 || cp->tv_ldd < cp->tv_N))
            return fail(CS_EINVAL, "tv_D needs tv_N >= 2 and tv_ldd >= tv_N (tv_N=%d tv_ldd=%d)", cp->tv_N,
                        cp->tv_ldd);
        if (cp->image_width < 0) return fail(CS_EINVAL, "image_width=%d must be >= 0", cp->image_width);
        if (!(cp->lv_weight >= 0.f) || !std::isfinite(cp->lv_weight))
            return fail(CS_EINVAL, "lv_weight must be finite and >= 0");
        if (!(cp->lv_eps >= 0.f) || !std::isfinite(cp->lv_eps))
            return fail(CS_EINVAL, "lv_eps must be finite and >= 0");
        if (cp->lv_weight > 0.f && cp->tv_D && (cp->tv_N < 1 || cp->tv_ldd < cp->tv_N))
            return fail(CS_EINVAL, "tv_D needs tv_ldd >= tv_N >= 1 (tv_N=%d tv_ldd=%d)", cp->tv_N, cp->tv_ldd);
    }
    if (B == 0) return CS_OK;
    if (op->prec == CS_CORR_FP8 && (!corr_tc_supported(m, n) || op->k > P->k_max))
        return fail(CS_ENOTSUP, "the FP8 correlation runs with m <= 256, n <= %d and k <= %d (m=%d n=%d k=%d)",
                    kCorrTcMaxN, P->k_max, m, n, op->k);
    if (needs_large(P, m, n, op->k, op->prec)) {
        std::vector<const float*> ys(B);
        std::vector<LargeOut> outs(B);
        for (int b = 0; b < B; ++b) {
            const size_t o = (size_t)b * op->k;
            ys[b] = Y + (size_t)b * ldy;
            outs[b] = LargeOut{support + o, coef + o, n_iter + b, res_norm + b, sig_status + b, op->k};
        }
        return solve_large(P, A, m, n, lda, ys, outs, op, cp, s);
    }
    DeviceGuard dg(P->device);
    if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");

    IterArgs a = make_args(P, m, n, B, op, support, coef, n_iter, res_norm, sig_status);
    const bool bf16 = (op->prec == CS_CORR_BF16);
    const bool fp8 = (op->prec == CS_CORR_FP8);
    const bool lowp = bf16 || fp8;   // tensor-core correlation, certified candidates
    a.need_gcol = cp ? 0 : 1;
    a.need_gram = (cp && cp->form == CS_CL_GRAM) ? 1 : 0;

    ClArgs c{};
    if (cp) {
        const int len = (cp->reset_adam_each_iter ? 1 : a.iters) * std::max(cp->steps, 1);
        st = ensure_tab(P, len);
        if (st != CS_OK) return st;
        c.steps = cp->steps;
        c.beta1 = cp->beta1;
        c.beta2 = cp->beta2;
        c.eps = cp->eps;
        c.reset = cp->reset_adam_each_iter ? 1 : 0;
        c.tab = P->tab;
        c.tab_len = len;
        c.th = (cp->select_threshold > 0.f && cp->select_threshold < 1.f) ? cp->select_threshold : 0.f;
    }

    // total-variation prior: added once to A^T A, from which the fit's Gram
    // matrices are gathered
    const bool tv = cp && cp->tv_weight > 0.f;
    int tvN = 0, tvEp = 0;
    if (tv) {
        if (cp->form != CS_CL_GRAM || !a.GA)
            return fail(CS_ENOTSUP, "the TV prior needs the Gram form and n <= %d", kGramAMax);
        tvN = cp->tv_D ? cp->tv_N : n;
        if (tvN < 2) return fail(CS_EINVAL, "the TV prior needs a signal of length >= 2");
        tvEp = round_up(tvN - 1, 4);
        st = ensure_tv(P, (size_t)n * tvEp);
        if (st != CS_OK) return st;
    }
    // the image priors (Eq. 6 and 7): images of imgW consecutive columns
    const bool lv = cp && cp->lv_weight > 0.f;
    const int imgW = (tv || lv) ? cp->image_width : 0;
    const bool img = imgW >= 2;
    const int imgH = cp && cp->tv_D ? cp->tv_N : n;     // pixels per column
    float lv_scale = 0.f;
    if (lv) {
        if (!img) return fail(CS_EINVAL, "lv_weight needs image_width >= 2 (image_width=%d)", cp->image_width);
        if (cp->form != CS_CL_GRAM || !a.GA)
            return fail(CS_ENOTSUP, "the LV prior needs the Gram form and n <= %d", kGramAMax);
        if (imgH >= 3 && imgW >= 3) lv_scale = cp->lv_weight / ((float)(imgH - 2) * (float)(imgW - 2));
    }
    if (img) {
        if (c.th > 0.f || !clfit_image_supported(a, imgW, lv_scale != 0.f, imgH))
            return fail(CS_ENOTSUP, "the image priors (image_width=%d) need one atom per iteration, k <= 32, "
                                    "2 <= image_width <= 512, a batch of whole images (batch=%d) and, with "
                                    "lv_weight, at most 256 pixels per column", imgW, B);
        const int shape = imgW * 2 + (lv_scale != 0.f ? 1 : 0);
        if (P->img_ready != shape || P->img_ready_h != imgH) {
            int ok = 0;
            const cudaError_t e = clfit_image_prepare(imgW, lv_scale != 0.f, imgH, &ok);
            if (e != cudaSuccess) return cuda_fail(e, "image prior: cluster check");
            if (!ok) return fail(CS_ENOTSUP, "image prior: clusters for image_width=%d do not fit this device", imgW);
            P->img_ready = shape;
            P->img_ready_h = imgH;
        }
    }

    // A prepared by an earlier solve of this plan (same A, generation != 0)
    const bool need_gram = a.GA && (a.need_gcol || a.need_gram);
    const cs_plan::Prep& pr = P->prep;
    const void* a_key = P->a_host ? P->a_host : (const void*)A;
    const bool reuse_a = P->a_gen != 0 && pr.gen == P->a_gen && pr.A == a_key && pr.m == m && pr.n == n &&
                         pr.lda == lda && (pr.bf16 || !bf16) && (pr.fp8 || !fp8) && (pr.gram || !need_gram) && !tv;

    // plain OMP on small batches: the whole solve in one kernel, one CTA per signal
    const bool omp_fused = !cp && P->fused_omp && a.B <= device_sm_count() && omp_fused_supported(a);
    // ... and A resident in the kernel's shared memory: it reads the caller's
    // A and Y and does the set-up itself (the only launch of the solve)
    const bool omp_self = omp_fused && omp_fused_self_contained(a);

    // CLOMP in Gram form runs selection, fit and residual as one kernel, or
    // (bf16 correlation) the whole solve as one persistent kernel
    const bool fused = cp && cp->form == CS_CL_GRAM && P->fuse_update && !img && update_clomp_fused_supported(a);
    const bool persist = cp && cp->form == CS_CL_GRAM && bf16 && P->persist && !img &&
                         clomp_persist_supported(a, c);
    // threshold rule: float32 correlation of every atom, then one fused
    // selection + fit + residual kernel per iteration
    const bool th_rule = cp && c.th > 0.f;
    if (th_rule) {
        if (cp->form != CS_CL_GRAM || lowp || !clomp_th_supported(a))
            return fail(CS_ENOTSUP, "select_threshold in (0, 1) runs with the float32 correlation "
                                    "(CS_CORR_FP32), the Gram-form fit, m <= 1024 and k <= 32");
        st = ensure_cbuf(P);
        if (st != CS_OK) return st;
    }

    // Every launch of the solve, on stream `st`.
    auto enqueue = [&](cudaStream_t st) -> cs_status {
        if (omp_self) {
            CS_TRY_LAUNCH(timed(P, CS_PHASE_PERSIST, st, [&] { return launch_omp_fused(a, A, lda, Y, ldy, st); }),
                          "fused OMP");
            return CS_OK;
        }
        if (cp)
            CS_TRY_LAUNCH(timed(P, CS_PHASE_SETUP, st, [&] {
                              return launch_adam_table(P->tab, c.tab_len, cp->lr, cp->beta1, cp->beta2, st);
                          }), "adam table");
        if (!reuse_a) {
            CS_TRY_LAUNCH(timed(P, CS_PHASE_SETUP, st, [&] {
                              return launch_prep_A(A, lda, m, n, a.mp, a.mh, P->A32, bf16 ? P->A16 : nullptr,
                                                   P->colnorm_max, st);
                          }), "prep A");
            if (fp8) {
                CS_TRY_LAUNCH(cudaMemsetAsync(P->ea, 0, sizeof(float), st), "clear FP8 error norm");
                CS_TRY_LAUNCH(timed(P, CS_PHASE_SETUP, st, [&] {
                                  return launch_prep_A8(A, lda, m, n, a.mq, P->A8, P->sa, P->ea, st);
                              }), "prep A (FP8)");
            }
            if (need_gram)
                CS_TRY_LAUNCH(timed(P, CS_PHASE_SETUP, st, [&] { return launch_gram_A(P->A32, a.mp, n, P->GA, st); }),
                              "gram of A");
        }
        if (tv)
            CS_TRY_LAUNCH(timed(P, CS_PHASE_SETUP, st, [&] {
                              return launch_tv_prior(cp->tv_D, tvN, cp->tv_ldd, n, 2.f * cp->tv_weight / (float)tvN,
                                                     P->tvE, tvEp, P->tvT, P->GA, st);
                          }), "TV prior");
        CS_TRY_LAUNCH(timed(P, CS_PHASE_SETUP, st, [&] { return launch_setup(a, Y, ldy, cp ? 1 : 0, st); }), "setup");
        if (th_rule) {
            for (int it = 0; it < a.iters; ++it) {
                c.tau0 = c.reset ? 0 : it * c.steps;
                CS_TRY_LAUNCH(timed(P, CS_PHASE_CORR, st, [&] { return launch_corr_fp32_dense_live(a, P->cbuf, n, st); }),
                              "correlation (fp32, dense)");
                CS_TRY_LAUNCH(timed(P, CS_PHASE_UPDATE, st, [&] { return launch_clomp_th(a, c, P->cbuf, n, it, st); }),
                              "threshold-rule update");
            }
            return CS_OK;
        }
        if (persist) {
            const int stall = P->stall_test;
            P->stall_test = 0;
            CS_TRY_LAUNCH(timed(P, CS_PHASE_PERSIST, st, [&] { return launch_clomp_persist(a, c, stall, st); }),
                          "persistent solve");
            return CS_OK;
        }
        if (omp_fused) {
            CS_TRY_LAUNCH(timed(P, CS_PHASE_PERSIST, st, [&] { return launch_omp_fused(a, nullptr, 0, nullptr, 0, st); }),
                          "fused OMP");
            return CS_OK;
        }
        if (lowp) {
            // tensor-core tile width: forced, tuned for this size class, or 256
            static const int widths[2] = {256, 128};
            int tile = 256;
            if (P->force_tile == 128 || P->force_tile == 256) {
                tile = P->force_tile;
            } else {
                const int ci = autotune(P, size_key("tc-correlation tile", op->prec, m, n, B), 2,
                                        [&](int cand) {
                                            IterArgs t = a;
                                            t.tc_tile = widths[cand];
                                            t.nch = ceil_div(n, widths[cand]);
                                            t.topc = 2 * widths[cand] / kTcGroup;
                                            return launch_corr_tc(t, st);
                                        }, st, 0);
                tile = widths[ci];
            }
            a.tc_tile = tile;
            a.nch = ceil_div(n, tile);
            a.topc = 2 * tile / kTcGroup;
        }
        for (int it = 0; it < a.iters; ++it) {
            c.tau0 = c.reset ? 0 : it * c.steps;
            if (lowp)
                CS_TRY_LAUNCH(timed(P, CS_PHASE_CORR, st, [&] { return launch_corr_tc(a, st); }), "correlation (tcgen05)");
            else
                CS_TRY_LAUNCH(timed(P, CS_PHASE_CORR, st, [&] { return launch_corr_fp32(a, st); }), "correlation (fp32)");
            if (fused) {
                CS_TRY_LAUNCH(timed(P, CS_PHASE_UPDATE, st, [&] { return launch_update_clomp(a, c, it, st); }),
                              "fused update");
                continue;
            }
            CS_TRY_LAUNCH(timed(P, CS_PHASE_SELECT, st, [&] { return launch_select(a, st); }), "select");
            if (!cp)
                CS_TRY_LAUNCH(timed(P, CS_PHASE_FIT, st, [&] { return launch_chol(a, st); }), "cholesky");
            else if (img)
                CS_TRY_LAUNCH(timed(P, CS_PHASE_FIT, st, [&] {
                                  return launch_clfit_image(a, c, it, imgW, tv ? 2.f * cp->tv_weight / (float)imgW : 0.f,
                                                            lv_scale, cp->lv_eps, cp->tv_D, imgH,
                                                            cp->tv_D ? cp->tv_ldd : imgH, st);
                              }), "cl fit (image priors)");
            else if (cp->form == CS_CL_GRAM)
                CS_TRY_LAUNCH(timed(P, CS_PHASE_FIT, st, [&] { return launch_clfit_gram(a, c, it, st); }), "cl fit (gram)");
            else
                CS_TRY_LAUNCH(timed(P, CS_PHASE_FIT, st, [&] { return launch_clfit_gather(a, c, it, st); }),
                              "cl fit (gather)");
            CS_TRY_LAUNCH(timed(P, CS_PHASE_RESID, st, [&] { return launch_resid(a, st); }), "residual");
        }
        return CS_OK;
    };
    // Eagerly or as a replayed CUDA graph; on any failure nothing counts as prepared.
    if (!reuse_a) {
        // what this solve leaves prepared (the TV prior changes A^T A in place)
        cs_plan::Prep np;
        np.A = a_key;
        np.m = m;
        np.n = n;
        np.lda = lda;
        np.gen = P->a_gen;
        np.bf16 = bf16 ? 1 : 0;
        np.fp8 = fp8 ? 1 : 0;
        np.gram = (need_gram && !tv) ? 1 : 0;
        if (omp_self) np.gen = 0;     // the self-contained solve prepares nothing
        P->prep = np;
    }
    const cs_status rs = run_solve(P, s, enqueue, [&](std::string& key) {
        auto put = [&](const void* v, size_t nb) { key.append(static_cast<const char*>(v), nb); };
        const void* ptrs[] = {A, Y, support, coef, n_iter, res_norm, sig_status, P->tab, P->cbuf,
                              (tv || lv) ? (const void*)cp->tv_D : nullptr, P->tvE, P->tvT};
        put(ptrs, sizeof(ptrs));
        const int ints[] = {m, n, lda, ldy, B, c.tab_len, fused ? 1 : 0, persist ? 1 : 0, omp_fused ? 1 : 0,
                            reuse_a ? 1 : 0};
        put(ints, sizeof(ints));
        // field by field (struct padding is not part of the key)
        const double dk[] = {(double)op->k, op->tol, (double)op->max_iter, (double)op->prec,
                             cp ? (double)cp->steps : -1.0, cp ? (double)cp->lr : 0.0,
                             cp ? (double)cp->beta1 : 0.0, cp ? (double)cp->beta2 : 0.0,
                             cp ? (double)cp->eps : 0.0, cp ? (double)cp->reset_adam_each_iter : 0.0,
                             cp ? (double)cp->form : -1.0, cp ? (double)c.th : 0.0,
                             tv ? (double)cp->tv_weight : 0.0, (double)tvN, tv ? (double)cp->tv_ldd : 0.0,
                             (double)imgW, lv ? (double)cp->lv_weight : 0.0, lv ? (double)cp->lv_eps : 0.0,
                             (double)imgH,
                             cp && cp->tv_D ? (double)cp->tv_ldd : 0.0};
        put(dk, sizeof(dk));
    }, P->use_graphs && !P->profiling && !(persist && P->stall_test));
    if (rs != CS_OK) P->prep = cs_plan::Prep{};
    return rs;
}

// Runs a solve's launches eagerly (graphs off, or the first call with a key),
// or captures them into a CUDA graph on the second identical call and replays
// that graph from then on.
template <class E, class K>
cs_status run_solve(cs_plan* P, cudaStream_t s, E& enqueue, K&& make_key, bool graphs) {
    if (!graphs) return enqueue(s);

    // graph cache key: everything the launches bake in
    std::string key;
    make_key(key);
    if (P->graphs.size() > 16 && !P->graphs.count(key)) {
        for (auto& kv : P->graphs)
            if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        P->graphs.clear();
    }
    cs_plan::GraphEntry& ge = P->graphs[key];
    if (!ge.exec && ge.seen++ == 0) return enqueue(s);     // first call: eager
    if (!ge.exec) {
        // second identical call: capture on the private stream
        if (!P->cap_stream) {
            cudaError_t e = cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
        }
        int64_t before[CS_PHASES];
        for (int i = 0; i < CS_PHASES; ++i) before[i] = P->launches[i];
        cudaError_t e = cudaStreamBeginCapture(P->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
        const cs_status st_cap = enqueue(P->cap_stream);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(P->cap_stream, &g);
        for (int i = 0; i < CS_PHASES; ++i) {
            ge.launches[i] = P->launches[i] - before[i];
            P->launches[i] = before[i];
        }
        if (st_cap != CS_OK || e != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            P->graphs.erase(key);
            P->use_graphs = 0;              // capture unavailable here: stay eager
            cudaGetLastError();
            return enqueue(s);
        }
        e = cudaGraphInstantiate(&ge.exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            ge.exec = nullptr;
            P->graphs.erase(key);
            P->use_graphs = 0;
            cudaGetLastError();
            return enqueue(s);
        }
    }
    for (int i = 0; i < CS_PHASES; ++i) P->launches[i] += ge.launches[i];
    CS_TRY_LAUNCH(cudaGraphLaunch(ge.exec, s), "cudaGraphLaunch");
    return CS_OK;
}

// Copy the four device counters at `dev` to out (after the stream's work),
// optionally zero them, and turn a set error flag into CS_ETIMEOUT.
cs_status read_counters(unsigned* dev, uint32_t* out, int32_t reset, cudaStream_t s) {
    CS_TRY_LAUNCH(cudaMemcpyAsync(out, dev, 4 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s), "copy counters");
    if (reset) CS_TRY_LAUNCH(cudaMemsetAsync(dev, 0, 4 * sizeof(uint32_t), s), "reset counters");
    CS_TRY_LAUNCH(cudaStreamSynchronize(s), "stream synchronize");
    if (out[1] != 0) return fail(CS_ETIMEOUT, "a bounded device-side wait gave up (flags 0x%x)", out[1]);
    return CS_OK;
}

cs_status ensure_io(cs_plan* P, size_t bytes) {
    if (bytes <= P->io_bytes) return CS_OK;
    if (P->io) {
        cudaFree(P->io);
        P->io = nullptr;
        P->io_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&P->io, bytes);
    if (e != cudaSuccess) return fail(CS_ENOMEM, "cudaMalloc(io): %s", cudaGetErrorString(e));
    P->io_bytes = bytes;
    return CS_OK;
}

cs_status solve_host(cs_plan* P, const float* A, int m, int n, int lda, const float* Y, int ldy,
                     int B, int32_t* support, float* coef, int32_t* n_iter, float* res_norm,
                     int32_t* sig_status, const cs_omp_params* op, const cs_clomp_params* cp,
                     cudaStream_t s) {
    cs_status st = validate(P, A, m, n, lda, Y, ldy, B, support, coef, n_iter, res_norm,
                            sig_status, op);
    if (st != CS_OK) return st;
    if (B == 0) return CS_OK;
    DeviceGuard dg(P->device);
    if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
    const int k = op->k;
    Carver cv;
    const size_t oA = cv.take<float>((size_t)m * n);
    const size_t oY = cv.take<float>((size_t)m * B);
    const size_t oS = cv.take<int32_t>((size_t)k * B);
    const size_t oC = cv.take<float>((size_t)k * B);
    const size_t oN = cv.take<int32_t>(B);
    const size_t oR = cv.take<float>(B);
    const size_t oT = cv.take<int32_t>(B);
    st = ensure_io(P, cv.off);
    if (st != CS_OK) return st;
    float* dA = reinterpret_cast<float*>(P->io + oA);
    float* dY = reinterpret_cast<float*>(P->io + oY);
    int32_t* dS = reinterpret_cast<int32_t*>(P->io + oS);
    float* dC = reinterpret_cast<float*>(P->io + oC);
    int32_t* dN = reinterpret_cast<int32_t*>(P->io + oN);
    float* dR = reinterpret_cast<float*>(P->io + oR);
    int32_t* dT = reinterpret_cast<int32_t*>(P->io + oT);
    CS_TRY_LAUNCH(cudaMemcpy2DAsync(dA, sizeof(float) * m, A, sizeof(float) * lda, sizeof(float) * m, n,
                                    cudaMemcpyHostToDevice, s), "copy A");
    CS_TRY_LAUNCH(cudaMemcpy2DAsync(dY, sizeof(float) * m, Y, sizeof(float) * ldy, sizeof(float) * m, B,
                                    cudaMemcpyHostToDevice, s), "copy Y");
    P->a_host = A;
    st = solve(P, dA, m, n, m, dY, m, B, dS, dC, dN, dR, dT, op, cp, s);
    P->a_host = nullptr;
    if (st != CS_OK) {
        cudaStreamSynchronize(s);   // the copies of the caller's A and Y have finished on return
        return st;
    }
    CS_TRY_LAUNCH(cudaMemcpyAsync(support, dS, sizeof(int32_t) * k * B, cudaMemcpyDeviceToHost, s), "copy support");
    CS_TRY_LAUNCH(cudaMemcpyAsync(coef, dC, sizeof(float) * k * B, cudaMemcpyDeviceToHost, s), "copy coef");
    CS_TRY_LAUNCH(cudaMemcpyAsync(n_iter, dN, sizeof(int32_t) * B, cudaMemcpyDeviceToHost, s), "copy n_iter");
    CS_TRY_LAUNCH(cudaMemcpyAsync(res_norm, dR, sizeof(float) * B, cudaMemcpyDeviceToHost, s), "copy res_norm");
    CS_TRY_LAUNCH(cudaMemcpyAsync(sig_status, dT, sizeof(int32_t) * B, cudaMemcpyDeviceToHost, s), "copy status");
    CS_TRY_LAUNCH(cudaStreamSynchronize(s), "stream synchronize");
    return CS_OK;
}

// Batched IHT: set-up, then per iteration the float32 correlation of the
// live signals and the thresholded update (eagerly or as a replayed graph).
cs_status iht_solve(cs_plan* P, const float* A, int m, int n, int lda, const float* Y, int ldy, int B,
                    int32_t* support, float* coef, int32_t* n_iter, float* res_norm, int32_t* sig_status,
                    const cs_iht_params* ip, cudaStream_t s) {
    if (!ip) return fail(CS_EINVAL, "params is NULL");
    cs_omp_params op{};
    op.k = ip->k;
    op.tol = ip->tol;
    op.max_iter = ip->max_iter > 0 ? ip->max_iter : 200;
    op.prec = CS_CORR_FP32;
    cs_status st = validate(P, A, m, n, lda, Y, ldy, B, support, coef, n_iter, res_norm, sig_status, &op);
    if (st != CS_OK) return st;
    if (!(ip->step > 0.f) || !std::isfinite(ip->step)) return fail(CS_EINVAL, "step must be finite and > 0");
    if (B == 0) return CS_OK;
    if (m > kMaxRowChunks * 128 || n > kIhtMaxN || op.k > 64 || op.k > P->k_max)
        return fail(CS_ENOTSUP, "IHT runs with m <= %d, n <= %d and k <= min(64, the plan's on-chip %d)",
                    kMaxRowChunks * 128, kIhtMaxN, P->k_max);
    DeviceGuard dg(P->device);
    if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
    st = ensure_cbuf(P);
    if (st != CS_OK) return st;
    if (!P->ihts) {
        cudaError_t e = cudaMalloc(&P->ihts, sizeof(float) * (size_t)P->B_max * (size_t)P->n_max);
        if (e != cudaSuccess) {
            P->ihts = nullptr;
            return fail(CS_ENOMEM, "cudaMalloc(IHT coefficients): %s", cudaGetErrorString(e));
        }
    }
    IterArgs a = make_args(P, m, n, B, &op, support, coef, n_iter, res_norm, sig_status);
    a.iters = op.max_iter;     // IHT runs iterations, not atoms: R may exceed k
    a.need_gcol = 0;
    a.need_gram = 0;
    const cs_plan::Prep& pr = P->prep;
    const bool reuse_a = P->a_gen != 0 && pr.gen == P->a_gen && pr.A == (const void*)A && pr.m == m &&
                         pr.n == n && pr.lda == lda;
    const float step = ip->step;
    auto enqueue = [&](cudaStream_t st_) -> cs_status {
        if (!reuse_a)
            CS_TRY_LAUNCH(timed(P, CS_PHASE_SETUP, st_, [&] {
                              return launch_prep_A(A, lda, m, n, a.mp, a.mh, P->A32, nullptr, P->colnorm_max, st_);
                          }), "prep A");
        CS_TRY_LAUNCH(cudaMemsetAsync(P->ihts, 0, sizeof(float) * (size_t)B * n, st_), "clear s");
        CS_TRY_LAUNCH(timed(P, CS_PHASE_SETUP, st_, [&] { return launch_setup(a, Y, ldy, 0, st_); }), "setup");
        for (int it = 0; it < a.iters; ++it) {
            CS_TRY_LAUNCH(timed(P, CS_PHASE_CORR, st_, [&] { return launch_corr_fp32_dense_live(a, P->cbuf, n, st_); }),
                          "correlation (fp32, dense)");
            CS_TRY_LAUNCH(timed(P, CS_PHASE_UPDATE, st_, [&] { return launch_iht_update(a, P->cbuf, n, P->ihts, step, it, st_); }),
                          "IHT update");
        }
        return CS_OK;
    };
    if (!reuse_a) {
        cs_plan::Prep np;
        np.A = A;
        np.m = m;
        np.n = n;
        np.lda = lda;
        np.gen = P->a_gen;
        P->prep = np;
    }
    const cs_status rs = run_solve(P, s, enqueue, [&](std::string& key) {
        const char tag[] = "iht";
        key.append(tag, sizeof(tag));
        const void* ptrs[] = {A, Y, support, coef, n_iter, res_norm, sig_status, P->cbuf, P->ihts};
        key.append(reinterpret_cast<const char*>(ptrs), sizeof(ptrs));
        const int ints[] = {m, n, lda, ldy, B, op.k, op.max_iter, reuse_a ? 1 : 0};
        key.append(reinterpret_cast<const char*>(ints), sizeof(ints));
        const double dk[] = {op.tol, (double)step};
        key.append(reinterpret_cast<const char*>(dk), sizeof(dk));
    }, P->use_graphs && !P->profiling);
    if (rs != CS_OK) P->prep = cs_plan::Prep{};
    return rs;
}

// Uneven batches: group instances by (A, m, n, lda, k), gather each group's
// measurements into a batch, solve it with the batched path, scatter back.
cs_status solve_varlen(cs_plan* P, const cs_instance* inst, int count, const cs_omp_params* op,
                       const cs_clomp_params* cp, cudaStream_t s) {
    if (!P) return fail(CS_EINVAL, "plan is NULL");
    if (!op) return fail(CS_EINVAL, "params is NULL");
    if (cp && cp->image_width >= 2 && (cp->tv_weight > 0.f || cp->lv_weight > 0.f))
        return fail(CS_ENOTSUP, "the image priors need a batched call (the uneven-batch regrouping mixes images)");
    if (count < 0) return fail(CS_EINVAL, "count=%d", count);
    if (count == 0) return CS_OK;
    if (!inst) return fail(CS_EINVAL, "instances is NULL");
    for (int i = 0; i < count; ++i) {
        const cs_instance& x = inst[i];
        if (!x.A || !x.y || !x.support || !x.coef || !x.n_iter || !x.res_norm || !x.sig_status)
            return fail(CS_EINVAL, "instance %d has a NULL pointer", i);
        if (x.m < 1 || x.n < 1 || x.lda < x.m || x.k < 1 || x.k > x.m || x.k > x.n)
            return fail(CS_EINVAL, "instance %d: bad sizes m=%d n=%d lda=%d k=%d", i, x.m, x.n, x.lda, x.k);
    }
    // Instances beyond the plan are not solved; those beyond the on-chip
    // kernels run on the large-instance path (OMP, Gram-form CLOMP), or are
    // not solved (other CLOMP forms, FP8, or sizes beyond that path).
    auto large = [&](const cs_instance& x) { return needs_large(P, x.m, x.n, x.k, op->prec); };
    auto refused = [&](const cs_instance& x) {
        if (op->prec == CS_CORR_FP8)   // the FP8 correlation has no large-instance form
            return x.m > P->m_max || x.n > P->n_max || x.k > P->k_max || !corr_tc_supported(x.m, x.n);
        return x.m > P->m_max || x.n > P->n_max || x.k > P->k_user ||
               (large(x) && ((cp && !large_clomp_ok(cp)) || P->no_large || !large_supported(x.m, x.n, x.k)));
    };
    // groups in order of first appearance: on-chip groups share (A, m, n,
    // lda, k); large groups share (A, m, n, lda), each instance with its k
    std::vector<std::vector<int>> groups, lgroups;
    std::vector<int> refuse;
    {
        std::map<std::string, int> at, lat;
        for (int i = 0; i < count; ++i) {
            const cs_instance& x = inst[i];
            if (refused(x)) {
                refuse.push_back(i);
                continue;
            }
            const bool lg = large(x);
            std::string key;
            key.append(reinterpret_cast<const char*>(&x.A), sizeof(x.A));
            const int dims[] = {x.m, x.n, x.lda, lg ? 0 : x.k};
            key.append(reinterpret_cast<const char*>(dims), sizeof(dims));
            auto& where = lg ? lat : at;
            auto& list = lg ? lgroups : groups;
            auto it = where.find(key);
            if (it == where.end()) {
                where[key] = (int)list.size();
                list.push_back({i});
            } else {
                list[it->second].push_back(i);
            }
        }
    }
    // staging: batch measurements, batch outputs and the pointer tables
    const size_t Bm = (size_t)P->B_max, K = (size_t)P->k_max;
    Carver cv;
    const size_t oY = cv.take<float>((size_t)std::min(P->m_max, kMaxRowChunks * 128) * Bm);
    const size_t oS = cv.take<int32_t>(K * Bm);
    const size_t oC = cv.take<float>(K * Bm);
    const size_t oN = cv.take<int32_t>(Bm);
    const size_t oR = cv.take<float>(Bm);
    const size_t oT = cv.take<int32_t>(Bm);
    const size_t oYp = cv.take<const float*>(Bm);
    const size_t oOut = cv.take<VarlenOut>(Bm);
    const size_t oRef = cv.take<VarlenRefuse>(Bm);
    if (cv.off > P->vl_bytes) {
        if (P->vl) {
            cudaFree(P->vl);
            P->vl = nullptr;
            P->vl_bytes = 0;
        }
        cudaError_t e = cudaMalloc(&P->vl, cv.off);
        if (e != cudaSuccess) return fail(CS_ENOMEM, "cudaMalloc(varlen staging): %s", cudaGetErrorString(e));
        P->vl_bytes = cv.off;
    }
    DeviceGuard dg(P->device);
    if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
    float* Yb = reinterpret_cast<float*>(P->vl + oY);
    int32_t* Sb = reinterpret_cast<int32_t*>(P->vl + oS);
    float* Cb = reinterpret_cast<float*>(P->vl + oC);
    int32_t* Nb = reinterpret_cast<int32_t*>(P->vl + oN);
    float* Rb = reinterpret_cast<float*>(P->vl + oR);
    int32_t* Tb = reinterpret_cast<int32_t*>(P->vl + oT);
    const float** Yp = reinterpret_cast<const float**>(P->vl + oYp);
    VarlenOut* Ot = reinterpret_cast<VarlenOut*>(P->vl + oOut);
    VarlenRefuse* Rt = reinterpret_cast<VarlenRefuse*>(P->vl + oRef);
    std::vector<const float*> yp;
    std::vector<VarlenOut> ot;
    std::vector<VarlenRefuse> rt;
    // A does not change during the call: groups sharing it keep its
    // preparation (copies, A^T A) under a generation of this call alone
    const uint64_t saved_gen = P->a_gen;
    static std::atomic<uint64_t> call_gen{1};
    P->a_gen = (uint64_t)0x8000000000000000ull | call_gen.fetch_add(1);
    struct Restore {
        cs_plan* P;
        uint64_t gen;
        ~Restore() {
            P->a_gen = gen;
            P->prep = cs_plan::Prep{};
        }
    } restore{P, saved_gen};   // the caller's generation back, nothing of this call kept
    for (size_t r0 = 0; r0 < refuse.size(); r0 += Bm) {
        const int nr = (int)std::min(Bm, refuse.size() - r0);
        rt.assign(nr, VarlenRefuse{});
        for (int j = 0; j < nr; ++j) {
            const cs_instance& x = inst[refuse[r0 + j]];
            rt[j] = VarlenRefuse{VarlenOut{x.support, x.coef, x.n_iter, x.res_norm, x.sig_status}, x.y, x.m, x.k};
        }
        // pageable source: staged before the call returns
        CS_TRY_LAUNCH(cudaMemcpyAsync(Rt, rt.data(), sizeof(VarlenRefuse) * nr, cudaMemcpyHostToDevice, s),
                      "copy varlen table");
        CS_TRY_LAUNCH(launch_varlen_refuse(Rt, nr, s), "varlen refuse");
    }
    for (const auto& g : groups) {
        const cs_instance& x0 = inst[g[0]];
        cs_omp_params o = *op;
        o.k = x0.k;
        cs_clomp_params c;
        if (cp) {
            c = *cp;
            c.base = o;
        }
        for (size_t b0 = 0; b0 < g.size(); b0 += Bm) {
            const int Bg = (int)std::min(Bm, g.size() - b0);
            yp.assign(Bg, nullptr);
            ot.assign(Bg, VarlenOut{});
            for (int j = 0; j < Bg; ++j) {
                const cs_instance& x = inst[g[b0 + j]];
                yp[j] = x.y;
                ot[j] = VarlenOut{x.support, x.coef, x.n_iter, x.res_norm, x.sig_status};
            }
            // the host vectors are pageable: the copies are staged before the call returns
            CS_TRY_LAUNCH(cudaMemcpyAsync(Yp, yp.data(), sizeof(const float*) * Bg, cudaMemcpyHostToDevice, s),
                          "copy varlen table");
            CS_TRY_LAUNCH(cudaMemcpyAsync(Ot, ot.data(), sizeof(VarlenOut) * Bg, cudaMemcpyHostToDevice, s),
                          "copy varlen table");
            CS_TRY_LAUNCH(launch_varlen_gather(Yp, x0.m, Bg, Yb, s), "varlen gather");
            cs_status st = solve(P, x0.A, x0.m, x0.n, x0.lda, Yb, x0.m, Bg, Sb, Cb, Nb, Rb, Tb, &o,
                                 cp ? &c : nullptr, s);
            if (st != CS_OK) return st;
            CS_TRY_LAUNCH(launch_varlen_scatter(Ot, x0.k, Bg, Sb, Cb, Nb, Rb, Tb, s), "varlen scatter");
        }
    }
    auto group_args = [&](const std::vector<int>& g, std::vector<const float*>& ys, std::vector<LargeOut>& outs) {
        ys.resize(g.size());
        outs.resize(g.size());
        for (size_t j = 0; j < g.size(); ++j) {
            const cs_instance& x = inst[g[j]];
            ys[j] = x.y;
            outs[j] = LargeOut{x.support, x.coef, x.n_iter, x.res_norm, x.sig_status, x.k};
        }
    };
    // a single large group: on s
    if (lgroups.size() < 2) {
        for (const auto& g : lgroups) {
            const cs_instance& x0 = inst[g[0]];
            std::vector<const float*> ys;
            std::vector<LargeOut> outs;
            group_args(g, ys, outs);
            cs_status st = solve_large(P, x0.A, x0.m, x0.n, x0.lda, ys, outs, op, cp, s);
            if (st != CS_OK) return st;
        }
        return CS_OK;
    }
    // Large groups side by side: each group's iterations are latency-bound
    // launches that leave most of the GPU idle, so up to kVarlenWorkers
    // groups run at once, each worker with its own host thread, stream and
    // workspace, taking the groups in order of decreasing work (k x n x m)
    // from a shared counter.  The workers' streams start after the work
    // already on s, and s continues after all of them.  CLOMP: the Adam table
    // is made once, here, for the longest group, and the fits run without
    // cooperative launches (a cooperative grid's CTAs could not all be
    // resident beside the other groups' kernels).
    const int nw = (int)std::min<size_t>(kVarlenWorkers, lgroups.size());
    while ((int)P->lgw.size() < nw) {
        cs_plan::LgWorker w;
        cudaError_t e = cudaStreamCreateWithFlags(&w.s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            if (w.s) cudaStreamDestroy(w.s);
            return cuda_fail(e, "varlen worker stream");
        }
        P->lgw.push_back(w);
    }
    std::vector<size_t> order(lgroups.size());
    std::vector<double> cost(lgroups.size());
    for (size_t g = 0; g < lgroups.size(); ++g) {
        const cs_instance& x0 = inst[lgroups[g][0]];
        int kmax = 0;
        for (int i : lgroups[g]) kmax = std::max(kmax, inst[i].k);
        cost[g] = (double)kmax * x0.n * x0.m;
        order[g] = g;
    }
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return cost[a] > cost[b]; });
    if (cp) {
        int len = 1;
        for (const auto& g : lgroups) {
            int kmax = 1;
            for (int i : g) kmax = std::max(kmax, inst[i].k);
            const int iters = op->max_iter > 0 ? std::min(kmax, op->max_iter) : kmax;
            len = std::max(len, (cp->reset_adam_each_iter ? 1 : iters) * std::max(cp->steps, 1));
        }
        cs_status st = ensure_tab(P, len);
        if (st != CS_OK) return st;
        CS_TRY_LAUNCH(launch_adam_table(P->tab, len, cp->lr, cp->beta1, cp->beta2, s), "adam table");
    }
    cudaEvent_t start = pool_event(P);
    if (!start) return fail(CS_ECUDA, "varlen: no event");
    CS_TRY_LAUNCH(cudaEventRecord(start, s), "varlen start event");
    for (int w = 0; w < nw; ++w) CS_TRY_LAUNCH(cudaStreamWaitEvent(P->lgw[w].s, start, 0), "varlen worker wait");
    std::atomic<size_t> next{0};
    std::mutex tune_mu;
    std::vector<cs_status> wst(nw, CS_OK);
    std::vector<std::string> wmsg(nw);
    auto work = [&](int w) {
        cudaSetDevice(P->device);
        cs_plan::LgWorker& W = P->lgw[w];
        for (;;) {
            const size_t q = next.fetch_add(1);
            if (q >= order.size()) break;
            const auto& g = lgroups[order[q]];
            const cs_instance& x0 = inst[g[0]];
            std::vector<const float*> ys;
            std::vector<LargeOut> outs;
            group_args(g, ys, outs);
            const cs_status st = solve_large_on(P, x0.A, x0.m, x0.n, x0.lda, ys, outs, op, cp, W.s, &W.ws,
                                                &W.bytes, false, &tune_mu);
            if (st != CS_OK) {
                wst[w] = st;
                wmsg[w] = g_last_error;
                next.store(order.size());      // the other workers stop after their current group
                break;
            }
        }
        cudaEventRecord(W.done, W.s);
    };
    std::vector<std::thread> threads;
    for (int w = 1; w < nw; ++w) threads.emplace_back(work, w);
    work(0);
    for (auto& t : threads) t.join();
    for (int w = 0; w < nw; ++w) CS_TRY_LAUNCH(cudaStreamWaitEvent(s, P->lgw[w].done, 0), "varlen join");
    P->pool.push_back(start);
    for (int w = 0; w < nw; ++w)
        if (wst[w] != CS_OK) return fail(wst[w], "%s", wmsg[w].c_str());
    return CS_OK;
}

}  // namespace

extern "C" {

cs_status cs_plan_create(cs_plan** plan, int32_t m_max, int32_t n_max, int32_t batch_max,
                         int32_t k_max) {
    if (!plan) return fail(CS_EINVAL, "plan out-pointer is NULL");
    *plan = nullptr;
    if (m_max < 1 || n_max < 1 || batch_max < 1 || k_max < 1)
        return fail(CS_EINVAL, "plan sizes must be >= 1 (m_max=%d n_max=%d batch_max=%d k_max=%d)",
                    m_max, n_max, batch_max, k_max);
    if (k_max > kLargeMaxK) return fail(CS_ENOTSUP, "k_max=%d exceeds %d", k_max, kLargeMaxK);
    if (m_max > kLargeMaxM) return fail(CS_ENOTSUP, "m_max=%d exceeds %d", m_max, kLargeMaxM);
    cs_plan* P = new cs_plan();
    cudaError_t e = cudaGetDevice(&P->device);
    if (e != cudaSuccess) {
        delete P;
        return cuda_fail(e, "cudaGetDevice");
    }
    P->m_max = m_max;
    P->n_max = n_max;
    P->B_max = batch_max;
    P->k_user = k_max;
    P->k_max = k_max <= 32 ? 32 : 64;   // on-chip kernels are built for 32 or 64
    // the on-chip kernels' workspace (m <= 1024); larger instances run on the
    // large-instance path, whose workspace is allocated on first use
    const int m_chip = std::min(m_max, kMaxRowChunks * 128);
    P->mp_max = round_up(m_chip, 4);
    P->mh_max = round_up(m_chip, 64);
    P->nw_max = ceil_div(n_max, 32);
    P->nch_max = ceil_div(n_max, kCorrFp32TileN);
    const bool gram_a = n_max <= kGramAMax;
    const WsLayout L = ws_layout(m_chip, n_max, batch_max, P->k_max, true, gram_a);
    e = cudaMalloc(&P->ws, L.total);
    if (e != cudaSuccess) {
        delete P;
        return fail(CS_ENOMEM, "cudaMalloc(%zu bytes): %s", L.total, cudaGetErrorString(e));
    }
    P->ws_bytes = L.total;
    bind_workspace(P, P->ws, L);
    // zero everything once so that padding rows of the bf16 operands are 0
    e = cudaMemset(P->ws, 0, L.total);
    if (e != cudaSuccess) {
        cudaFree(P->ws);
        delete P;
        return cuda_fail(e, "cudaMemset");
    }
    *plan = P;
    return CS_OK;
}

cs_status cs_plan_destroy(cs_plan* plan) {
    if (!plan) return CS_OK;
    DeviceGuard dg(plan->device);
    cudaDeviceSynchronize();
    for (auto& mk : plan->marks) {
        cudaEventDestroy(mk.a);
        cudaEventDestroy(mk.b);
    }
    for (auto e : plan->pool) cudaEventDestroy(e);
    for (auto& kv : plan->graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (plan->cap_stream) cudaStreamDestroy(plan->cap_stream);
    if (plan->ws) cudaFree(plan->ws);
    if (plan->tab) cudaFree(plan->tab);
    if (plan->cbuf) cudaFree(plan->cbuf);
    if (plan->ihts) cudaFree(plan->ihts);
    if (plan->tvE) cudaFree(plan->tvE);
    if (plan->tvT) cudaFree(plan->tvT);
    if (plan->io) cudaFree(plan->io);
    if (plan->vl) cudaFree(plan->vl);
    if (plan->lg) cudaFree(plan->lg);
    for (auto& w : plan->lgw) {
        if (w.s) cudaStreamDestroy(w.s);
        if (w.ws) cudaFree(w.ws);
        if (w.done) cudaEventDestroy(w.done);
    }
    delete plan;
    return CS_OK;
}

cs_status omp_solve_batched(cs_plan* plan, const float* A, int32_t m, int32_t n, int32_t lda,
                            const float* Y, int32_t ldy, int32_t batch, int32_t* support,
                            float* coef, int32_t* n_iter, float* res_norm, int32_t* sig_status,
                            const cs_omp_params* params, void* stream) {
    return solve(plan, A, m, n, lda, Y, ldy, batch, support, coef, n_iter, res_norm, sig_status,
                 params, nullptr, (cudaStream_t)stream);
}

cs_status omp_solve(cs_plan* plan, const float* A, int32_t m, int32_t n, int32_t lda,
                    const float* y, int32_t* support, float* coef, int32_t* n_iter,
                    float* res_norm, int32_t* sig_status, const cs_omp_params* params,
                    void* stream) {
    return solve(plan, A, m, n, lda, y, m, 1, support, coef, n_iter, res_norm, sig_status, params,
                 nullptr, (cudaStream_t)stream);
}

cs_status clomp_solve_batched(cs_plan* plan, const float* A, int32_t m, int32_t n, int32_t lda,
                              const float* Y, int32_t ldy, int32_t batch, int32_t* support,
                              float* coef, int32_t* n_iter, float* res_norm,
                              int32_t* sig_status, const cs_clomp_params* params, void* stream) {
    if (!params) return fail(CS_EINVAL, "params is NULL");
    return solve(plan, A, m, n, lda, Y, ldy, batch, support, coef, n_iter, res_norm, sig_status,
                 &params->base, params, (cudaStream_t)stream);
}

cs_status clomp_solve(cs_plan* plan, const float* A, int32_t m, int32_t n, int32_t lda,
                      const float* y, int32_t* support, float* coef, int32_t* n_iter,
                      float* res_norm, int32_t* sig_status, const cs_clomp_params* params,
                      void* stream) {
    if (!params) return fail(CS_EINVAL, "params is NULL");
    return solve(plan, A, m, n, lda, y, m, 1, support, coef, n_iter, res_norm, sig_status,
                 &params->base, params, (cudaStream_t)stream);
}

cs_status omp_solve_batched_host(cs_plan* plan, const float* A, int32_t m, int32_t n,
                                 int32_t lda, const float* Y, int32_t ldy, int32_t batch,
                                 int32_t* support, float* coef, int32_t* n_iter,
                                 float* res_norm, int32_t* sig_status,
                                 const cs_omp_params* params, void* stream) {
    return solve_host(plan, A, m, n, lda, Y, ldy, batch, support, coef, n_iter, res_norm,
                      sig_status, params, nullptr, (cudaStream_t)stream);
}

cs_status clomp_solve_batched_host(cs_plan* plan, const float* A, int32_t m, int32_t n,
                                   int32_t lda, const float* Y, int32_t ldy, int32_t batch,
                                   int32_t* support, float* coef, int32_t* n_iter,
                                   float* res_norm, int32_t* sig_status,
                                   const cs_clomp_params* params, void* stream) {
    if (!params) return fail(CS_EINVAL, "params is NULL");
    return solve_host(plan, A, m, n, lda, Y, ldy, batch, support, coef, n_iter, res_norm,
                      sig_status, &params->base, params, (cudaStream_t)stream);
}

cs_status omp_solve_varlen(cs_plan* plan, const cs_instance* instances, int32_t count,
                           const cs_omp_params* params, void* stream) {
    return solve_varlen(plan, instances, count, params, nullptr, (cudaStream_t)stream);
}

cs_status clomp_solve_varlen(cs_plan* plan, const cs_instance* instances, int32_t count,
                             const cs_clomp_params* params, void* stream) {
    if (!params) return fail(CS_EINVAL, "params is NULL");
    return solve_varlen(plan, instances, count, &params->base, params, (cudaStream_t)stream);
}

cs_status clfit_forward(const float* A, int32_t m, int32_t n, int32_t lda, const int32_t* S,
                        const float* Sv, int32_t t, int32_t lds, const float* Y, int32_t ldy,
                        int32_t batch, float* R, int32_t ldr, float* loss, void* stream) {
    if (m < 1 || n < 1 || t < 0 || batch < 0) return fail(CS_EINVAL, "bad sizes");
    if (lda < m || ldy < m || ldr < m || lds < t) return fail(CS_EINVAL, "bad leading dimension");
    if (batch == 0) return CS_OK;
    if (!A || !Y || !R || (t > 0 && (!S || !Sv))) return fail(CS_EINVAL, "NULL array");
    cudaError_t e = launch_clfit_forward(A, m, lda, S, Sv, t, lds, Y, ldy, batch, R, ldr, loss,
                                         (cudaStream_t)stream);
    return e == cudaSuccess ? CS_OK : cuda_fail(e, "clfit_forward");
}

cs_status clfit_adjoint(const float* A, int32_t m, int32_t n, int32_t lda, const int32_t* S,
                        int32_t t, int32_t lds, const float* R, int32_t ldr, int32_t batch,
                        float* grad, void* stream) {
    if (m < 1 || n < 1 || t < 0 || batch < 0) return fail(CS_EINVAL, "bad sizes");
    if (lda < m || ldr < m || lds < t) return fail(CS_EINVAL, "bad leading dimension");
    if (batch == 0 || t == 0) return CS_OK;
    if (!A || !R || !S || !grad) return fail(CS_EINVAL, "NULL array");
    cudaError_t e = launch_clfit_adjoint(A, m, lda, S, nullptr, t, lds, R, ldr, batch, grad, nullptr,
                                         nullptr, 1, 0.f, 0.f, 0.f, 0.f, 0, (cudaStream_t)stream);
    return e == cudaSuccess ? CS_OK : cuda_fail(e, "clfit_adjoint");
}

cs_status clfit_adam_step(const float* A, int32_t m, int32_t n, int32_t lda, const int32_t* S,
                          float* Sv, int32_t t, int32_t lds, const float* R, int32_t ldr,
                          int32_t batch, float* mom, float* vel, int32_t tau, float lr,
                          float beta1, float beta2, float eps, float* grad, void* stream) {
    if (m < 1 || n < 1 || t < 0 || batch < 0 || tau < 1) return fail(CS_EINVAL, "bad sizes/tau");
    if (lda < m || ldr < m || lds < t) return fail(CS_EINVAL, "bad leading dimension");
    if (!(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f)) return fail(CS_EINVAL, "bad betas");
    if (batch == 0 || t == 0) return CS_OK;
    if (!A || !R || !S || !Sv || !mom || !vel) return fail(CS_EINVAL, "NULL array");
    cudaError_t e = launch_clfit_adjoint(A, m, lda, S, Sv, t, lds, R, ldr, batch, grad, mom, vel,
                                         tau, lr, beta1, beta2, eps, 1, (cudaStream_t)stream);
    return e == cudaSuccess ? CS_OK : cuda_fail(e, "clfit_adam_step");
}

cs_status iht_solve_batched(cs_plan* plan, const float* A, int32_t m, int32_t n, int32_t lda, const float* Y,
                            int32_t ldy, int32_t batch, int32_t* support, float* coef, int32_t* n_iter,
                            float* res_norm, int32_t* sig_status, const cs_iht_params* params, void* stream) {
    return iht_solve(plan, A, m, n, lda, Y, ldy, batch, support, coef, n_iter, res_norm, sig_status, params,
                     (cudaStream_t)stream);
}

cs_status cs_correlate(cs_plan* plan, const float* A, int32_t m, int32_t n, int32_t lda,
                       const float* R, int32_t ldr, int32_t batch, int32_t prec, float* C,
                       int32_t ldc, void* stream) {
    if (!plan) return fail(CS_EINVAL, "plan is NULL");
    if (m < 1 || n < 1 || batch < 0) return fail(CS_EINVAL, "bad sizes m=%d n=%d batch=%d", m, n, batch);
    if (lda < m || ldr < m || ldc < n) return fail(CS_EINVAL, "bad leading dimension");
    if (m > plan->m_max || n > plan->n_max || batch > plan->B_max)
        return fail(CS_EINVAL, "problem exceeds the plan");
    if (m > kMaxRowChunks * 128) return fail(CS_ENOTSUP, "cs_correlate takes m <= %d (m=%d)", kMaxRowChunks * 128, m);
    if (prec != CS_CORR_FP32 && prec != CS_CORR_BF16 && prec != CS_CORR_FP8) return fail(CS_EINVAL, "prec=%d", prec);
    if (prec != CS_CORR_FP32 && !corr_tc_supported(m, n))
        return fail(CS_ENOTSUP, "tensor-core correlation unavailable for m=%d n=%d", m, n);
    if (batch == 0) return CS_OK;
    if (!A || !R || !C) return fail(CS_EINVAL, "NULL array");
    DeviceGuard dg(plan->device);
    if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    const int mp = round_up(m, 4), mh = round_up(m, 64), mq = round_up(m, 128);
    const bool bf16 = (prec == CS_CORR_BF16);
    plan->prep = cs_plan::Prep{};   // A32 / A16 / A8 are overwritten
    if (prec == CS_CORR_FP8) {
        CS_TRY_LAUNCH(cudaMemsetAsync(plan->ea, 0, sizeof(float), s), "clear FP8 error norm");
        CS_TRY_LAUNCH(launch_prep_A8(A, lda, m, n, mq, plan->A8, plan->sa, plan->ea, s), "prep A (FP8)");
        CS_TRY_LAUNCH(launch_prep_R8(R, ldr, m, batch, mq, plan->R8, plan->sr, plan->er, s), "prep R (FP8)");
        CS_TRY_LAUNCH(launch_corr_tc8_dense(plan->R8, plan->A8, plan->sr, plan->sa, mq, batch, n, C, ldc,
                                            plan->counters + 1, s), "correlation (tcgen05, FP8)");
        return CS_OK;
    }
    CS_TRY_LAUNCH(launch_prep_A(A, lda, m, n, mp, mh, plan->A32, bf16 ? plan->A16 : nullptr, nullptr, s),
                  "prep A");
    CS_TRY_LAUNCH(launch_prep_R(R, ldr, m, batch, mp, mh, bf16 ? nullptr : plan->R32,
                                bf16 ? plan->R16 : nullptr, s), "prep R");
    if (bf16)
        CS_TRY_LAUNCH(launch_corr_tc_dense(plan->R16, plan->A16, mh, batch, n, C, ldc, plan->counters + 1, s),
                      "correlation (tcgen05)");
    else
        CS_TRY_LAUNCH(launch_corr_fp32_dense(plan->R32, plan->A32, mp, batch, n, C, ldc, s),
                      "correlation (fp32)");
    return CS_OK;
}

cs_status cs_synthesize(const float* D, int32_t N, int32_t n, int32_t ldd, const int32_t* support,
                        const float* coef, const int32_t* n_iter, int32_t k, int32_t batch, float* X,
                        int32_t ldx, void* stream) {
    if (N < 1 || n < 1 || k < 1 || batch < 0) return fail(CS_EINVAL, "bad sizes N=%d n=%d k=%d batch=%d", N, n, k, batch);
    if (!D && N != n) return fail(CS_EINVAL, "without a basis the signal length is n (N=%d n=%d)", N, n);
    if ((D && ldd < N) || ldx < N) return fail(CS_EINVAL, "bad leading dimension (ldd=%d ldx=%d, N=%d)", ldd, ldx, N);
    if (batch == 0) return CS_OK;
    if (!support || !coef || !n_iter || !X) return fail(CS_EINVAL, "NULL array");
    CS_TRY_LAUNCH(launch_synthesize(D, N, n, ldd, support, coef, n_iter, k, batch, X, ldx, (cudaStream_t)stream),
                  "synthesize");
    return CS_OK;
}

cs_status cs_image_quality(const float* X, const float* Xref, int32_t H, int32_t W, int32_t count, float peak,
                           float* psnr, float* ssim, void* stream) {
    if (H < 11 || W < 11 || count < 0)
        return fail(CS_EINVAL, "images must be at least 11 x 11 (H=%d W=%d count=%d)", H, W, count);
    if ((int64_t)H * W > INT32_MAX) return fail(CS_EINVAL, "image too large");
    if (!std::isfinite(peak)) return fail(CS_EINVAL, "peak must be finite");
    if (count == 0) return CS_OK;
    if (!X || !Xref || !psnr || !ssim) return fail(CS_EINVAL, "NULL array");
    CS_TRY_LAUNCH(launch_image_quality(X, Xref, H, W, count, peak, psnr, ssim, (cudaStream_t)stream),
                  "image quality");
    return CS_OK;
}

cs_status cs_plan_counters(cs_plan* plan, uint32_t* out, int32_t reset, void* stream) {
    if (!plan || !out) return fail(CS_EINVAL, "NULL argument");
    DeviceGuard dg(plan->device);
    if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
    return read_counters(plan->counters, out, reset, (cudaStream_t)stream);
}

cs_status cs_plan_set_A_generation(cs_plan* plan, uint64_t generation) {
    if (!plan) return fail(CS_EINVAL, "plan is NULL");
    plan->a_gen = generation;
    if (generation == 0) plan->prep = cs_plan::Prep{};
    return CS_OK;
}

cs_status cs_plan_set_profiling(cs_plan* plan, int32_t enable) {
    if (!plan) return fail(CS_EINVAL, "plan is NULL");
    plan->profiling = enable ? 1 : 0;
    return CS_OK;
}

cs_status cs_plan_set_option(cs_plan* plan, int32_t option, int32_t value) {
    if (!plan) return fail(CS_EINVAL, "plan is NULL");
    switch (option) {
        case CS_OPT_GRAPHS: plan->use_graphs = value ? 1 : 0; return CS_OK;
        case CS_OPT_FUSE_UPDATE: plan->fuse_update = value ? 1 : 0; return CS_OK;
        case CS_OPT_PERSIST: plan->persist = value ? 1 : 0; return CS_OK;
        case CS_OPT_STALL_TEST: plan->stall_test = value ? 1 : 0; return CS_OK;
        case CS_OPT_FUSED_OMP: plan->fused_omp = value ? 1 : 0; return CS_OK;
        case CS_OPT_AUTOTUNE: plan->autotune = value ? 1 : 0; return CS_OK;
        case CS_OPT_TC_TILE:
            if (value != 0 && value != 128 && value != 256) return fail(CS_EINVAL, "tile width %d", value);
            plan->force_tile = value;
            return CS_OK;
        default: return fail(CS_EINVAL, "unknown option %d", option);
    }
}

cs_status cs_plan_profile(cs_plan* plan, double* ms, int64_t* launches, int32_t reset) {
    if (!plan) return fail(CS_EINVAL, "plan is NULL");
    DeviceGuard dg(plan->device);
    if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
    double acc[CS_PHASES] = {};
    for (auto& mk : plan->marks) {
        float t = 0.f;
        cudaError_t e = cudaEventSynchronize(mk.b);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
        e = cudaEventElapsedTime(&t, mk.a, mk.b);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
        acc[mk.phase] += t;
    }
    for (int i = 0; i < CS_PHASES; ++i) {
        if (ms) ms[i] = acc[i];
        if (launches) launches[i] = plan->launches[i];
    }
    if (reset) {
        for (auto& mk : plan->marks) {
            plan->pool.push_back(mk.a);
            plan->pool.push_back(mk.b);
        }
        plan->marks.clear();
        for (int i = 0; i < CS_PHASES; ++i) plan->launches[i] = 0;
    }
    return CS_OK;
}

cs_status cs_plan_autotune_report(cs_plan* plan, char* buf, int32_t len) {
    if (!plan || !buf || len < 1) return fail(CS_EINVAL, "NULL plan or buffer");
    std::string out;
    for (const auto& kv : plan->tuned) {
        out += kv.first;
        out += " -> ";
        out += std::to_string(kv.second);
        out += "\n";
    }
    const size_t nb = std::min(out.size(), (size_t)len - 1);
    memcpy(buf, out.data(), nb);
    buf[nb] = '\0';
    return out.size() < (size_t)len ? CS_OK : fail(CS_EINVAL, "buffer too short (%zu bytes needed)", out.size() + 1);
}

const char* cs_last_error(void) { return g_last_error.c_str(); }

const char* cs_version(void) { return "cs-omp-gb300 0.1 (sm_103a)"; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free batched OMP.
//
// Some callers cannot allocate device memory at the time they want to solve:
// real-time loops that forbid allocator calls after start-up (an allocation
// can block for an unbounded time), and host applications or plug-ins whose
// own device allocator owns all the memory and hands none to libraries.
// omp_solve_batched_noalloc serves them: it runs the
// same kernels as omp_solve_batched, but its scratch (the padded copies of A
// and Y, the residuals, candidate lists, support bitsets and the float64
// Cholesky factors) lives in one fixed file-scope device array instead of a
// plan.  Every GPU that loads this library reserves that array until the
// process exits.
//
// The host cannot use the array's name as a device address, so the first
// call on each device (with that device current) looks the address up with
// cudaGetSymbolAddress and caches it; later calls reuse it.  That first call
// therefore belongs before any stream capture, and the cached address is not
// valid across a reset of the device (cudaDeviceReset destroys the context
// the address belongs to).  All calls share the one array and find the
// previous call's contents in it: everything a solve reads is written by that
// solve first, and the device counters -- kept in the array's first 256
// bytes, where omp_solve_batched_noalloc_counters finds them whatever the
// problem's layout -- are cleared at the start of every call.  Two calls
// whose work overlaps on the GPU (different streams, or different host
// threads) race on the array.

static constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr int kNoAllocMaxDevices = 64;
constexpr size_t kNoAllocCounterBytes = 256;   // the counters, ahead of the solve's layout
std::mutex g_noalloc_mu;
void* g_noalloc_base[kNoAllocMaxDevices] = {};

// The array's device address on the current device (looked up on the first
// call per device).
cs_status noalloc_base(char** base, int* device) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(CS_ENOTSUP, "device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_base[dev]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        g_noalloc_base[dev] = ptr;
    }
    *base = static_cast<char*>(g_noalloc_base[dev]);
    *device = dev;
    return CS_OK;
}

}  // namespace

extern "C" cs_status omp_solve_batched_noalloc(const float* A, int32_t m, int32_t n, int32_t lda,
                                               const float* Y, int32_t ldy, int32_t batch,
                                               int32_t* support, float* coef, int32_t* n_iter,
                                               float* res_norm, int32_t* sig_status,
                                               const cs_omp_params* params, void* stream) {
    if (!params) return fail(CS_EINVAL, "params is NULL");
    if (m < 1 || n < 1 || batch < 0 || params->k < 1 || params->k > kKmaxLimit)
        return fail(CS_EINVAL, "bad sizes m=%d n=%d batch=%d k=%d", m, n, batch, params->k);
    if (m > kMaxRowChunks * 128) return fail(CS_ENOTSUP, "m=%d exceeds %d", m, kMaxRowChunks * 128);

    // Scratch layout for exactly this problem (same buffers as a plan).
    cs_plan P;
    P.m_max = m;
    P.n_max = n;
    P.B_max = std::max(batch, 1);
    P.k_max = params->k <= 32 ? 32 : 64;
    P.k_user = params->k;
    P.no_large = 1;
    P.mp_max = round_up(m, 4);
    P.mh_max = round_up(m, 64);
    P.nw_max = ceil_div(n, 32);
    P.nch_max = ceil_div(n, kCorrFp32TileN);
    const WsLayout L = ws_layout(m, n, P.B_max, P.k_max, false, false);
    if (L.total > kNoAllocScratchBytes - kNoAllocCounterBytes)
        return fail(CS_EINVAL,
                    "problem needs %zu bytes of scratch; omp_solve_batched_noalloc holds %zu "
                    "(use omp_solve_batched with a plan)",
                    L.total, kNoAllocScratchBytes - kNoAllocCounterBytes);
    if (batch == 0) return CS_OK;

    char* base = nullptr;
    int dev = 0;
    cs_status st = noalloc_base(&base, &dev);
    if (st != CS_OK) return st;
    P.device = dev;
    P.use_graphs = 0;
    // No tile tuning: this plan lives for one call, so tuning would time the
    // candidates (a stream synchronisation and two events) on every call.
    // The default tile computes the same bits as every other.
    P.autotune = 0;
    bind_workspace(&P, base + kNoAllocCounterBytes, L);
    P.counters = reinterpret_cast<unsigned*>(base);
    // The previous call's counters must not leak into this one.
    cudaError_t e = cudaMemsetAsync(P.counters, 0, 16 * sizeof(unsigned), (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(counters)");
    return solve(&P, A, m, n, lda, Y, ldy, batch, support, coef, n_iter, res_norm, sig_status, params,
                 nullptr, (cudaStream_t)stream);
}

extern "C" cs_status omp_solve_batched_noalloc_counters(uint32_t* out, int32_t reset, void* stream) {
    if (!out) return fail(CS_EINVAL, "out is NULL");
    char* base = nullptr;
    int dev = 0;
    cs_status st = noalloc_base(&base, &dev);
    if (st != CS_OK) return st;
    return read_counters(reinterpret_cast<unsigned*>(base), out, reset, (cudaStream_t)stream);
}
