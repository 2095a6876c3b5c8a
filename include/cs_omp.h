/*
 * cs_omp.h -- C ABI of the GB300 (sm_103a) sparse-reconstruction hot path:
 * batched Orthogonal Matching Pursuit (OMP) and its coefficients-learning
 * variant CLOMP, from arXiv 2501.11592 ("Training-free Ultra Small Model for
 * Universal Sparse Reconstruction in Compressed Sensing").
 *
 * Problem (Eq. 1 and Eq. 3): y = A s + xi for every column y of Y, with one
 * shared measurement matrix A (m x n, m < n) and k-sparse s.  Each solver
 * iteration (Methods, "Coefficients learning on OMP"):
 *   1. correlation c = A^T r (the residual-injection branch, a fixed-weight
 *      fully connected layer applied to r^T);
 *   2. selection of the atom with the largest |c_j| not yet selected (lowest
 *      index on exact ties), OR-ed into the support mask;
 *   3. coefficient fit on the support: least squares, i.e. pinv(A(:,Mask))
 *      (OMP, Table "s forward block"), or Adam steps on the residual loss
 *      1/2 ||y - A_S s_S||^2 with s learnable (CLOMP, structure 1);
 *   4. residual r = y - A_S s_S and the stopping test of Eq. 2.
 *
 * Conventions shared by every entry point:
 *   - All matrices are column-major float32.  A has leading dimension lda >= m;
 *     Y has leading dimension ldy >= m.  Per-signal outputs with k entries
 *     (support, coef) are k x batch column-major: signal b owns
 *     [b*k, b*k + k), in selection order; unused slots hold -1 / 0.
 *   - Unless an entry point says otherwise, every array pointer is a DEVICE
 *     pointer owned by the caller.  The library never frees it and keeps no
 *     reference to it after the call returns.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     are asynchronous and stream-ordered; results are valid once the stream
 *     has been synchronised.
 *   - Argument errors are reported synchronously (CS_EINVAL / CS_ENOTSUP)
 *     before anything is launched.  A CUDA error at launch returns CS_ECUDA.
 *     Per-signal failures never abort the batch: they are written to
 *     sig_status (see CS_SIG_*).  cs_last_error() gives a message for the
 *     last non-OK return on the calling thread.
 *   - A plan owns the device workspace.  It is not thread-safe; use one plan
 *     per stream (or serialise calls on one stream).
 */
#ifndef CS_OMP_H
#define CS_OMP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CS_OK = 0,
    CS_EINVAL = -1,    /* invalid argument (nothing was launched) */
    CS_ENOMEM = -2,    /* device allocation failed */
    CS_ECUDA = -3,     /* a CUDA call or launch failed */
    CS_ETIMEOUT = -4,  /* a bounded device-side wait gave up */
    CS_ENOTSUP = -5    /* valid but unsupported configuration (e.g. k above the plan limit) */
} cs_status;

/* Per-signal status written to sig_status (Eq. 2 stopping rule; R = max_iter). */
enum {
    CS_SIG_REACHED_K = 0,     /* |S| = k */
    CS_SIG_REACHED_TOL = 1,   /* ||r||_2 <= tol */
    CS_SIG_MAX_ITER = 2,      /* max_iter iterations without reaching k or tol */
    CS_SIG_DEPENDENT = 3,     /* the selected atom is linearly dependent on the support
                                 (pivot^2 <= 2^-20 ||a||^2); it is not added */
    CS_SIG_NONFINITE = 4,     /* y holds a NaN or Inf; no iteration is run */
    CS_SIG_UNSUPPORTED = 5    /* uneven batches only: the instance's sizes exceed what the
                                 plan or the kernels solve (see omp_solve_varlen); it is not
                                 solved: support -1, coef 0, n_iter 0, res_norm ||y||_2 */
};

/* Arithmetic of the correlation c = A^T r (step 1).  The selection always
 * re-scores the low-precision candidates in float32. */
typedef enum {
    CS_CORR_FP32 = 0,   /* float32 SIMT correlation, exact float32 argmax */
    CS_CORR_BF16 = 1,   /* bf16 tensor-core correlation (tcgen05, fp32 accumulate), two
                           best atoms per 16-atom group, fp32 re-score of the 8 best and of
                           every atom the rounding bound cannot rule out (n <= 4096,
                           m <= 256; OMP and Gram-form CLOMP beyond that run the
                           large-instance path with a bf16 copy of A, see
                           omp_solve_batched) */
    CS_CORR_FP8 = 2     /* FP8 (E4M3) tensor-core correlation (tcgen05 kind::f8f6f4, fp32
                           accumulate): each column of A scaled by max|a_j| / 448 once per
                           solve, each residual by max|r| / 448 every iteration; the same
                           candidates and fp32 re-score as bf16, with a rounding bound built
                           from the exact quantisation-error norms of both operands
                           (n <= 4096, m <= 256, k within the plan's on-chip 32 or 64;
                           CS_ENOTSUP otherwise) */
} cs_corr_prec;

/* How the CLOMP coefficient fit evaluates its gradient -A_S^T (y - A_S s_S). */
typedef enum {
    CS_CL_GATHER = 0,   /* residual and adjoint by gathering the columns of A_S (literal form) */
    CS_CL_GRAM = 1      /* same gradient as G s_S - A_S^T y with G = A_S^T A_S kept per signal */
} cs_cl_form;

typedef struct {
    int32_t k;          /* target sparsity, 1 <= k <= min(m, n, plan k_max) */
    double tol;         /* stop once ||r||_2 <= tol (epsilon of Eq. 2); 0 disables it */
    int32_t max_iter;   /* R: at most this many iterations; <= 0 means k */
    int32_t prec;       /* cs_corr_prec */
    int32_t topc;       /* reserved, must be 0..8 */
} cs_omp_params;

typedef struct {
    cs_omp_params base;
    int32_t steps;                  /* Adam steps per iteration (T >= 0) */
    float lr, beta1, beta2, eps;    /* Adam hyper-parameters (PyTorch update rule) */
    int32_t reset_adam_each_iter;   /* 0: one Adam state and step counter for the whole
                                       solve; 1: reset them at every iteration */
    int32_t form;                   /* cs_cl_form */
    float select_threshold;         /* Th.  0 (or >= 1): one atom per iteration, the largest
                                       |c_j| among unselected atoms.  0 < Th < 1: every
                                       unselected atom with |c_j| >= Th * max|c| joins the
                                       support in the iteration, largest first, until k
                                       (the paper's normalized cut-off threshold of the
                                       s forward block; Methods).  n_iter then counts
                                       atoms.  0 < Th < 1 needs the float32 correlation
                                       (CS_CORR_FP32), the Gram form, m <= 1024 and
                                       k <= 32, else CS_ENOTSUP; the plan then holds a
                                       batch_max x n_max float32 correlation buffer. */
    float tv_weight;                /* w >= 0: adds w * TV(x) to the fit's loss, the total-
                                       variation prior of a 1-D signal (Eq. 5) on x = D s:
                                       TV(x) = (1/N) sum_{j<N-1} (x_j - x_{j+1})^2.  0: no
                                       prior.  Needs the Gram form and n <= 4096 (the prior
                                       enters as (2w/N) (Delta D)^T (Delta D) added to A^T A);
                                       the plan then holds n_max x (n_max + N) float32
                                       scratch.  The selection and the residual are those of
                                       the data term. */
    const float* tv_D;              /* N x n sparsifying basis (device, column-major,
                                       leading dimension tv_ldd >= N), x = D s; NULL: x = s
                                       (N = n).  Used by both priors. */
    int32_t tv_N;                   /* N, the signal length (rows of tv_D, >= 2) */
    int32_t tv_ldd;
    int32_t image_width;            /* W.  0 or 1: the 1-D prior above on every column.
                                       W >= 2 (with tv_weight > 0): the batch is a sequence
                                       of images of W consecutive columns (signal b is
                                       column b mod W of image b / W) and the prior is the
                                       total variation of an image (Eq. 6):
                                       TV(I) = (1/N) sum_{i<N-1,j} (I_ij - I_i+1,j)^2
                                             + (1/W) sum_{i,j<W-1} (I_ij - I_i,j+1)^2,
                                       I = [D s_1 ... D s_W].  The horizontal part couples
                                       neighbouring columns, so an image's columns take
                                       their Adam steps together; it is evaluated as
                                       (1/W) sum_j ||s_j - s_j+1||^2, which needs tv_D with
                                       orthonormal columns (D^T D = I, e.g. the DCT) or NULL.
                                       Runs the per-iteration kernels (not the persistent
                                       solve); needs one atom per iteration, k <= 32,
                                       W <= 512 and batch a multiple of W, else CS_ENOTSUP.
                                       With lv_weight > 0 it is the width of the images the
                                       local variation is taken over. */
    float lv_weight;                /* w_lv >= 0: adds w_lv * LV(I) to the fit's loss, the
                                       local variation of an image (Eq. 7): the mean, over
                                       the 3 x 3 windows at every placement inside the
                                       image, of the window's sample standard deviation
                                       (nine pixels, divided by 8, smoothed as
                                       sqrt(var + lv_eps^2)), I = [D s_1 ... D s_W]
                                       (tv_D with any columns, or NULL: x = s; its N <= 256
                                       pixels per column).  A constant window adds no
                                       gradient.  Needs image_width >= 2 (CS_EINVAL
                                       otherwise; widths or heights below 3 have no window)
                                       and the limits of image_width above. */
    float lv_eps;                   /* >= 0: the deviation's smoothing.  With 0 (the plain
                                       deviation) the fit is ill-conditioned where windows
                                       are nearly constant: the deviation's gradient there
                                       follows the pixels' rounding.  Choose it small
                                       against the pixels' scale (the Python binding uses
                                       1e-4). */
} cs_clomp_params;

typedef struct cs_plan cs_plan;

/* Create a plan on the current CUDA device with workspace for problems up to
 * m_max x n_max (m_max <= 32768), batch_max signals and k_max <= 4096
 * iterations.  Allocates the on-chip kernels' workspace (for m up to 1024 and
 * k up to 32 or 64) at once.  Later calls allocate when a CLOMP call needs a
 * longer Adam bias-correction table than any earlier call, on the first use
 * of the host-buffer and varlen entry points, and when a solve first needs
 * the large-instance path (sized for that solve's chunk of signals: at most
 * about 8 GB plus one signal).  Returns CS_EINVAL for non-positive sizes,
 * CS_ENOTSUP for k_max > 4096 or m_max > 32768, CS_ENOMEM / CS_ECUDA on
 * allocation failure (then *plan is NULL). */
cs_status cs_plan_create(cs_plan** plan, int32_t m_max, int32_t n_max, int32_t batch_max,
                         int32_t k_max);

/* Release a plan's device memory (synchronises the device first).  NULL is a no-op. */
cs_status cs_plan_destroy(cs_plan* plan);

/* Batched plain OMP (Table "s forward block", OMP row: least squares on the
 * selected columns), one shared A, `batch` columns of Y.
 * Least squares by an incremental Cholesky factorisation of A_S^T A_S in
 * float64 (Gram entries from float32 dot products), triangular solves in
 * float64; correlation and residual in float32 (or bf16 correlation, see prec).
 * Outputs (device, caller-owned): support, coef (k x batch), n_iter, res_norm
 * (||r||_2 at exit), sig_status (batch each).  batch == 0 is a no-op.
 * Problems beyond the on-chip kernels (m > 1024, k above the plan's on-chip
 * 32 or 64, or bf16 with m > 256 or n > 4096) run the large-instance path:
 * A streamed from HBM every iteration (bf16 copy or the float32 A), the same
 * certified selection, float64 W = L^-T updated by grid-wide partial sums;
 * up to m = 32768 and k = 4096; the call synchronises `stream` every 64
 * iterations to end early once every signal has stopped. */
cs_status omp_solve_batched(cs_plan* plan, const float* A, int32_t m, int32_t n, int32_t lda,
                            const float* Y, int32_t ldy, int32_t batch, int32_t* support,
                            float* coef, int32_t* n_iter, float* res_norm, int32_t* sig_status,
                            const cs_omp_params* params, void* stream);

/* Single-signal OMP: omp_solve_batched with batch = 1 and y of length m. */
cs_status omp_solve(cs_plan* plan, const float* A, int32_t m, int32_t n, int32_t lda,
                    const float* y, int32_t* support, float* coef, int32_t* n_iter,
                    float* res_norm, int32_t* sig_status, const cs_omp_params* params,
                    void* stream);

/* Batched CLOMP (Methods, "Coefficients learning on OMP", structure 1): the
 * OMP selection, then `steps` Adam steps on L = 1/2 ||y - A(s .* Mask)||^2
 * per iteration, s starting at zero and persisting across iterations.  coef
 * holds s on the support.  Same layouts and outputs as omp_solve_batched.
 * Beyond the on-chip kernels (the sizes listed at omp_solve_batched) the
 * large-instance path runs the Gram form with one atom per iteration and no
 * prior (form CS_CL_GRAM, select_threshold 0 or 1, tv_weight and lv_weight
 * 0; otherwise CS_ENOTSUP): G = A_S^T A_S and A_S^T y grown by one row per
 * iteration, all Adam steps of an iteration in one cooperative launch whose
 * CTAs keep their rows of G on chip and wait for each other's coefficients
 * (bounded: a wait that runs out sets error flag 32, see cs_plan_counters). */
cs_status clomp_solve_batched(cs_plan* plan, const float* A, int32_t m, int32_t n, int32_t lda,
                              const float* Y, int32_t ldy, int32_t batch, int32_t* support,
                              float* coef, int32_t* n_iter, float* res_norm,
                              int32_t* sig_status, const cs_clomp_params* params, void* stream);

/* Single-signal CLOMP: clomp_solve_batched with batch = 1. */
cs_status clomp_solve(cs_plan* plan, const float* A, int32_t m, int32_t n, int32_t lda,
                      const float* y, int32_t* support, float* coef, int32_t* n_iter,
                      float* res_norm, int32_t* sig_status, const cs_clomp_params* params,
                      void* stream);

/* Host-buffer forms of the batched solvers: every array pointer is a HOST
 * pointer (pinned memory gives the fastest copies).  The call copies A and Y
 * into plan-owned device buffers, solves on `stream`, copies the five
 * outputs back and synchronises `stream` before returning -- also when the
 * solve fails after the input copies were issued, so the caller's buffers
 * are free to reuse on any return.  The plan must have been created with
 * room for the inputs (as for the device forms). */
cs_status omp_solve_batched_host(cs_plan* plan, const float* A, int32_t m, int32_t n,
                                 int32_t lda, const float* Y, int32_t ldy, int32_t batch,
                                 int32_t* support, float* coef, int32_t* n_iter,
                                 float* res_norm, int32_t* sig_status,
                                 const cs_omp_params* params, void* stream);
cs_status clomp_solve_batched_host(cs_plan* plan, const float* A, int32_t m, int32_t n,
                                   int32_t lda, const float* Y, int32_t ldy, int32_t batch,
                                   int32_t* support, float* coef, int32_t* n_iter,
                                   float* res_norm, int32_t* sig_status,
                                   const cs_clomp_params* params, void* stream);

/* One instance of an uneven batch (thousands of signals of different n, m
 * and k, e.g. image columns, blocks and 1-D sequences of several sizes):
 * its own dictionary, measurement vector, sparsity and outputs.  Every
 * pointer is a DEVICE pointer owned by the caller; A is m x n column-major
 * with leading dimension lda; support and coef hold k entries. */
typedef struct {
    const float* A;
    int32_t m, n, lda;
    const float* y;
    int32_t k;
    int32_t* support;
    float* coef;
    int32_t* n_iter;
    float* res_norm;
    int32_t* sig_status;
} cs_instance;

/* Uneven batches: instances is a HOST array of `count` descriptors.  The
 * call groups the instances the on-chip kernels take by (A, m, n, lda, k),
 * gathers each group's measurements into a batch, runs the batched solver on
 * it and scatters the outputs back; the others run on the large-instance
 * path grouped by (A, m, n, lda), each with its own k.  The on-chip groups
 * run one after another on `stream`; up to four large groups run at once,
 * each on its own host thread, stream and workspace (the plan keeps them for
 * later calls), started after the work already on `stream`, which waits for
 * all of them before the call returns (CLOMP's fits then run one launch per
 * Adam step instead of the cooperative launch).  Those concurrent groups are
 * not counted in cs_plan_profile.  params->k is ignored (each instance
 * has its own).
 * An instance is not solved -- its sig_status is set to CS_SIG_UNSUPPORTED
 * (its A is never read) and the call goes on with the others -- when its
 * sizes exceed the plan (m > m_max, n > n_max or k > k_max), when it needs
 * the large-instance path and CLOMP is asked for outside the Gram form with
 * one atom per iteration and no prior, and with the FP8 correlation when it
 * exceeds the tensor-core sizes (m <= 256, n <= 4096, k within the plan's
 * on-chip 32 or 64).  Groups larger than batch_max run in chunks.  Device staging for the gather/scatter is
 * allocated on first use.  Malformed instances (NULL pointers, k > m or
 * k > n, lda < m) are argument errors (CS_EINVAL, nothing launched).  The
 * image priors (image_width >= 2 with tv_weight or lv_weight > 0) couple
 * consecutive signals of a batch, which the regrouping would mix:
 * CS_ENOTSUP. */
cs_status omp_solve_varlen(cs_plan* plan, const cs_instance* instances, int32_t count,
                           const cs_omp_params* params, void* stream);
cs_status clomp_solve_varlen(cs_plan* plan, const cs_instance* instances, int32_t count,
                             const cs_clomp_params* params, void* stream);

/* CL fit, forward half (Methods, s forward branch: y' = A (s .* Mask)):
 *   R[:,b] = Y[:,b] - sum_q A[:, S[b*lds+q]] * Sv[b*lds+q]   (q < t)
 *   loss[b] = 1/2 ||R[:,b]||^2
 * S (int32) and Sv (float) are t x batch with leading dimension lds >= t;
 * R has leading dimension ldr >= m.  loss may be NULL.  Support indices must
 * lie in [0, n). */
cs_status clfit_forward(const float* A, int32_t m, int32_t n, int32_t lda, const int32_t* S,
                        const float* Sv, int32_t t, int32_t lds, const float* Y, int32_t ldy,
                        int32_t batch, float* R, int32_t ldr, float* loss, void* stream);

/* CL fit, adjoint half (back-propagation of the residual loss through the
 * fixed layer A):  grad[b*lds+q] = -A[:, S[b*lds+q]]^T R[:,b]  for q < t. */
cs_status clfit_adjoint(const float* A, int32_t m, int32_t n, int32_t lda, const int32_t* S,
                        int32_t t, int32_t lds, const float* R, int32_t ldr, int32_t batch,
                        float* grad, void* stream);

/* Adjoint fused with one Adam step (the optimizer that learns s): computes
 * g = -A_S^T R as clfit_adjoint does, then for q < t
 *   mom = b1 mom + (1-b1) g,  vel = b2 vel + (1-b2) g^2,
 *   Sv -= lr/(1-b1^tau) * mom / (sqrt(vel)/sqrt(1-b2^tau) + eps)
 * in place.  tau >= 1 is the step counter after this step.  mom and vel are
 * t x batch with leading dimension lds.  grad may be NULL. */
cs_status clfit_adam_step(const float* A, int32_t m, int32_t n, int32_t lda, const int32_t* S,
                          float* Sv, int32_t t, int32_t lds, const float* R, int32_t ldr,
                          int32_t batch, float* mom, float* vel, int32_t tau, float lr,
                          float beta1, float beta2, float eps, float* grad, void* stream);

/* The residual-injection layer alone (Methods, "Coefficients learning on
 * OMP": A^T r as a fully connected layer with fixed weights A):
 *   C = A^T R,  C is n x batch column-major with ldc >= n, R is m x batch
 * with ldr >= m.  prec selects float32 SIMT or bf16 tensor cores (fp32
 * accumulation).  Uses the plan's workspace; asynchronous on `stream`. */
cs_status cs_correlate(cs_plan* plan, const float* A, int32_t m, int32_t n, int32_t lda,
                       const float* R, int32_t ldr, int32_t batch, int32_t prec, float* C,
                       int32_t ldc, void* stream);

/* Image columns from sparse codes (Eq. 3: the solver sees A = M D with the
 * sparsifying basis D and returns s; the signal itself is x = D s):
 *   X[:, b] = sum_{q < n_iter[b]} coef[b*k + q] * D[:, support[b*k + q]]
 * summed in q order in float32.  D is N x n column-major (ldd >= N); D =
 * NULL gives the dense code itself, x = s (N must equal n; ldd ignored):
 * the optional dense output X (n x batch) of a solve;
 * support, coef (batch x k, row b = signal b) and n_iter are the outputs of
 * a solve; entries outside [0, n) are skipped and n_iter is clamped to
 * [0, k].  X is N x batch column-major (ldx >= N), written in full.  All
 * pointers are device memory owned by the caller; asynchronous on `stream`;
 * argument errors return CS_EINVAL with no launch. */
cs_status cs_synthesize(const float* D, int32_t N, int32_t n, int32_t ldd, const int32_t* support,
                        const float* coef, const int32_t* n_iter, int32_t k, int32_t batch, float* X,
                        int32_t ldx, void* stream);

/* Quality of `count` reconstructed images against references (the figures
 * the paper reports for its image experiments, Results).  Each image is H x W
 * column-major with leading dimension H, images consecutive (image i at
 * offset i*H*W) -- e.g. the columns of a column-wise 2D solve after
 * cs_synthesize.  Per image i:
 *   psnr[i] = 10 log10(L^2 / MSE)  (+inf when MSE = 0),
 *   ssim[i] = the SSIM index of Wang, Bovik, Sheikh and Simoncelli (2004):
 *             11 x 11 Gaussian window of standard deviation 1.5 (unit sum),
 *             C1 = (0.01 L)^2, C2 = (0.03 L)^2, averaged over every window
 *             placed fully inside the image,
 * with dynamic range L = peak if peak > 0, else max - min of the reference
 * image.  Window statistics in float32 (means, then centred moments), sums
 * over windows and pixels in float64.  H, W >= 11.  psnr and ssim are
 * device arrays of count floats; asynchronous on `stream`. */
cs_status cs_image_quality(const float* X, const float* Xref, int32_t H, int32_t W, int32_t count,
                           float peak, float* psnr, float* ssim, void* stream);

/* Parameters of IHT. */
typedef struct {
    int32_t k;          /* sparsity kept by H_k, 1 <= k <= min(n, plan k_max, 64) */
    double tol;         /* stop once ||r||_2 <= tol; 0 disables it */
    int32_t max_iter;   /* R, the iteration limit; <= 0 means 200 (the paper's setting) */
    float step;         /* t > 0, the scale factor of the update (t <= 1 / sigma_max(A)^2
                           keeps the residual norm from growing) */
} cs_iht_params;

/* Batched IHT (Methods, Table "s forward block", IHT row), the paper's
 * comparison method, on the same residual-injection layer:
 *   s <- H_k(s + t A^T r),  r = y - A s,  s starting at zero,
 * where H_k keeps the k entries of largest magnitude (lowest index on exact
 * ties) and zeroes the rest.  The correlation is float32.  Stops a signal
 * when ||r||_2 <= tol (checked before the first iteration and after each)
 * with CS_SIG_REACHED_TOL, else after max_iter iterations with
 * CS_SIG_MAX_ITER; a non-finite y gives CS_SIG_NONFINITE.  Outputs as for
 * omp_solve_batched, except that support lists the k kept atoms in ascending
 * index order (not selection order) and n_iter counts iterations.  Needs
 * m <= 1024, n <= 4096 and k <= 64 (CS_ENOTSUP otherwise); the plan then
 * holds two batch_max x n_max float32 buffers (the correlations and the dense
 * s), allocated on first use.  Same argument conventions as the other
 * batched calls. */
cs_status iht_solve_batched(cs_plan* plan, const float* A, int32_t m, int32_t n, int32_t lda,
                            const float* Y, int32_t ldy, int32_t batch, int32_t* support, float* coef,
                            int32_t* n_iter, float* res_norm, int32_t* sig_status,
                            const cs_iht_params* params, void* stream);

/* Synchronise `stream` and copy the plan's device counters to out[0..3]:
 * out[0] = picks where the bf16 candidates did not certify the winner and
 * further atoms (the "suspects") were re-scored in float32; out[1] = device error flags (non-zero
 * when a bounded wait inside a kernel gave up: 1, 2 the tensor-core
 * correlation's tile pipeline; 4, 8, 16 the persistent CLOMP solve's roles;
 * 32 the large-instance CLOMP fit's wait for other CTAs' coefficients; 64
 * the large-instance correlation's tile ring; 128 its tensor-core GEMM form).
 * reset != 0 zeroes them.  Returns CS_ETIMEOUT when out[1] != 0. */
cs_status cs_plan_counters(cs_plan* plan, uint32_t* out, int32_t reset, void* stream);

/* Batched plain OMP without any device allocation.  The paper has no
 * counterpart: this serves callers that cannot allocate device memory when
 * they solve -- real-time loops that forbid allocator calls after start-up,
 * or host applications and plug-ins whose own allocator already owns the
 * device memory and hands none to libraries.  Same arguments, kernels and
 * results as omp_solve_batched, minus the plan: the scratch is one fixed
 * 32 MiB device array that every GPU loading this library reserves until
 * the process exits (about 21 KiB per signal at m = 256, k <= 32, plus
 * 6 bytes per element of A; larger problems get CS_EINVAL and belong on
 * omp_solve_batched).  The first call on each device looks the array's
 * address up (make it before any stream capture) and keeps it for the life
 * of the process, so do not use this entry point on a device after a reset
 * of that device (cudaDeviceReset).  Calls whose GPU work overlaps -- on
 * different streams or threads -- race on the shared array.  Each call
 * clears the device counters (certificate fallbacks, error flags) when it
 * starts; omp_solve_batched_noalloc_counters reads them.  It tunes no tile
 * shape (the default tile gives the same results as a tuned one), so a call
 * creates no CUDA events and does not wait on the stream. */
cs_status omp_solve_batched_noalloc(const float* A, int32_t m, int32_t n, int32_t lda,
                                    const float* Y, int32_t ldy, int32_t batch, int32_t* support,
                                    float* coef, int32_t* n_iter, float* res_norm,
                                    int32_t* sig_status, const cs_omp_params* params,
                                    void* stream);

/* The counters of the last omp_solve_batched_noalloc call on the current
 * device, as cs_plan_counters gives them for a plan: synchronises `stream`,
 * copies them to out[0..3] (out[0] = certificate fallbacks of the bf16
 * correlation, out[1] = device error flags), zeroes them when reset != 0 and
 * returns CS_ETIMEOUT when out[1] != 0 -- the results of that call are then
 * unspecified, although the call itself returned CS_OK.  Read them after the
 * call and before the next one (which clears them).  Allocates nothing. */
cs_status omp_solve_batched_noalloc_counters(uint32_t* out, int32_t reset, void* stream);

/* Measurement support.  Phases of a solve: */
enum {
    CS_PHASE_SETUP = 0,    /* copy/convert A and Y, initial state, Adam table */
    CS_PHASE_CORR = 1,     /* correlation A^T r with the fused candidate epilogue */
    CS_PHASE_SELECT = 2,   /* candidate merge, float32 re-score, support update, Gram column */
    CS_PHASE_FIT = 3,      /* Cholesky update (OMP) or Adam coefficient fit (CLOMP) */
    CS_PHASE_RESID = 4,    /* residual, norm and stopping test */
    CS_PHASE_UPDATE = 5,   /* CLOMP Gram form: selection + fit + residual in one kernel */
    CS_PHASE_PERSIST = 6,  /* CLOMP Gram form, bf16: every iteration in one persistent kernel */
    CS_PHASES = 7
};

/* A as a fixed layer (Methods: A is set once as the fixed parameters of a
 * fully connected layer).  generation != 0: a solve leaves A's preparation in
 * the plan (the float32 and bf16 copies, the largest column norm, A^T A), and
 * a later solve whose generation, A pointer, m, n and lda all match reuses it
 * instead of preparing A again.  The generation is the authority: the caller
 * must change it whenever the contents of A change, under the same pointer or
 * not (a pointer check alone cannot tell a freed and reallocated buffer from
 * the old one).  The host-buffer entry points key on the caller's host A and
 * still copy A to the device on every call.  0 (the default): every solve
 * prepares A.  A solve with the TV prior re-prepares A and leaves A^T A
 * modified, so nothing of its A^T A is reused; cs_correlate, a failed solve
 * and a new generation drop what was kept.  Errors: CS_EINVAL for a NULL
 * plan. */
cs_status cs_plan_set_A_generation(cs_plan* plan, uint64_t generation);

/* enable != 0: bracket every later kernel launch of solves on this plan with
 * CUDA events on the solve's stream (adds a little GPU time per launch). */
cs_status cs_plan_set_profiling(cs_plan* plan, int32_t enable);

/* Plan options (all on by default):
 *   CS_OPT_GRAPHS: replay repeated identical solves as a captured CUDA graph
 *     (the first call of a configuration runs eagerly, the second is
 *     captured on a private stream, later ones replay it on `stream`);
 *   CS_OPT_FUSE_UPDATE: CLOMP in Gram form runs selection, Adam fit and
 *     residual of an iteration as one kernel (m <= 256);
 *   CS_OPT_PERSIST: CLOMP in Gram form with the bf16 correlation runs the
 *     whole solve as one persistent kernel, one CTA per SM owning a block of
 *     signals (m <= 256, n <= 2048, k <= 32; otherwise the per-iteration
 *     kernels run);
 *   CS_OPT_FUSED_OMP: plain OMP with the float32 correlation runs a batch
 *     of at most one signal per SM as one kernel, one CTA per signal (the
 *     whole solve in one launch; n <= 4096, m <= 1024).
 * Results are identical either way: every form selects the float32 argmax of
 * |A^T r| (certified from the bf16 correlation) and runs the same float32
 * fit and residual arithmetic. */
enum { CS_OPT_GRAPHS = 0, CS_OPT_FUSE_UPDATE = 1, CS_OPT_PERSIST = 2, CS_OPT_STALL_TEST = 3,
       CS_OPT_FUSED_OMP = 4, CS_OPT_AUTOTUNE = 5, CS_OPT_TC_TILE = 6 };
/* CS_OPT_AUTOTUNE (on by default): the first solve of each size class
 * (kernel, correlation precision, m, n, batch) times the candidate
 * configurations of its tunable kernels on its own data -- the tensor-core
 * correlation's tile width (128 or 256 atoms per CTA) and the large-instance
 * correlation's signals per pass -- and keeps the fastest
 * in the plan for later solves.  Every configuration computes the same bits,
 * so tuning changes only timing; the tuning solve synchronises its stream
 * while it measures, and no tuning happens inside stream capture (the
 * defaults run there until a class is tuned).  cs_plan_autotune_report lists
 * the choices.
 * CS_OPT_TC_TILE: 128 or 256 forces the tensor-core correlation's tile
 * width; 0 (default) leaves it to the autotuner (256 untuned). */
/* CS_OPT_STALL_TEST (test hook for the failure path, value 1): the next
 * persistent CLOMP solve on this plan runs without graphs and withholds the
 * completion signal of the last atom tile of its first correlation pass, so
 * that the signal warps' bounded wait (about 2 s) runs out.  The kernel then
 * stops every role, lets its copies and MMAs finish, frees its tensor memory
 * and returns; cs_plan_counters reports CS_ETIMEOUT; that solve's outputs are
 * unspecified; the context and the plan stay usable.  The option clears
 * itself after that solve. */
cs_status cs_plan_set_option(cs_plan* plan, int32_t option, int32_t value);

/* The autotuner's choices so far, one line per size class ("<kernel>
 * prec=.. m=.. n=.. B=.. -> <configuration index>"), NUL-terminated in buf
 * (len bytes).  Configuration indices: tensor-core tile 0 = 256 atoms,
 * 1 = 128; large-instance correlation 2 x log2(signals per pass: 1, 2 or
 * 4).  CS_EINVAL when buf is too short (then truncated). */
cs_status cs_plan_autotune_report(cs_plan* plan, char* buf, int32_t len);

/* Kernel launches per phase since the last reset (always counted), and --
 * when profiling was enabled -- the summed event time per phase in
 * milliseconds.  ms and launches hold CS_PHASES entries each (either may be
 * NULL).  Waits for the recorded events.  reset != 0 clears both. */
cs_status cs_plan_profile(cs_plan* plan, double* ms, int64_t* launches, int32_t reset);

/* Message describing the last non-OK return on the calling thread ("" if none). */
const char* cs_last_error(void);

/* Library version string. */
const char* cs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CS_OMP_H */
