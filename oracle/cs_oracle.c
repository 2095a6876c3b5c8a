/*
 * cs_oracle.c -- plain, slow, FP64 CPU oracle for OMP and CLOMP.
 *
 * TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load this library.  It shares
 * no code, header, table or helper with the CUDA implementation.
 *
 * What it computes (arXiv 2501.11592):
 *   - Problem: y = A s + xi (Eq. 1), columns of Y = A S + xi share A (Eq. 3);
 *     solve min ||s||_0 s.t. ||A s - y||_2 < eps (Eq. 2).
 *   - OMP (Methods, Table "s forward block", row OMP; Methods "Coefficients
 *     learning on OMP"): per iteration correlate A^T r, take the position of
 *     the largest |A^T r| among atoms not yet selected, fit the coefficients on
 *     the selected columns by least squares (the pinv of A(:,Mask)), update
 *     the residual.  The least-squares fit here is a Householder QR of A_S
 *     recomputed from scratch at every iteration (a different algorithm from
 *     the GPU's incremental Cholesky) while m k^3 / 3 <= 1e9; larger problems
 *     (k in the thousands) grow a QR factorisation by one column per
 *     iteration instead: modified Gram-Schmidt of the new column against the
 *     previous orthonormal columns, applied twice, then back substitution.
 *   - IHT (Table "s forward block", IHT row), the paper's comparison method:
 *     s <- H_k(s + t A^T r), keeping the k largest magnitudes.
 *   - CLOMP, structure 1 (Methods "Coefficients learning on OMP"): the same
 *     selection, but s (n learnable parameters) is masked by the OR-accumulated
 *     Mask, y' = A (s .* Mask) is formed, and s is learned by back-propagating
 *     the residual loss; the optimizer is Adam.
 *
 * Readings of points the paper leaves open (each one is also listed in the
 * design notes):
 *   - one atom per iteration (argmax), lowest index on exact ties; or, as an
 *     option (the paper's threshold Th of the "s forward block", used with
 *     stOMP-style selection), every atom not yet selected with
 *     |c_j| >= Th * max |c|, largest |c| first, at most k atoms in total;
 *   - already-selected atoms are excluded from the argmax;
 *   - residual r = y - A s (the sign of Eq. 2's r does not change |A^T r|);
 *   - residual loss L = 1/2 ||y - A (s .* Mask)||_2^2, gradient
 *     -(A^T r) .* Mask;
 *   - Adam with one state (m, v) and one step counter tau for the whole solve,
 *     PyTorch/Paddle update rule s -= lr * (m/(1-b1^tau)) / (sqrt(v/(1-b2^tau)) + eps);
 *     optional reset of (m, v, tau) at every iteration;
 *   - s starts at zero; stop when |S| = k, ||r||_2 <= tol, or after max_iter
 *     iterations (R of the paper);
 *   - an atom whose QR pivot satisfies R_tt^2 <= 1e-12 ||a||^2 is dependent:
 *     it is not added and the signal stops (status 3);
 *   - a non-finite measurement stops the signal before any iteration (status 4).
 *   - prior losses (Eq. 4-6) join the fit's loss with weight w: the 1-D total
 *     variation of each column x = D s (Eq. 5), or, for a batch of images of
 *     W consecutive columns, the image form (Eq. 6) whose horizontal part
 *     couples neighbouring columns, as does the local variation of Eq. 7
 *     (standard deviations over 3 x 3 windows); the columns of an image then take their
 *     Adam steps together, each step's gradients from the coefficients
 *     before it.
 *
 * Per-signal status codes: 0 reached k, 1 reached tol, 2 hit max_iter,
 * 3 dependent atom, 4 non-finite input.
 *
 * Layouts: A is m x n column-major with leading dimension lda; Y is m x B with
 * leading dimension ldy; per-iteration outputs (support, coef, top1, top2,
 * res_hist) are k x B column-major, i.e. signal b owns [b*k, b*k + k).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ST_K 0
#define ST_TOL 1
#define ST_MAXIT 2
#define ST_DEP 3
#define ST_NONFINITE 4

static double dot(const double* a, const double* b, int m) {
    double s = 0.0;
    for (int i = 0; i < m; ++i) s += a[i] * b[i];
    return s;
}

static double nrm2(const double* a, int m) { return sqrt(dot(a, a, m)); }

/*
 * Least squares min_z ||y - As z||_2 for As (m x t, column-major, leading
 * dimension lda) by Householder QR: As = Q R, z = R^{-1} (Q^T y)[0:t].
 * Returns 0, or 3 when the last column is dependent on the others
 * (R_tt^2 <= 1e-12 ||a_t||^2).  work must hold m*t + m doubles.
 */
int cs_oracle_lstsq(int m, int t, const double* As, int lda, const double* y,
                    double* z, double* work) {
    double* Rm = work;            /* m x t copy, overwritten by R and the reflectors */
    double* qty = work + (size_t)m * t;
    for (int j = 0; j < t; ++j) memcpy(Rm + (size_t)j * m, As + (size_t)j * lda, sizeof(double) * m);
    memcpy(qty, y, sizeof(double) * m);
    double last_norm = nrm2(As + (size_t)(t - 1) * lda, m);
    for (int j = 0; j < t; ++j) {
        double* col = Rm + (size_t)j * m;
        if (j >= m) return ST_DEP;
        double norm = 0.0;
        for (int i = j; i < m; ++i) norm += col[i] * col[i];
        norm = sqrt(norm);
        if (norm == 0.0) {
            if (j == t - 1) return ST_DEP;
            continue;
        }
        double alpha = (col[j] >= 0.0) ? -norm : norm;   /* R_jj */
        /* reflector v = x - alpha e_j stored in place below the diagonal */
        double v0 = col[j] - alpha;
        double vtv = v0 * v0;
        for (int i = j + 1; i < m; ++i) vtv += col[i] * col[i];
        col[j] = v0;
        /* apply H = I - 2 v v^T / (v^T v) to the remaining columns and to y */
        for (int q = j + 1; q < t; ++q) {
            double* c = Rm + (size_t)q * m;
            double s = 0.0;
            for (int i = j; i < m; ++i) s += col[i] * c[i];
            s = 2.0 * s / vtv;
            for (int i = j; i < m; ++i) c[i] -= s * col[i];
        }
        {
            double s = 0.0;
            for (int i = j; i < m; ++i) s += col[i] * qty[i];
            s = 2.0 * s / vtv;
            for (int i = j; i < m; ++i) qty[i] -= s * col[i];
        }
        col[j] = alpha;   /* keep R_jj on the diagonal (reflector no longer needed) */
    }
    {
        double rtt = Rm[(size_t)(t - 1) * m + (t - 1)];
        if (rtt * rtt <= 1e-12 * last_norm * last_norm) return ST_DEP;
    }
    /* back substitution R z = (Q^T y)[0:t] */
    for (int i = t - 1; i >= 0; --i) {
        double s = qty[i];
        for (int q = i + 1; q < t; ++q) s -= Rm[(size_t)q * m + i] * z[q];
        z[i] = s / Rm[(size_t)i * m + i];
    }
    return 0;
}

/* r = y - sum_q a_{S_q} x_q  (Eq. 2's residual with the sign flipped) */
static void residual(const double* A, int m, int lda, const int32_t* S, int t,
                     const double* x, const double* y, double* r) {
    for (int i = 0; i < m; ++i) r[i] = y[i];
    for (int q = 0; q < t; ++q) {
        const double* a = A + (size_t)S[q] * lda;
        for (int i = 0; i < m; ++i) r[i] -= a[i] * x[q];
    }
}

/*
 * Residual injection + selection: c = A^T r over all n atoms, then the
 * position of the largest |c_j| among j not in S (lowest index on ties).
 * Writes |c| of the best and of the runner-up (or -1 if there is none).
 */
static int select_atom(const double* A, int m, int n, int lda, const double* r,
                       const unsigned char* inS, double* top1, double* top2) {
    int best = -1;
    double b1 = -1.0, b2 = -1.0;
    for (int j = 0; j < n; ++j) {
        if (inS[j]) continue;
        double a = fabs(dot(A + (size_t)j * lda, r, m));
        if (a > b1) { b2 = b1; b1 = a; best = j; }
        else if (a > b2) { b2 = a; }
    }
    *top1 = b1;
    *top2 = b2;
    return best;
}

/*
 * Threshold selection: every j not in S with |c_j| >= th * M, M = the largest
 * |c_j| over j not in S; largest |c| first (lowest index on exact ties); at
 * most `room` of them.  Returns the count (0: no atom left).  *margin is the
 * smallest relative gap (over M) that decides the chosen set and its order:
 * chosen atoms above the threshold, the others below it (or below the last
 * chosen one when `room` cuts the list), and consecutive chosen atoms.
 */
static int select_atoms_th(const double* A, int m, int n, int lda, const double* r,
                           const unsigned char* inS, double th, int room, int32_t* out,
                           double* margin) {
    double* c = (double*)malloc(sizeof(double) * n);
    int* idx = (int*)malloc(sizeof(int) * n);
    double M = -1.0;
    int cnt = 0;
    for (int j = 0; j < n; ++j) {
        c[j] = inS[j] ? -1.0 : fabs(dot(A + (size_t)j * lda, r, m));
        if (c[j] > M) M = c[j];
    }
    *margin = INFINITY;
    if (M < 0.0) { free(c); free(idx); return 0; }
    if (M == 0.0) *margin = 0.0;                  /* r = 0: every remaining atom ties */
    const double thr = th * M;
    for (int j = 0; j < n; ++j)
        if (!inS[j] && c[j] >= thr) idx[cnt++] = j;
    /* insertion sort by (|c| descending, index ascending) */
    for (int a = 1; a < cnt; ++a) {
        int v = idx[a], b = a - 1;
        while (b >= 0 && (c[idx[b]] < c[v] || (c[idx[b]] == c[v] && idx[b] > v))) {
            idx[b + 1] = idx[b];
            --b;
        }
        idx[b + 1] = v;
    }
    const int take = cnt < room ? cnt : room;
    for (int a = 0; a < take; ++a) out[a] = idx[a];
    const double lowest = c[idx[take - 1]];
    for (int a = 0; a < take; ++a) {
        if (M == 0.0) break;
        double g = (c[idx[a]] - thr) / M;
        if (g < *margin) *margin = g;
        if (a + 1 < take && (c[idx[a]] - c[idx[a + 1]]) / M < *margin) *margin = (c[idx[a]] - c[idx[a + 1]]) / M;
    }
    for (int j = 0; j < n && M > 0.0; ++j) {
        if (inS[j]) continue;
        int chosen = 0;
        for (int a = 0; a < take; ++a) if (idx[a] == j) { chosen = 1; break; }
        if (chosen) continue;
        /* not chosen: below the threshold, or cut by `room` below the last chosen */
        double g = (c[j] < thr) ? (thr - c[j]) / M : (lowest - c[j]) / M;
        if (g < *margin) *margin = g;
    }
    free(c);
    free(idx);
    return take;
}

/*
 * Incremental QR of A_S for large supports: Q (m x t, orthonormal columns)
 * and R (t x t upper triangular, column-major with leading dimension kmax)
 * gain column t from atom a.  Modified Gram-Schmidt against q_0..q_{t-1},
 * run twice (the second pass removes what rounding left of the first), then
 * R_tt = ||v|| and q_t = v / R_tt.  Returns 0, or 3 when the atom is
 * dependent (R_tt^2 <= 1e-12 ||a||^2, the Householder path's rule).
 */
static int iqr_append(double* Q, double* Rm, int kmax, int m, int t, const double* a) {
    double* v = Q + (size_t)t * m;
    memcpy(v, a, sizeof(double) * m);
    double* rc = Rm + (size_t)t * kmax;
    for (int q = 0; q <= t; ++q) rc[q] = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
        for (int q = 0; q < t; ++q) {
            const double* qq = Q + (size_t)q * m;
            double h = dot(qq, v, m);
            for (int i = 0; i < m; ++i) v[i] -= h * qq[i];
            rc[q] += h;
        }
    }
    double anorm = nrm2(a, m), vn = nrm2(v, m);
    if (vn * vn <= 1e-12 * anorm * anorm) return ST_DEP;
    rc[t] = vn;
    for (int i = 0; i < m; ++i) v[i] /= vn;
    return 0;
}

/* Correlation + selection of select_atom with the atoms split over threads
 * (used for a single large signal); the argmax is taken afterwards in atom
 * order, so ties still go to the lowest index. */
static int select_atom_par(const double* A, int m, int n, int lda, const double* r,
                           const unsigned char* inS, double* c, double* top1, double* top2) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int j = 0; j < n; ++j) c[j] = inS[j] ? -1.0 : fabs(dot(A + (size_t)j * lda, r, m));
    int best = -1;
    double b1 = -1.0, b2 = -1.0;
    for (int j = 0; j < n; ++j) {
        if (inS[j]) continue;
        double a = c[j];
        if (a > b1) { b2 = b1; b1 = a; best = j; }
        else if (a > b2) { b2 = a; }
    }
    *top1 = b1;
    *top2 = b2;
    return best;
}

static int all_finite(const double* y, int m) {
    for (int i = 0; i < m; ++i) if (!isfinite(y[i])) return 0;
    return 1;
}

/* OMP with the incremental QR (iqr_append), for supports too large to
 * refactorise every iteration; same selection, stopping rules and outputs as
 * omp_one.  par != 0 splits the correlation over threads. */
static void omp_one_iqr(const double* A, int m, int n, int lda, const double* y, int k,
                        double tol, int max_iter, int par, int32_t* support, double* coef,
                        int32_t* n_iter, double* res_norm, int32_t* status,
                        double* top1, double* top2, double* res_hist) {
    for (int q = 0; q < k; ++q) { support[q] = -1; coef[q] = 0.0; top1[q] = -1.0; top2[q] = -1.0; res_hist[q] = NAN; }
    if (!all_finite(y, m)) { *n_iter = 0; *res_norm = NAN; *status = ST_NONFINITE; return; }
    double* r = (double*)malloc(sizeof(double) * m);
    double* Q = (double*)malloc(sizeof(double) * (size_t)m * k);
    double* Rm = (double*)malloc(sizeof(double) * (size_t)k * k);
    double* qty = (double*)malloc(sizeof(double) * k);
    double* z = (double*)malloc(sizeof(double) * k);
    double* c = par ? (double*)malloc(sizeof(double) * n) : NULL;
    unsigned char* inS = (unsigned char*)calloc(n, 1);
    memcpy(r, y, sizeof(double) * m);
    double rho = nrm2(r, m);
    int iters = k < max_iter ? k : max_iter;
    int t = 0, st = -1;
    if (rho <= tol) st = ST_TOL;
    while (st < 0 && t < iters) {
        int j = par ? select_atom_par(A, m, n, lda, r, inS, c, &top1[t], &top2[t])
                    : select_atom(A, m, n, lda, r, inS, &top1[t], &top2[t]);
        if (j < 0) { st = ST_MAXIT; break; }
        if (iqr_append(Q, Rm, k, m, t, A + (size_t)j * lda) != 0) { st = ST_DEP; top1[t] = top2[t] = -1.0; break; }
        qty[t] = dot(Q + (size_t)t * m, y, m);
        support[t] = j;
        inS[j] = 1;
        ++t;
        /* back substitution R z = Q^T y */
        for (int i = t - 1; i >= 0; --i) {
            double sacc = qty[i];
            for (int q = i + 1; q < t; ++q) sacc -= Rm[(size_t)q * k + i] * z[q];
            z[i] = sacc / Rm[(size_t)i * k + i];
        }
        for (int q = 0; q < t; ++q) coef[q] = z[q];
        residual(A, m, lda, support, t, coef, y, r);
        rho = nrm2(r, m);
        res_hist[t - 1] = rho;
        if (rho <= tol) st = ST_TOL;
    }
    if (st < 0) st = (t == k) ? ST_K : ST_MAXIT;
    *n_iter = t;
    *res_norm = rho;
    *status = st;
    free(r); free(Q); free(Rm); free(qty); free(z); free(c); free(inS);
}

static void omp_one(const double* A, int m, int n, int lda, const double* y, int k,
                    double tol, int max_iter, int32_t* support, double* coef,
                    int32_t* n_iter, double* res_norm, int32_t* status,
                    double* top1, double* top2, double* res_hist) {
    for (int q = 0; q < k; ++q) { support[q] = -1; coef[q] = 0.0; top1[q] = -1.0; top2[q] = -1.0; res_hist[q] = NAN; }
    if (!all_finite(y, m)) { *n_iter = 0; *res_norm = NAN; *status = ST_NONFINITE; return; }
    double* r = (double*)malloc(sizeof(double) * m);
    double* As = (double*)malloc(sizeof(double) * (size_t)m * k);
    double* z = (double*)malloc(sizeof(double) * k);
    double* work = (double*)malloc(sizeof(double) * ((size_t)m * k + m));
    unsigned char* inS = (unsigned char*)calloc(n, 1);
    memcpy(r, y, sizeof(double) * m);
    double rho = nrm2(r, m);
    int iters = k < max_iter ? k : max_iter;
    int t = 0, st = -1;
    if (rho <= tol) st = ST_TOL;
    while (st < 0 && t < iters) {
        int j = select_atom(A, m, n, lda, r, inS, &top1[t], &top2[t]);
        if (j < 0) { st = ST_MAXIT; break; }
        memcpy(As + (size_t)t * m, A + (size_t)j * lda, sizeof(double) * m);
        if (cs_oracle_lstsq(m, t + 1, As, m, y, z, work) != 0) { st = ST_DEP; top1[t] = top2[t] = -1.0; break; }
        support[t] = j;
        inS[j] = 1;
        ++t;
        for (int q = 0; q < t; ++q) coef[q] = z[q];
        residual(A, m, lda, support, t, coef, y, r);
        rho = nrm2(r, m);
        res_hist[t - 1] = rho;
        if (rho <= tol) st = ST_TOL;
    }
    if (st < 0) st = (t == k) ? ST_K : ST_MAXIT;
    *n_iter = t;
    *res_norm = rho;
    *status = st;
    free(r); free(As); free(z); free(work); free(inS);
}

/*
 * Loss and gradient of the CL s-forward branch restricted to the support:
 *   r = y - A (s .* Mask),  L = 1/2 ||r||^2,  grad_q = -(a_{S_q})^T r.
 * (Unmasked coordinates have zero gradient because of the mask.)
 */
void cs_oracle_clfit_loss_grad(const double* A, int m, int lda, const int32_t* S, int t,
                               const double* s_S, const double* y, double* loss,
                               double* grad_S, double* r_out) {
    double* r = r_out ? r_out : (double*)malloc(sizeof(double) * m);
    residual(A, m, lda, S, t, s_S, y, r);
    if (loss) *loss = 0.5 * dot(r, r, m);
    if (grad_S)
        for (int q = 0; q < t; ++q) grad_S[q] = -dot(A + (size_t)S[q] * lda, r, m);
    if (!r_out) free(r);
}

/*
 * Total-variation prior of a 1-D signal (Eq. 5) on x = D s, restricted to the
 * support: x = sum_q s_q D[:, S_q] (length N; D = NULL means x = s, N = the
 * number of atoms), TV(x) = (1/N) sum_{j < N-1} (x_j - x_{j+1})^2.  Returns
 * w * TV and adds w * dTV/ds_S to grad_S:
 *   dTV/dx_j = (2/N) (d_j - d_{j-1}),  d_j = x_j - x_{j+1}  (d_{-1} = d_{N-1} = 0),
 *   dTV/ds_q = sum_j D[j, S_q] dTV/dx_j.
 */
double cs_oracle_tv_loss_grad(const double* D, int N, int ldd, const int32_t* S, int t,
                              const double* s_S, double w, double* grad_S) {
    if (w == 0.0 || N < 2) return 0.0;
    double* x = (double*)calloc(N, sizeof(double));
    double* gx = (double*)calloc(N, sizeof(double));
    for (int q = 0; q < t; ++q) {
        if (D) {
            const double* dq = D + (size_t)S[q] * ldd;
            for (int j = 0; j < N; ++j) x[j] += s_S[q] * dq[j];
        } else {
            x[S[q]] += s_S[q];
        }
    }
    double tv = 0.0;
    for (int j = 0; j + 1 < N; ++j) {
        const double d = x[j] - x[j + 1];
        tv += d * d;
        gx[j] += 2.0 * d / N;
        gx[j + 1] -= 2.0 * d / N;
    }
    tv /= N;
    if (grad_S)
        for (int q = 0; q < t; ++q) {
            double g = 0.0;
            if (D) {
                const double* dq = D + (size_t)S[q] * ldd;
                for (int j = 0; j < N; ++j) g += dq[j] * gx[j];
            } else {
                g = gx[S[q]];
            }
            grad_S[q] += w * g;
        }
    free(x);
    free(gx);
    return w * tv;
}

/*
 * `steps` Adam steps on L(s_S) = 1/2 ||y - A_S s_S||^2 (the CL coefficient
 * fit), plus tv_w * TV(D_S s_S) when tv_w != 0 (the prior loss of Eq. 5).
 * mom, vel and *tau carry the optimizer state between calls.  Coordinates
 * outside the mask are not touched: their gradient is zero, so their
 * moments stay at zero and their Adam step is exactly zero.
 */
void cs_oracle_clfit_adam_tv(const double* A, int m, int lda, const int32_t* S, int t,
                             const double* y, double* s_S, double* mom, double* vel,
                             int32_t* tau, int steps, double lr, double beta1,
                             double beta2, double eps, double tv_w, const double* D, int N,
                             int ldd) {
    double* r = (double*)malloc(sizeof(double) * m);
    double* g = (double*)malloc(sizeof(double) * (t > 0 ? t : 1));
    for (int it = 0; it < steps; ++it) {
        cs_oracle_clfit_loss_grad(A, m, lda, S, t, s_S, y, NULL, g, r);
        cs_oracle_tv_loss_grad(D, N, ldd, S, t, s_S, tv_w, g);
        *tau += 1;
        double bc1 = 1.0 - pow(beta1, (double)*tau);
        double bc2 = 1.0 - pow(beta2, (double)*tau);
        for (int q = 0; q < t; ++q) {
            mom[q] = beta1 * mom[q] + (1.0 - beta1) * g[q];
            vel[q] = beta2 * vel[q] + (1.0 - beta2) * g[q] * g[q];
            double mhat = mom[q] / bc1;
            double vhat = vel[q] / bc2;
            s_S[q] -= lr * mhat / (sqrt(vhat) + eps);
        }
    }
    free(r); free(g);
}

void cs_oracle_clfit_adam(const double* A, int m, int lda, const int32_t* S, int t,
                          const double* y, double* s_S, double* mom, double* vel,
                          int32_t* tau, int steps, double lr, double beta1,
                          double beta2, double eps) {
    cs_oracle_clfit_adam_tv(A, m, lda, S, t, y, s_S, mom, vel, tau, steps, lr, beta1, beta2, eps,
                            0.0, NULL, 0, 0);
}

/* CLOMP on one signal.  par != 0 splits the correlation of the argmax rule
 * over threads (select_atom_par: same values, same tie rule). */
static void clomp_one(const double* A, int m, int n, int lda, const double* y, int k,
                      double tol, int max_iter, int steps, double lr, double beta1,
                      double beta2, double eps, int reset_adam, double th, double tv_w,
                      const double* D, int N, int ldd, int par, int32_t* support,
                      double* coef, int32_t* n_iter, double* res_norm, int32_t* status,
                      double* top1, double* top2, double* res_hist) {
    for (int q = 0; q < k; ++q) { support[q] = -1; coef[q] = 0.0; top1[q] = -1.0; top2[q] = -1.0; res_hist[q] = NAN; }
    if (!all_finite(y, m)) { *n_iter = 0; *res_norm = NAN; *status = ST_NONFINITE; return; }
    double* r = (double*)malloc(sizeof(double) * m);
    double* mom = (double*)calloc(k, sizeof(double));
    double* vel = (double*)calloc(k, sizeof(double));
    unsigned char* inS = (unsigned char*)calloc(n, 1);
    double* cpar = par ? (double*)malloc(sizeof(double) * n) : NULL;
    int32_t tau = 0;
    memcpy(r, y, sizeof(double) * m);              /* s = 0  =>  r = y */
    double rho = nrm2(r, m);
    int iters = k < max_iter ? k : max_iter;
    int t = 0, st = -1, it = 0;
    const int multi = th > 0.0 && th < 1.0;
    if (rho <= tol) st = ST_TOL;
    while (st < 0 && t < k && it < iters) {
        if (!multi) {
            int j = cpar ? select_atom_par(A, m, n, lda, r, inS, cpar, &top1[t], &top2[t])
                         : select_atom(A, m, n, lda, r, inS, &top1[t], &top2[t]);
            if (j < 0) { st = ST_MAXIT; break; }
            support[t] = j;                       /* Mask |= e_j (bitwise or) */
            inS[j] = 1;
            coef[t] = 0.0;
            ++t;
        } else {
            double margin;
            int cnt = select_atoms_th(A, m, n, lda, r, inS, th, k - t, support + t, &margin);
            if (cnt == 0) { st = ST_MAXIT; break; }
            for (int a = 0; a < cnt; ++a) {
                inS[support[t + a]] = 1;
                coef[t + a] = 0.0;
                top1[t + a] = 1.0;                /* parity rule reads (top1 - top2) / top1 */
                top2[t + a] = 1.0 - margin;
            }
            t += cnt;
        }
        ++it;
        if (reset_adam) {
            memset(mom, 0, sizeof(double) * k);
            memset(vel, 0, sizeof(double) * k);
            tau = 0;
        }
        cs_oracle_clfit_adam_tv(A, m, lda, support, t, y, coef, mom, vel, &tau, steps,
                                lr, beta1, beta2, eps, tv_w, D, N, ldd);
        residual(A, m, lda, support, t, coef, y, r);
        rho = nrm2(r, m);
        res_hist[t - 1] = rho;
        if (rho <= tol) st = ST_TOL;
    }
    if (st < 0) st = (t == k) ? ST_K : ST_MAXIT;
    *n_iter = t;
    *res_norm = rho;
    *status = st;
    free(r); free(mom); free(vel); free(inS); free(cpar);
}

static int bad_args(const double* A, int m, int n, int lda, const double* Y, int ldy,
                    int B, int k) {
    if (m <= 0 || n <= 0 || B < 0 || k <= 0 || k > n || k > m) return 1;
    if (lda < m || ldy < m) return 1;
    if (!A || (B > 0 && !Y)) return 1;
    return 0;
}

/* method: 0 chooses by size (the incremental QR when the refactorisations
 * would cost m k^3 / 3 > 1e9 flops in all, else the
 * Householder QR recomputed each iteration), 1 forces the Householder QR,
 * 2 the incremental QR.  A single signal (B = 1) correlates with the atoms
 * split over the threads; larger batches split the signals. */
int cs_oracle_omp_method(const double* A, int m, int n, int lda, const double* Y, int ldy, int B,
                         int k, double tol, int max_iter, int method, int32_t* support, double* coef,
                         int32_t* n_iter, double* res_norm, int32_t* status, double* top1,
                         double* top2, double* res_hist, int nthreads) {
    if (bad_args(A, m, n, lda, Y, ldy, B, k) || max_iter <= 0 || method < 0 || method > 2) return -1;
    const int iqr = method == 2 || (method == 0 && (double)m * (double)k * (double)k * (double)k / 3.0 > 1e9);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4) if (B > 1)
#endif
    for (int b = 0; b < B; ++b) {
        size_t o = (size_t)b * k;
        if (iqr)
            omp_one_iqr(A, m, n, lda, Y + (size_t)b * ldy, k, tol, max_iter, B == 1, support + o, coef + o,
                        n_iter + b, res_norm + b, status + b, top1 + o, top2 + o, res_hist + o);
        else
            omp_one(A, m, n, lda, Y + (size_t)b * ldy, k, tol, max_iter, support + o, coef + o,
                    n_iter + b, res_norm + b, status + b, top1 + o, top2 + o, res_hist + o);
    }
    return 0;
}

int cs_oracle_omp(const double* A, int m, int n, int lda, const double* Y, int ldy, int B,
                  int k, double tol, int max_iter, int32_t* support, double* coef,
                  int32_t* n_iter, double* res_norm, int32_t* status, double* top1,
                  double* top2, double* res_hist, int nthreads) {
    return cs_oracle_omp_method(A, m, n, lda, Y, ldy, B, k, tol, max_iter, 0, support, coef, n_iter,
                                res_norm, status, top1, top2, res_hist, nthreads);
}

/* th: 0 (or >= 1) selects one atom per iteration; 0 < th < 1 selects by the
 * threshold rule (n_iter then counts atoms, not iterations).  tv_w > 0 adds
 * the total-variation prior of Eq. 5 on x = D s to the fit's loss (D: N x n
 * column-major with leading dimension ldd; NULL: x = s, N = n). */
int cs_oracle_clomp(const double* A, int m, int n, int lda, const double* Y, int ldy, int B,
                    int k, double tol, int max_iter, int steps, double lr, double beta1,
                    double beta2, double eps, int reset_adam, double th, double tv_w,
                    const double* D, int N, int ldd, int32_t* support,
                    double* coef, int32_t* n_iter, double* res_norm, int32_t* status,
                    double* top1, double* top2, double* res_hist, int nthreads) {
    if (bad_args(A, m, n, lda, Y, ldy, B, k) || max_iter <= 0 || steps < 0 || !(th >= 0.0)) return -1;
    if (!(tv_w >= 0.0) || (tv_w > 0.0 && D && (N < 2 || ldd < N))) return -1;
    if (!D) N = n;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4) if (B > 1)
#endif
    for (int b = 0; b < B; ++b) {
        size_t o = (size_t)b * k;
        clomp_one(A, m, n, lda, Y + (size_t)b * ldy, k, tol, max_iter, steps, lr, beta1,
                  beta2, eps, reset_adam, th, tv_w, D, N, ldd, B == 1, support + o, coef + o, n_iter + b, res_norm + b,
                  status + b, top1 + o, top2 + o, res_hist + o);
    }
    return 0;
}

/*
 * Horizontal part of the total variation of an image (Eq. 6).  The image has
 * W columns, column j being the signal x_j = D s_j (length N; D = NULL means
 * x_j = s_j placed in a length-n vector, N = n), so I_{i,j} = (x_j)_i and
 *   TV_h = (1/W) sum_i sum_{j < W-1} (I_{i,j} - I_{i,j+1})^2
 *        = (1/W) sum_{j < W-1} ||x_j - x_{j+1}||^2.
 * (The vertical part, (1/H) sum over columns of sum_i (I_{i,j} - I_{i+1,j})^2
 * with H = N, is the per-column 1-D form of Eq. 5: cs_oracle_tv_loss_grad.)
 * Column j's support is S[j*k .. j*k + t[j]) with coefficients s[j*k ..].
 * Returns w * TV_h; when grad is not NULL adds w * dTV_h/ds to it (same
 * layout as s, support entries only):
 *   dTV_h/dx_j = (2/W) ((x_j - x_{j+1}) [j < W-1] + (x_j - x_{j-1}) [j > 0]),
 *   dTV_h/ds_{j,q} = D[:, S_{j,q}]^T dTV_h/dx_j.
 */
double cs_oracle_tv2d_h_loss_grad(const double* D, int N, int ldd, int W, int k,
                                  const int32_t* S, const int32_t* t, const double* s,
                                  double w, double* grad) {
    if (w == 0.0 || W < 2) return 0.0;
    double* x = (double*)calloc((size_t)N * W, sizeof(double));
    double* gx = (double*)calloc((size_t)N * W, sizeof(double));
    for (int j = 0; j < W; ++j) {
        double* xj = x + (size_t)j * N;
        for (int q = 0; q < t[j]; ++q) {
            const int a = S[(size_t)j * k + q];
            const double v = s[(size_t)j * k + q];
            if (D) {
                const double* da = D + (size_t)a * ldd;
                for (int i = 0; i < N; ++i) xj[i] += v * da[i];
            } else {
                xj[a] += v;
            }
        }
    }
    double tv = 0.0;
    for (int j = 0; j + 1 < W; ++j) {
        const double* xa = x + (size_t)j * N;
        const double* xb = x + (size_t)(j + 1) * N;
        double* ga = gx + (size_t)j * N;
        double* gb = gx + (size_t)(j + 1) * N;
        for (int i = 0; i < N; ++i) {
            const double d = xa[i] - xb[i];
            tv += d * d;
            ga[i] += 2.0 * d / W;
            gb[i] -= 2.0 * d / W;
        }
    }
    tv /= W;
    if (grad)
        for (int j = 0; j < W; ++j) {
            const double* gj = gx + (size_t)j * N;
            for (int q = 0; q < t[j]; ++q) {
                const int a = S[(size_t)j * k + q];
                double g = 0.0;
                if (D) {
                    const double* da = D + (size_t)a * ldd;
                    for (int i = 0; i < N; ++i) g += da[i] * gj[i];
                } else {
                    g = gj[a];
                }
                grad[(size_t)j * k + q] += w * g;
            }
        }
    free(x);
    free(gx);
    return w * tv;
}

/*
 * Local variation of an image (Eq. 7): the mean, over the 3 x 3 windows at
 * every placement inside the image (sliding step 1, no padding; B = (N-2) *
 * (W-2) windows), of the standard deviation of the window's nine pixels,
 * taken with the sample normalisation (divide by 9 - 1) and smoothed by eps:
 *   LV = (1/B) sum_b sigma_b,  sigma_b = sqrt(sum_{p in b} (I_p - mu_b)^2 / 8 + eps^2)
 * (eps = 0: the plain deviation).
 * The columns are x_j = D s_j as in cs_oracle_tv2d_h_loss_grad.  Returns
 * w * LV; when grad is not NULL adds w * dLV/ds (support entries only):
 *   dLV/dI_p = (1/B) sum_{b containing p} (I_p - mu_b) / (8 sigma_b),
 * a window with sigma_b = 0 (constant, eps = 0) contributing 0 (the
 * subgradient there), and dLV/ds_{j,q} = D[:, S_{j,q}]^T dLV/dx_j.
 */
double cs_oracle_lv_loss_grad(const double* D, int N, int ldd, int W, int k, const int32_t* S,
                              const int32_t* t, const double* s, double w, double eps, double* grad) {
    if (w == 0.0 || N < 3 || W < 3) return 0.0;
    double* x = (double*)calloc((size_t)N * W, sizeof(double));
    double* gx = (double*)calloc((size_t)N * W, sizeof(double));
    for (int j = 0; j < W; ++j) {
        double* xj = x + (size_t)j * N;
        for (int q = 0; q < t[j]; ++q) {
            const int a = S[(size_t)j * k + q];
            const double v = s[(size_t)j * k + q];
            if (D) {
                const double* da = D + (size_t)a * ldd;
                for (int i = 0; i < N; ++i) xj[i] += v * da[i];
            } else {
                xj[a] += v;
            }
        }
    }
    const double nb = (double)(N - 2) * (double)(W - 2);
    double lv = 0.0;
    for (int c0 = 0; c0 + 2 < W; ++c0)
        for (int r0 = 0; r0 + 2 < N; ++r0) {
            double mu = 0.0;
            for (int dc = 0; dc < 3; ++dc)
                for (int dr = 0; dr < 3; ++dr) mu += x[(size_t)(c0 + dc) * N + r0 + dr];
            mu /= 9.0;
            double ss = 0.0;
            for (int dc = 0; dc < 3; ++dc)
                for (int dr = 0; dr < 3; ++dr) {
                    const double d = x[(size_t)(c0 + dc) * N + r0 + dr] - mu;
                    ss += d * d;
                }
            const double sigma = sqrt(ss / 8.0 + eps * eps);
            lv += sigma;
            if (sigma > 0.0)
                for (int dc = 0; dc < 3; ++dc)
                    for (int dr = 0; dr < 3; ++dr) {
                        const size_t p = (size_t)(c0 + dc) * N + r0 + dr;
                        gx[p] += (x[p] - mu) / (8.0 * sigma) / nb;
                    }
        }
    lv /= nb;
    if (grad)
        for (int j = 0; j < W; ++j) {
            const double* gj = gx + (size_t)j * N;
            for (int q = 0; q < t[j]; ++q) {
                const int a = S[(size_t)j * k + q];
                double g = 0.0;
                if (D) {
                    const double* da = D + (size_t)a * ldd;
                    for (int i = 0; i < N; ++i) g += da[i] * gj[i];
                } else {
                    g = gj[a];
                }
                grad[(size_t)j * k + q] += w * g;
            }
        }
    free(x);
    free(gx);
    return w * lv;
}

/*
 * CLOMP on images with the image priors: the total variation of Eq. 6 and
 * the local variation of Eq. 7.  The batch is a sequence of images of W
 * consecutive columns (B a multiple of W), and the fit's loss of an image is
 *   sum_j 1/2 ||y_j - A (s_j .* Mask_j)||^2 + tv_w TV(I) + lv_w LV(I),
 *   I = [D s_1 ... D s_W],
 * which couples neighbouring columns.  Per iteration every live column
 * selects its atom from its own residual (as in cs_oracle_clomp), then all
 * live columns of the image take the `steps` Adam steps together: every
 * step's gradients come from the coefficients before that step.  A stopped
 * column keeps its coefficients and still enters its neighbours' terms.
 * Outputs, status codes and the remaining readings are those of
 * cs_oracle_clomp (one atom per iteration).
 */
static void clomp_image(const double* A, int m, int n, int lda, const double* Y, int ldy,
                        int W, int k, double tol, int max_iter, int steps, double lr,
                        double beta1, double beta2, double eps, int reset_adam, double tv_w,
                        double lv_w, double lv_eps, const double* D, int N, int ldd, int32_t* support,
                        double* coef, int32_t* n_iter, double* res_norm, int32_t* status, double* top1,
                        double* top2, double* res_hist) {
    double* r = (double*)malloc(sizeof(double) * (size_t)m * W);
    double* mom = (double*)calloc((size_t)k * W, sizeof(double));
    double* vel = (double*)calloc((size_t)k * W, sizeof(double));
    double* g = (double*)calloc((size_t)k * W, sizeof(double));
    double* rg = (double*)malloc(sizeof(double) * m);
    unsigned char* inS = (unsigned char*)calloc((size_t)n * W, 1);
    int32_t* tau = (int32_t*)calloc(W, sizeof(int32_t));
    int32_t* st = (int32_t*)malloc(sizeof(int32_t) * W);
    unsigned char* fit = (unsigned char*)calloc(W, 1);
    double* rho = (double*)malloc(sizeof(double) * W);
    for (int j = 0; j < W; ++j) {
        const double* y = Y + (size_t)j * ldy;
        for (int q = 0; q < k; ++q) {
            size_t o = (size_t)j * k + q;
            support[o] = -1; coef[o] = 0.0; top1[o] = -1.0; top2[o] = -1.0; res_hist[o] = NAN;
        }
        n_iter[j] = 0;
        st[j] = -1;
        if (!all_finite(y, m)) { st[j] = ST_NONFINITE; rho[j] = NAN; continue; }
        memcpy(r + (size_t)j * m, y, sizeof(double) * m);          /* s = 0  =>  r = y */
        rho[j] = nrm2(y, m);
        if (rho[j] <= tol) st[j] = ST_TOL;
    }
    const int iters = k < max_iter ? k : max_iter;
    for (int it = 0; it < iters; ++it) {
        int any = 0;
        for (int j = 0; j < W; ++j) {
            fit[j] = 0;
            if (st[j] >= 0) continue;
            const size_t o = (size_t)j * k;
            const int t = n_iter[j];
            const int a = select_atom(A, m, n, lda, r + (size_t)j * m, inS + (size_t)j * n,
                                      &top1[o + t], &top2[o + t]);
            if (a < 0) { st[j] = ST_MAXIT; continue; }
            support[o + t] = a;                    /* Mask |= e_a */
            inS[(size_t)j * n + a] = 1;
            coef[o + t] = 0.0;
            n_iter[j] = t + 1;
            fit[j] = 1;
            any = 1;
            if (reset_adam) {
                memset(mom + o, 0, sizeof(double) * k);
                memset(vel + o, 0, sizeof(double) * k);
                tau[j] = 0;
            }
        }
        if (!any) break;
        for (int step = 0; step < steps; ++step) {
            /* every gradient of this step from the coefficients before it */
            for (int j = 0; j < W; ++j) {
                const size_t o = (size_t)j * k;
                const int t = n_iter[j];
                for (int q = 0; q < k; ++q) g[o + q] = 0.0;
                if (!fit[j]) continue;
                cs_oracle_clfit_loss_grad(A, m, lda, support + o, t, coef + o, Y + (size_t)j * ldy,
                                          NULL, g + o, rg);
                cs_oracle_tv_loss_grad(D, N, ldd, support + o, t, coef + o, tv_w, g + o);
            }
            cs_oracle_tv2d_h_loss_grad(D, N, ldd, W, k, support, n_iter, coef, tv_w, g);
            cs_oracle_lv_loss_grad(D, N, ldd, W, k, support, n_iter, coef, lv_w, lv_eps, g);
            for (int j = 0; j < W; ++j) {
                if (!fit[j]) continue;
                const size_t o = (size_t)j * k;
                tau[j] += 1;
                const double bc1 = 1.0 - pow(beta1, (double)tau[j]);
                const double bc2 = 1.0 - pow(beta2, (double)tau[j]);
                for (int q = 0; q < n_iter[j]; ++q) {
                    mom[o + q] = beta1 * mom[o + q] + (1.0 - beta1) * g[o + q];
                    vel[o + q] = beta2 * vel[o + q] + (1.0 - beta2) * g[o + q] * g[o + q];
                    const double mhat = mom[o + q] / bc1;
                    const double vhat = vel[o + q] / bc2;
                    coef[o + q] -= lr * mhat / (sqrt(vhat) + eps);
                }
            }
        }
        for (int j = 0; j < W; ++j) {
            if (!fit[j]) continue;
            const size_t o = (size_t)j * k;
            const int t = n_iter[j];
            residual(A, m, lda, support + o, t, coef + o, Y + (size_t)j * ldy, r + (size_t)j * m);
            rho[j] = nrm2(r + (size_t)j * m, m);
            res_hist[o + t - 1] = rho[j];
            if (rho[j] <= tol) st[j] = ST_TOL;
            else if (t == k) st[j] = ST_K;
        }
    }
    for (int j = 0; j < W; ++j) {
        if (st[j] < 0) st[j] = (n_iter[j] == k) ? ST_K : ST_MAXIT;
        status[j] = st[j];
        res_norm[j] = rho[j];
    }
    free(r); free(mom); free(vel); free(g); free(rg); free(inS); free(tau); free(st); free(fit); free(rho);
}

/* The batch as B / W images of W columns each (see clomp_image); the priors'
 * weights tv_w, lv_w >= 0, the deviation's smoothing lv_eps >= 0 (see
 * cs_oracle_lv_loss_grad), D as in cs_oracle_clomp. */
int cs_oracle_clomp_image(const double* A, int m, int n, int lda, const double* Y, int ldy, int B,
                          int W, int k, double tol, int max_iter, int steps, double lr, double beta1,
                          double beta2, double eps, int reset_adam, double tv_w, double lv_w,
                          double lv_eps, const double* D,
                         int N, int ldd, int32_t* support, double* coef, int32_t* n_iter,
                         double* res_norm, int32_t* status, double* top1, double* top2,
                         double* res_hist, int nthreads) {
    if (bad_args(A, m, n, lda, Y, ldy, B, k) || max_iter <= 0 || steps < 0) return -1;
    if (W < 1 || B % W != 0 || !(tv_w >= 0.0) || !(lv_w >= 0.0) || !(lv_eps >= 0.0) ||
        (D && (N < 2 || ldd < N)))
        return -1;
    if (!D) N = n;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int g = 0; g < B / W; ++g) {
        const size_t b0 = (size_t)g * W, o = b0 * k;
        clomp_image(A, m, n, lda, Y + b0 * ldy, ldy, W, k, tol, max_iter, steps, lr, beta1,
                    beta2, eps, reset_adam, tv_w, lv_w, lv_eps, D, N, ldd, support + o, coef + o, n_iter + b0,
                    res_norm + b0, status + b0, top1 + o, top2 + o, res_hist + o);
    }
    return 0;
}

/*
 * IHT (Methods, Table "s forward block", IHT row): s <- H_k(s + t A^T r)
 * with r = y - A s, where H_k keeps the k entries of largest magnitude
 * (lowest index on exact ties) and zeroes the others, and t is the caller's
 * scale factor.  s starts at zero.  Before the first iteration and after each
 * one: stop with status 1 once ||r||_2 <= tol, else with status 2 after
 * max_iter iterations (R).  Outputs: the k kept indices in ascending order
 * and their values, the iterations run, ||r||_2, the status, and margin =
 * the smallest relative gap (|u|_(k) - |u|_(k+1)) / |u|_(k) between the k-th
 * and (k+1)-th largest |u| over the iterations (the float64 resolution of
 * the kept set; 1 when k = n).
 */
static void iht_one(const double* A, int m, int n, int lda, const double* y, int k, double t,
                    double tol, int max_iter, int32_t* support, double* coef, int32_t* n_iter,
                    double* res_norm, int32_t* status, double* margin) {
    for (int q = 0; q < k; ++q) { support[q] = -1; coef[q] = 0.0; }
    *margin = 1.0;
    if (!all_finite(y, m)) { *n_iter = 0; *res_norm = NAN; *status = ST_NONFINITE; return; }
    double* s = (double*)calloc(n, sizeof(double));
    double* u = (double*)malloc(sizeof(double) * n);
    double* r = (double*)malloc(sizeof(double) * m);
    int* idx = (int*)malloc(sizeof(int) * n);
    memcpy(r, y, sizeof(double) * m);
    double rho = nrm2(r, m);
    int it = 0, st = -1;
    if (rho <= tol) st = ST_TOL;
    while (st < 0 && it < max_iter) {
        for (int j = 0; j < n; ++j) u[j] = s[j] + t * dot(A + (size_t)j * lda, r, m);
        /* order the indices by |u| descending, index ascending (insertion sort
           into the first k + 1 places is enough for H_k and the margin) */
        int top = k + 1 < n ? k + 1 : n, cnt = 0;
        for (int j = 0; j < n; ++j) {
            double a = fabs(u[j]);
            int pos = cnt;
            while (pos > 0 && fabs(u[idx[pos - 1]]) < a) --pos;   /* equal: the earlier index stays first */
            if (pos >= top) continue;
            int last = cnt < top ? cnt : top - 1;
            for (int q = last; q > pos; --q) idx[q] = idx[q - 1];
            idx[pos] = j;
            if (cnt < top) ++cnt;
        }
        if (k < n) {
            double a1 = fabs(u[idx[k - 1]]), a2 = fabs(u[idx[k]]);
            double g = a1 > 0.0 ? (a1 - a2) / a1 : 0.0;
            if (g < *margin) *margin = g;
        }
        for (int j = 0; j < n; ++j) s[j] = 0.0;
        for (int q = 0; q < k; ++q) s[idx[q]] = u[idx[q]];
        memcpy(r, y, sizeof(double) * m);
        for (int j = 0; j < n; ++j) {
            if (s[j] == 0.0) continue;
            const double* a = A + (size_t)j * lda;
            for (int i = 0; i < m; ++i) r[i] -= a[i] * s[j];
        }
        rho = nrm2(r, m);
        ++it;
        if (rho <= tol) st = ST_TOL;
    }
    if (st < 0) st = ST_MAXIT;
    /* the kept set in ascending index order (the last H_k's k indices) */
    if (it > 0) {
        int q = 0;
        for (int j = 0; j < n && q < k; ++j) {
            int kept = 0;
            for (int p = 0; p < k; ++p) if (idx[p] == j) { kept = 1; break; }
            if (kept) { support[q] = j; coef[q] = s[j]; ++q; }
        }
    }
    *n_iter = it;
    *res_norm = rho;
    *status = st;
    free(s); free(u); free(r); free(idx);
}

int cs_oracle_iht(const double* A, int m, int n, int lda, const double* Y, int ldy, int B, int k,
                  double t, double tol, int max_iter, int32_t* support, double* coef, int32_t* n_iter,
                  double* res_norm, int32_t* status, double* margin, int nthreads) {
    if (m <= 0 || n <= 0 || B < 0 || k <= 0 || k > n || lda < m || ldy < m || !A || (B > 0 && !Y)) return -1;
    if (max_iter <= 0 || !(t > 0.0)) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (int b = 0; b < B; ++b) {
        size_t o = (size_t)b * k;
        iht_one(A, m, n, lda, Y + (size_t)b * ldy, k, t, tol, max_iter, support + o, coef + o, n_iter + b,
                res_norm + b, status + b, margin + b);
    }
    return 0;
}

int cs_oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
