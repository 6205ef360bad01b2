/*
 * gp_oracle.c -- plain, slow, obviously correct FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check in
 * __graft_entry__.py and the CPU-baseline leg of bench.py may load this
 * library.  It shares no code, header, table or constant with the CUDA
 * library in paper_2605_13209_b300/, and the CUDA library never calls it.
 *
 * What it computes (Thuering, Strack, Pflueger, "Comparing the Performance of
 * Heterogeneous Conjugate Gradient and Cholesky Solvers on Various Hardware
 * Using SYCL"):
 *   - the squared-exponential GP kernel matrix the solvers are applied to
 *     (Sec. 4.1 uses GP covariance matrices; the SE form and its
 *     hyper-parameters are the synthetic stand-in for the paper's dataset);
 *   - the Cholesky factor L with L L^T = A, L lower triangular with a positive
 *     diagonal (Sec. 2.2), by the textbook unblocked algorithm;
 *   - the blocked right-looking Cholesky of Algorithm 1 (right), steps 1-3 in
 *     the paper's order, as a second statement of the same factor;
 *   - forward and back substitution L y = b, L^T x = y (Sec. 2.2);
 *   - classic CG exactly as Algorithm 1 (left), with the residual recomputed
 *     from scratch every R iterations (Sec. 2.1);
 *   - preconditioned CG with M = Lt Lt^T (standard PCG; the paper names mixed
 *     precision only as future work, Sec. 5), used to state the refined solve;
 *   - an emulation of the low-precision factor (Algorithm 1 with the step-3
 *     operands rounded to bfloat16, or split into two bfloat16 parts);
 *   - the error measures: backward error, relative factor error, forward error.
 *
 * All matrices are column-major with a leading dimension; only the lower
 * triangle of A and L is referenced unless stated otherwise.
 *
 * Parity status: every function here is pinned by tests/test_oracle_*.py
 * against closed forms, brute force or library routines; none is unpinned.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define IDX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

/* ------------------------------------------------------------------------ */
/* Squared-exponential kernel matrix                                          */
/* ------------------------------------------------------------------------ */

/* K_ij = sf2 * exp(-||x_i - x_j||^2 / (2 ell^2)) + sn2 * delta_ij.
 * X is n x d row-major (point i at X + i*d).  The squared distance is summed
 * term by term, so the diagonal is exactly sf2 + sn2 and K is exactly
 * symmetric.  Fills the full n x n matrix. */
void or_se_matrix(int64_t n, int d, const double *X, double sf2, double ell,
                  double sn2, double *A, int64_t lda)
{
    double inv2l2 = 1.0 / (2.0 * ell * ell);
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t i = 0; i < n; ++i) {
            double d2 = 0.0;
            for (int k = 0; k < d; ++k) {
                double diff = X[i * d + k] - X[j * d + k];
                d2 += diff * diff;
            }
            double v = sf2 * exp(-d2 * inv2l2);
            if (i == j) v += sn2;
            A[IDX(i, j, lda)] = v;
        }
    }
}

/* One entry of the same matrix, for sampled checks at sizes where the full
 * matrix is not formed on the host. */
double or_se_entry(int d, const double *xi, const double *xj, int same,
                   double sf2, double ell, double sn2)
{
    double d2 = 0.0;
    for (int k = 0; k < d; ++k) {
        double diff = xi[k] - xj[k];
        d2 += diff * diff;
    }
    double v = sf2 * exp(-d2 / (2.0 * ell * ell));
    if (same) v += sn2;
    return v;
}

/* ------------------------------------------------------------------------ */
/* Cholesky factor                                                            */
/* ------------------------------------------------------------------------ */

/* Textbook unblocked Cholesky (outer-product form), in place on the lower
 * triangle: for each column j, l_jj = sqrt(a_jj), l_ij = a_ij / l_jj, then the
 * remaining lower triangle loses the rank-1 term l_ij l_kj.  The strict upper
 * triangle is not touched.  Returns 0, or j+1 if the pivot of column j is not
 * positive (or not finite), LAPACK's info convention. */
int64_t or_cholesky(int64_t n, double *A, int64_t lda)
{
    for (int64_t j = 0; j < n; ++j) {
        double ajj = A[IDX(j, j, lda)];
        if (!(ajj > 0.0) || !isfinite(ajj)) return j + 1;
        double ljj = sqrt(ajj);
        A[IDX(j, j, lda)] = ljj;
        for (int64_t i = j + 1; i < n; ++i) A[IDX(i, j, lda)] /= ljj;
        for (int64_t k = j + 1; k < n; ++k) {
            double lkj = A[IDX(k, j, lda)];
            for (int64_t i = k; i < n; ++i)
                A[IDX(i, k, lda)] -= A[IDX(i, j, lda)] * lkj;
        }
    }
    return 0;
}

/* Algorithm 1 (right): in-place right-looking blocked Cholesky with square
 * blocks of size b (the last block row/column may be smaller).
 *   step 1  A_jj = chol(A_jj)                       (textbook factor above)
 *   step 2  A_ij = A_ij * A_jj^{-T}        for i > j (triangular solve)
 *   step 3  A_ii -= A_ij A_ij^T             for i > j
 *           A_ik -= A_ij A_kj^T      for j < k < i
 * Returns 0 or the 1-based failing global column. */
int64_t or_blocked_cholesky(int64_t n, int64_t b, double *A, int64_t lda)
{
    int64_t N = (n + b - 1) / b;
    for (int64_t J = 0; J < N; ++J) {
        int64_t j0 = J * b, nj = (n - j0 < b) ? n - j0 : b;
        /* step 1 */
        int64_t info = or_cholesky(nj, &A[IDX(j0, j0, lda)], lda);
        if (info) return j0 + info;
        /* step 2: for every block below, X L^T = B, column by column */
        for (int64_t I = J + 1; I < N; ++I) {
            int64_t i0 = I * b, ni = (n - i0 < b) ? n - i0 : b;
            for (int64_t c = 0; c < nj; ++c) {
                double lcc = A[IDX(j0 + c, j0 + c, lda)];
                for (int64_t r = 0; r < ni; ++r) {
                    double s = A[IDX(i0 + r, j0 + c, lda)];
                    for (int64_t k = 0; k < c; ++k)
                        s -= A[IDX(i0 + r, j0 + k, lda)] * A[IDX(j0 + c, j0 + k, lda)];
                    A[IDX(i0 + r, j0 + c, lda)] = s / lcc;
                }
            }
        }
        /* step 3 */
        for (int64_t I = J + 1; I < N; ++I) {
            int64_t i0 = I * b, ni = (n - i0 < b) ? n - i0 : b;
            /* A_II -= A_IJ A_IJ^T (lower part of the diagonal block) */
            for (int64_t c = 0; c < ni; ++c)
                for (int64_t r = c; r < ni; ++r) {
                    double s = 0.0;
                    for (int64_t k = 0; k < nj; ++k)
                        s += A[IDX(i0 + r, j0 + k, lda)] * A[IDX(i0 + c, j0 + k, lda)];
                    A[IDX(i0 + r, i0 + c, lda)] -= s;
                }
            /* A_IK -= A_IJ A_KJ^T for J < K < I */
            for (int64_t K = J + 1; K < I; ++K) {
                int64_t k0 = K * b, nk = (n - k0 < b) ? n - k0 : b;
                for (int64_t c = 0; c < nk; ++c)
                    for (int64_t r = 0; r < ni; ++r) {
                        double s = 0.0;
                        for (int64_t k = 0; k < nj; ++k)
                            s += A[IDX(i0 + r, j0 + k, lda)] * A[IDX(k0 + c, j0 + k, lda)];
                        A[IDX(i0 + r, k0 + c, lda)] -= s;
                    }
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Low-precision factor emulation                                             */
/* ------------------------------------------------------------------------ */

/* Round an IEEE binary32 value to bfloat16 (round to nearest, ties to even),
 * returned widened back to double.  NaN stays NaN. */
static double or_round_bf16_f(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x007fffffu)) return (double)f;
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    u &= 0xffff0000u;
    float r;
    memcpy(&r, &u, 4);
    return (double)r;
}

double or_round_bf16(double x) { return or_round_bf16_f((float)x); }
double or_round_f32(double x) { return (double)(float)x; }

/* IEEE binary16, round to nearest even, from the definition: the spacing of
 * binary16 numbers at |x| is 2^(E - 10) for a leading-bit exponent E >= -14
 * and 2^-24 below (subnormals); |x| >= 65520 overflows to infinity. */
double or_round_f16(double x)
{
    if (x == 0.0 || !isfinite(x)) return x;
    double a = fabs(x);
    if (a >= 65520.0) return x > 0.0 ? INFINITY : -INFINITY;
    int ex;
    frexp(a, &ex);   /* a = m 2^ex, m in [0.5, 1): leading bit 2^(ex - 1) */
    int E = ex - 1;
    if (E < -14) E = -14;
    double q = ldexp(1.0, E - 10);
    double r = rint(a / q) * q;   /* default rounding mode: ties to even */
    return x > 0.0 ? r : -r;
}

/* Power-of-two scale exponent for values bounded by mx: the scaled bound
 * lies in [2^14, 2^15); clamped to [-60, 60]. */
static int or_f16_scale_exp(double mx)
{
    if (!(mx > 0.0)) return 0;
    int ex;
    frexp(mx, &ex);
    int e = 14 - (ex - 1);
    if (e < -60) e = -60;
    if (e > 60) e = 60;
    return e;
}

/* Emulated mixed-precision factor (the preconditioner of the refined solve):
 * Algorithm 1 (right) on a binary32 copy of A where
 *   step 1 factors the diagonal block in FP64 (from the binary32 values),
 *   step 2 solves in FP64 and stores the panel rounded to binary32,
 *   step 3 multiplies operands rounded to bfloat16 (mode 1) or split into a
 *          bfloat16 head plus a bfloat16 tail, keeping head*head + head*tail +
 *          tail*head (mode 2), or, mode 3, split into a binary16 head and
 *          tail after scaling by 2^e, the three products divided by 2^2e;
 *          one e for the whole factor, from the bound |L_ij| <= sqrt(W_ii)
 *          of an SPD W = L L^T: sqrt(max_i W_ii) (rounded to binary32) is
 *          scaled into [2^14, 2^15); the products are summed in FP64 and the
 *          updated block is stored rounded to binary32.
 * mode 0 keeps step 3's operands in binary32.  Lt receives the factor as
 * doubles (lower triangle).  Returns 0 or the 1-based failing column. */
int64_t or_mixed_factor(int64_t n, int64_t b, const double *A, int64_t lda,
                        int mode, double shift, double *Lt, int64_t ldl)
{
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = j; i < n; ++i)
            Lt[IDX(i, j, ldl)] = or_round_f32(A[IDX(i, j, lda)] + (i == j ? shift : 0.0));
    double sc = 1.0;
    if (mode == 3) {
        double dm = 0.0;
        for (int64_t i = 0; i < n; ++i)
            if (Lt[IDX(i, i, ldl)] > dm) dm = Lt[IDX(i, i, ldl)];
        sc = ldexp(1.0, or_f16_scale_exp((double)(float)sqrt(dm)));
    }
    /* Row-major copies of the current panel: Ljj (the diagonal block, row c
     * at Ljj + c*b), and for step 3 every panel entry's head H and tail T as
     * defined by the mode.  They only give the loops unit stride: each value
     * and each summation order is the one of the textbook loops. */
    double *Ljj = malloc(sizeof(double) * (size_t)b * (size_t)b);
    double *row = malloc(sizeof(double) * (size_t)b);
    double *H = malloc(sizeof(double) * (size_t)n * (size_t)b);
    double *T = malloc(sizeof(double) * (size_t)n * (size_t)b);
    int64_t info = 0;
    int64_t N = (n + b - 1) / b;
    for (int64_t J = 0; J < N && !info; ++J) {
        int64_t j0 = J * b, nj = (n - j0 < b) ? n - j0 : b;
        info = or_cholesky(nj, &Lt[IDX(j0, j0, ldl)], ldl);
        if (info) { info += j0; break; }
        for (int64_t c = 0; c < nj; ++c)
            for (int64_t r = c; r < nj; ++r)
                Lt[IDX(j0 + r, j0 + c, ldl)] = or_round_f32(Lt[IDX(j0 + r, j0 + c, ldl)]);
        for (int64_t c = 0; c < nj; ++c)
            for (int64_t k = 0; k <= c; ++k) Ljj[c * b + k] = Lt[IDX(j0 + c, j0 + k, ldl)];
        /* step 2: row i of the panel solves x L_jj^T = a_i, column by column */
        for (int64_t i = j0 + nj; i < n; ++i) {
            for (int64_t c = 0; c < nj; ++c) row[c] = Lt[IDX(i, j0 + c, ldl)];
            for (int64_t c = 0; c < nj; ++c) {
                double s = row[c];
                for (int64_t k = 0; k < c; ++k) s -= row[k] * Ljj[c * b + k];
                row[c] = s / Ljj[c * b + c];
            }
            for (int64_t c = 0; c < nj; ++c) Lt[IDX(i, j0 + c, ldl)] = or_round_f32(row[c]);
        }
        /* the step-3 operands of every panel row */
        for (int64_t i = j0 + nj; i < n; ++i)
            for (int64_t c = 0; c < nj; ++c) {
                double a = Lt[IDX(i, j0 + c, ldl)], *h = &H[(size_t)i * b + c], *t = &T[(size_t)i * b + c];
                if (mode == 1) {
                    *h = or_round_bf16(a);
                    *t = 0.0;
                } else if (mode == 2) {
                    *h = or_round_bf16(a);
                    *t = or_round_bf16(a - *h);
                } else if (mode == 3) {
                    double as = a * sc;
                    *h = or_round_f16(as);
                    *t = or_round_f16(as - *h);
                } else {
                    *h = a;
                    *t = 0.0;
                }
            }
        /* step 3 over the whole trailing lower triangle */
        for (int64_t k = j0 + nj; k < n; ++k) {
            const double *bh_row = &H[(size_t)k * b], *bt_row = &T[(size_t)k * b];
            for (int64_t i = k; i < n; ++i) {
                const double *ah_row = &H[(size_t)i * b], *at_row = &T[(size_t)i * b];
                double s = 0.0;
                if (mode == 2) {
                    for (int64_t c = 0; c < nj; ++c)
                        s += ah_row[c] * bh_row[c] + ah_row[c] * bt_row[c] + at_row[c] * bh_row[c];
                } else if (mode == 3) {
                    for (int64_t c = 0; c < nj; ++c)
                        s += (ah_row[c] * bh_row[c] + ah_row[c] * bt_row[c] + at_row[c] * bh_row[c]) / (sc * sc);
                } else {   /* modes 0 and 1: one product of the (rounded) values */
                    for (int64_t c = 0; c < nj; ++c) s += ah_row[c] * bh_row[c];
                }
                Lt[IDX(i, k, ldl)] = or_round_f32(Lt[IDX(i, k, ldl)] - s);
            }
        }
    }
    free(Ljj); free(row); free(H); free(T);
    return info;
}

/* ------------------------------------------------------------------------ */
/* Substitution                                                               */
/* ------------------------------------------------------------------------ */

/* L Y = B in place (B is n x nrhs, column-major, ldb). */
void or_forward_sub(int64_t n, const double *L, int64_t ldl, double *B,
                    int64_t ldb, int nrhs)
{
    for (int r = 0; r < nrhs; ++r) {
        double *y = B + (size_t)r * ldb;
        for (int64_t i = 0; i < n; ++i) {
            double s = y[i];
            for (int64_t k = 0; k < i; ++k) s -= L[IDX(i, k, ldl)] * y[k];
            y[i] = s / L[IDX(i, i, ldl)];
        }
    }
}

/* L^T X = Y in place (back substitution with the transpose of L). */
void or_back_sub(int64_t n, const double *L, int64_t ldl, double *B,
                 int64_t ldb, int nrhs)
{
    for (int r = 0; r < nrhs; ++r) {
        double *x = B + (size_t)r * ldb;
        for (int64_t i = n - 1; i >= 0; --i) {
            double s = x[i];
            for (int64_t k = i + 1; k < n; ++k) s -= L[IDX(k, i, ldl)] * x[k];
            x[i] = s / L[IDX(i, i, ldl)];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* GP quantities on the factor (the GP behaviour prediction of Sec. 4.1)      */
/* ------------------------------------------------------------------------ */

/* log det A of an SPD matrix from its Cholesky factor: A = L L^T gives
 * det A = prod_i L_ii^2, so log det A = 2 sum_i log L_ii.  The factor is the
 * textbook one above, taken on a private copy of A (lower triangle read).
 * Returns 0 and *out, or the 1-based failing column (then *out is NaN). */
int64_t or_logdet(int64_t n, const double *A, int64_t lda, double *out)
{
    double *L = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * (size_t)(n > 0 ? n : 1));
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = j; i < n; ++i) L[IDX(i, j, n)] = A[IDX(i, j, lda)];
    int64_t info = or_cholesky(n, L, n > 0 ? n : 1);
    double s = 0.0;
    if (info == 0)
        for (int64_t i = 0; i < n; ++i) s += log(L[IDX(i, i, n)]);
    *out = info == 0 ? 2.0 * s : NAN;
    free(L);
    return info;
}

/* GP predictive mean at m test points: mean_k = sum_i k(x*_k, x_i) alpha_i
 * with the noise-free squared-exponential covariance
 * k(x, y) = sf2 exp(-||x - y||^2 / (2 ell^2)) between test and training
 * points (the noise term belongs to the training covariance only) and
 * alpha = (K + sn2 I)^-1 y the solution of the GP system.  Xs: m x d and
 * X: n x d, row-major.  alpha: n x nrhs (lda_alpha), mean: m x nrhs (ldm),
 * column-major. */
void or_predict_mean(int64_t m, int64_t n, int d, const double *Xs, const double *X, double sf2,
                     double ell, const double *alpha, int64_t lda_alpha, int nrhs, double *mean,
                     int64_t ldm)
{
    for (int r = 0; r < nrhs; ++r)
        for (int64_t k = 0; k < m; ++k) {
            double s = 0.0;
            for (int64_t i = 0; i < n; ++i)
                s += or_se_entry(d, Xs + k * d, X + i * d, 0, sf2, ell, 0.0) * alpha[IDX(i, r, lda_alpha)];
            mean[IDX(k, r, ldm)] = s;
        }
}

/* ------------------------------------------------------------------------ */
/* Conjugate gradients                                                        */
/* ------------------------------------------------------------------------ */

/* y = A x with the full n x n matrix A (both triangles stored). */
static void or_matvec_full(int64_t n, const double *A, int64_t lda,
                           const double *x, double *y)
{
    for (int64_t i = 0; i < n; ++i) y[i] = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        double xj = x[j];
        for (int64_t i = 0; i < n; ++i) y[i] += A[IDX(i, j, lda)] * xj;
    }
}

static double or_dot(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Algorithm 1 (left), one right-hand side, full matrix storage:
 *   s = r = b - A x;  u = u0 = r^T r
 *   while u > eps^2 u0:
 *       t = A s;  alpha = u / s^T t;  x += alpha s
 *       r = b - A x   if this is the R-th, 2R-th, ... iteration (R > 0)
 *       r -= alpha t  otherwise
 *       v = u;  u = r^T r;  beta = u / v;  s = r + beta s
 * x holds the start vector on entry.  Stops after maxit iterations at most.
 * Returns the iteration count; *relres_out = sqrt(u / u0) at exit. */
int or_cg(int64_t n, const double *A, int64_t lda, const double *b, double *x,
          double eps, int maxit, int R, double *relres_out)
{
    double *r = malloc(sizeof(double) * n), *s = malloc(sizeof(double) * n);
    double *t = malloc(sizeof(double) * n);
    or_matvec_full(n, A, lda, x, t);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - t[i];
    memcpy(s, r, sizeof(double) * n);
    double u = or_dot(n, r, r), u0 = u;
    int it = 0;
    while (u > eps * eps * u0 && it < maxit) {
        or_matvec_full(n, A, lda, s, t);
        double alpha = u / or_dot(n, s, t);
        for (int64_t i = 0; i < n; ++i) x[i] += alpha * s[i];
        ++it;
        if (R > 0 && it % R == 0) {
            or_matvec_full(n, A, lda, x, r);
            for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
        } else {
            for (int64_t i = 0; i < n; ++i) r[i] -= alpha * t[i];
        }
        double v = u;
        u = or_dot(n, r, r);
        double beta = u / v;
        for (int64_t i = 0; i < n; ++i) s[i] = r[i] + beta * s[i];
    }
    if (relres_out) *relres_out = (u0 > 0.0) ? sqrt(u / u0) : 0.0;
    free(r); free(s); free(t);
    return it;
}

/* Single-reduction CG (Chronopoulos and Gear's rearrangement of Algorithm 1
 * (left); the pipelined CG variants the paper's related work cites, Sec. 1):
 * the same iterates as classic CG in exact arithmetic, with the two inner
 * products of an iteration taken together after its one product with A.
 *   r = b - A x;  w = A r;  gamma = r^T r;  delta = w^T r
 *   alpha = gamma / delta;  beta = 0;  p = 0;  s = 0
 *   while gamma > eps^2 gamma_0:
 *       p = r + beta p;  s = w + beta s          (s = A p)
 *       x += alpha p;  r -= alpha s
 *       r = b - A x and s = A p on the R-th, 2R-th, ... iteration (R > 0)
 *       w = A r;  gamma' = r^T r;  delta = w^T r
 *       beta = gamma' / gamma;  alpha = gamma' / (delta - beta gamma' / alpha)
 *       gamma = gamma'
 * Returns the iteration count; *relres_out = sqrt(gamma / gamma_0). */
int or_cg_single_reduction(int64_t n, const double *A, int64_t lda, const double *b, double *x,
                           double eps, int maxit, int R, double *relres_out)
{
    double *r = malloc(sizeof(double) * n), *w = malloc(sizeof(double) * n);
    double *p = calloc((size_t)n, sizeof(double)), *s = calloc((size_t)n, sizeof(double));
    or_matvec_full(n, A, lda, x, r);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
    or_matvec_full(n, A, lda, r, w);
    double gamma = or_dot(n, r, r), gamma0 = gamma, delta = or_dot(n, w, r);
    double alpha = gamma > 0.0 ? gamma / delta : 0.0, beta = 0.0;
    int it = 0;
    while (gamma > eps * eps * gamma0 && it < maxit) {
        for (int64_t i = 0; i < n; ++i) {
            p[i] = r[i] + beta * p[i];
            s[i] = w[i] + beta * s[i];
        }
        for (int64_t i = 0; i < n; ++i) {
            x[i] += alpha * p[i];
            r[i] -= alpha * s[i];
        }
        ++it;
        if (R > 0 && it % R == 0) {
            or_matvec_full(n, A, lda, x, r);
            for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
            or_matvec_full(n, A, lda, p, s);
        }
        or_matvec_full(n, A, lda, r, w);
        double g = or_dot(n, r, r);
        delta = or_dot(n, w, r);
        beta = g / gamma;
        alpha = g / (delta - beta * g / alpha);
        gamma = g;
    }
    if (relres_out) *relres_out = (gamma0 > 0.0) ? sqrt(gamma / gamma0) : 0.0;
    free(r); free(w); free(p); free(s);
    return it;
}

/* C -= A B^T (C: m x n, A: m x k, B: n x k, column-major), every entry's
 * sum of products accumulated in long double and rounded once: the FP64
 * trailing update of Algorithm 1 step 3 stated as a definition, with a
 * rounding error (about k 2^-64 of sum |a b|) far below FP64's, so it can
 * judge an FP64-accurate product.  lower != 0: only entries with row >=
 * column (C square). */
void or_gemm_update(int64_t m, int64_t n, int64_t k, const double *A, int64_t lda, const double *B,
                    int64_t ldb, double *C, int64_t ldc, int lower)
{
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < m; ++i) {
            if (lower && i < j) continue;
            long double s = 0.0L;
            for (int64_t c = 0; c < k; ++c) s += (long double)A[IDX(i, c, lda)] * (long double)B[IDX(j, c, ldb)];
            C[IDX(i, j, ldc)] = (double)((long double)C[IDX(i, j, ldc)] - s);
        }
}

/* ------------------------------------------------------------------------ */
/* Error measures                                                             */
/* ------------------------------------------------------------------------ */

/* ||A x - b||_inf / (||A||_inf ||x||_inf + ||b||_inf), full A; the residual
 * and the row sums are accumulated in long double. */
double or_backward_error(int64_t n, const double *A, int64_t lda,
                         const double *x, const double *b)
{
    long double rmax = 0.0L, amax = 0.0L;
    double xmax = 0.0, bmax = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        long double ri = -(long double)b[i], ai = 0.0L;
        for (int64_t j = 0; j < n; ++j) {
            ri += (long double)A[IDX(i, j, lda)] * (long double)x[j];
            ai += fabsl((long double)A[IDX(i, j, lda)]);
        }
        if (fabsl(ri) > rmax) rmax = fabsl(ri);
        if (ai > amax) amax = ai;
        if (fabs(x[i]) > xmax) xmax = fabs(x[i]);
        if (fabs(b[i]) > bmax) bmax = fabs(b[i]);
    }
    long double den = amax * (long double)xmax + (long double)bmax;
    return den > 0.0L ? (double)(rmax / den) : 0.0;
}

/* Preconditioned CG with M = Lt Lt^T applied by forward and back
 * substitution; residual, dot products and A in FP64.  The recurrence
 * residual is replaced by the true residual b - A x every R iterations and
 * whenever the recurrence says ||r||/||b|| <= eps; the loop ends when the
 * true backward error is at most bwd_tol.  Returns the iteration count
 * (negative if maxit was reached). */
int or_pcg(int64_t n, const double *A, int64_t lda, const double *Lt,
           int64_t ldl, const double *b, double *x, double bwd_tol, double eps,
           int maxit, int R, double *bwd_out)
{
    double *r = malloc(sizeof(double) * n), *z = malloc(sizeof(double) * n);
    double *s = malloc(sizeof(double) * n), *t = malloc(sizeof(double) * n);
    or_matvec_full(n, A, lda, x, t);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - t[i];
    double bnorm2 = or_dot(n, b, b);
    memcpy(z, r, sizeof(double) * n);
    or_forward_sub(n, Lt, ldl, z, n, 1);
    or_back_sub(n, Lt, ldl, z, n, 1);
    memcpy(s, z, sizeof(double) * n);
    double u = or_dot(n, r, z);
    int it = 0, done = 0;
    double bwd = or_backward_error(n, A, lda, x, b);
    if (bwd <= bwd_tol) done = 1;
    while (!done && it < maxit) {
        or_matvec_full(n, A, lda, s, t);
        double alpha = u / or_dot(n, s, t);
        for (int64_t i = 0; i < n; ++i) x[i] += alpha * s[i];
        ++it;
        for (int64_t i = 0; i < n; ++i) r[i] -= alpha * t[i];
        int replace = (R > 0 && it % R == 0) || or_dot(n, r, r) <= eps * eps * bnorm2;
        if (replace) {
            or_matvec_full(n, A, lda, x, r);
            for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
            bwd = or_backward_error(n, A, lda, x, b);
            if (bwd <= bwd_tol) { done = 1; break; }
        }
        memcpy(z, r, sizeof(double) * n);
        or_forward_sub(n, Lt, ldl, z, n, 1);
        or_back_sub(n, Lt, ldl, z, n, 1);
        double v = u;
        u = or_dot(n, r, z);
        double beta = u / v;
        for (int64_t i = 0; i < n; ++i) s[i] = z[i] + beta * s[i];
    }
    if (bwd_out) *bwd_out = bwd;
    free(r); free(z); free(s); free(t);
    return done ? it : -it;
}
