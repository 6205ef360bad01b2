/*
 * gpchol.h -- C ABI of the B300 (sm_103a) dense SPD solver library for
 * Gaussian-process kernel systems A x = b.
 *
 * The operations are those of Thuering, Strack, Pflueger, "Comparing the
 * Performance of Heterogeneous Conjugate Gradient and Cholesky Solvers on
 * Various Hardware Using SYCL" (IWOCL '26):
 *   - the blocked right-looking Cholesky factorization of Algorithm 1 (right),
 *     steps 1-3 (Sec. 2.2, Sec. 3.2);
 *   - forward and back substitution with the factor (Sec. 2.2);
 *   - classic conjugate gradients, Algorithm 1 (left), with the residual
 *     recomputed from scratch every few iterations (Sec. 2.1, Sec. 3.1);
 * plus the entry points that build on them (the squared-exponential kernel
 * matrix the solvers are applied to, a mixed-precision refined solve, a
 * batched solve and a serving loop), each documented where it is declared.
 *
 * Conventions shared by every entry point
 *   - Matrices are column-major with a leading dimension ld >= max(1, n);
 *     element (i, j) of A is A[i + j*lda].  Only the lower triangle of a
 *     symmetric matrix or of a factor is read or written unless stated.
 *   - Matrix and vector pointers are DEVICE pointers owned by the caller,
 *     unless a parameter says "host".  The library never frees them.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on it; results in device memory are valid
 *     once the stream reaches the point after the call.  Calls that return
 *     host-side results (info, statistics) synchronize the stream first and
 *     say so.
 *   - Every call returns a gpch_status; no C++ exception crosses the ABI.
 *     On failure gpch_last_error(ctx) holds a one-line message.  There is no
 *     host fallback: without a usable GPU every compute call fails with
 *     GPCH_CUDA_ERROR.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef GPCHOL_H
#define GPCHOL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GPCH_VERSION 1

typedef enum gpch_status {
    GPCH_OK = 0,
    GPCH_INVALID_ARG = 1,    /* a size, pointer or option is out of range        */
    GPCH_NOT_SPD = 2,        /* a pivot was not positive; *info = 1-based column */
    GPCH_NOT_CONVERGED = 3,  /* iteration cap reached before the tolerance       */
    GPCH_OOM_BUDGET = 4,     /* workspace would exceed the context's HBM budget  */
    GPCH_TIMEOUT = 5,        /* a bounded device-side wait gave up               */
    GPCH_CUDA_ERROR = 6      /* a CUDA runtime call failed                       */
} gpch_status;

/* Storage type of a matrix operand. */
typedef enum gpch_dtype {
    GPCH_F64 = 0,
    GPCH_F32 = 1
} gpch_dtype;

/* Arithmetic of the factorization's trailing update (Algorithm 1, step 3). */
typedef enum gpch_prec {
    GPCH_PREC_FP64 = 0,        /* everything in FP64                              */
    GPCH_PREC_BF16 = 1,        /* bf16 tensor-core products, FP32 accumulation     */
    GPCH_PREC_SPLIT_BF16 = 2,  /* head+tail bf16 split, three products, FP32 acc.  */
    GPCH_PREC_SPLIT_F16 = 3    /* head+tail binary16 split of the panel scaled by a
                                  power of two (largest |entry| into [2^14, 2^15)),
                                  three products, FP32 acc.                       */
} gpch_prec;

typedef struct gpch_ctx gpch_ctx;

/* ------------------------------------------------------------------ context */

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the
 * workspace the context may allocate (0 = no cap beyond free memory).
 * The caller's own matrices do not count against the budget. */
gpch_status gpch_create(gpch_ctx **out, int device, size_t hbm_budget_bytes);

/* Free the context's workspace (synchronizes the device). NULL is a no-op. */
gpch_status gpch_destroy(gpch_ctx *ctx);

/* Static strings; never NULL. */
const char *gpch_status_string(gpch_status s);
const char *gpch_last_error(const gpch_ctx *ctx);
int gpch_version(void);

/* Bytes of workspace currently held by the context. */
size_t gpch_workspace_bytes(const gpch_ctx *ctx);

/* ------------------------------------------------------------ tracing */

/* Phases whose kernels can be timed with CUDA events recorded on the
 * launching stream around every launch of the phase. */
typedef enum gpch_phase {
    GPCH_PHASE_SE = 0,          /* A1 kernel matrix                               */
    GPCH_PHASE_DIAG = 1,        /* Algorithm 1 step 1 (diagonal tile)             */
    GPCH_PHASE_PANEL = 2,       /* Algorithm 1 step 2 (panel solve)               */
    GPCH_PHASE_TRAILING = 3,    /* Algorithm 1 step 3, FP64 (SYRK/GEMM)            */
    GPCH_PHASE_SOLVE = 4,       /* forward + back substitution                    */
    GPCH_PHASE_CG_MATVEC = 5,   /* CG matrix-vector product (one pass over A)      */
    GPCH_PHASE_CG_VECTOR = 6,   /* CG dot/axpy/xpay kernels                        */
    GPCH_PHASE_MIXED_TRAILING = 7, /* step 3 on tensor cores (bf16 / split)       */
    GPCH_PHASE_BATCHED = 8,     /* a whole batched solve (one graph launch)       */
    GPCH_PHASE_COUNT = 9
} gpch_phase;

/* Turn event timing on or off (off by default; costs two event records per
 * timed launch).  Turning it on clears the accumulated totals. */
gpch_status gpch_timing_enable(gpch_ctx *ctx, int enable);

/* Totals for one phase since timing was enabled: summed launch durations
 * (ms), launches timed, and the algorithmic work of those launches (flops
 * for factorization phases, bytes for CG phases; see the phase list).
 * Synchronizes on the recorded events.  Any output pointer may be NULL. */
gpch_status gpch_timing_read(gpch_ctx *ctx, int phase, double *total_ms, int64_t *launches, double *work);

/* Number of kernels this context has launched since it was created. */
int64_t gpch_launch_count(const gpch_ctx *ctx);

/* ------------------------------------------------ A1: GP kernel matrix */

/* Squared-exponential GP covariance of n points X (device, n x d,
 * row-major: point i at X + i*d):
 *     A_ij = sf2 * exp(-sum_k (X_ik - X_jk)^2 / (2 ell^2)) + sn2 * [i == j]
 * written to the full n x n matrix A (both triangles), FP64.  The squared
 * distance is summed term by term, so A is exactly symmetric and its
 * diagonal is exactly sf2 + sn2.  The paper's systems are GP covariance
 * matrices (Sec. 4.1); this is the synthetic kernel the solvers are run on.
 * Errors: INVALID_ARG if n < 0, d < 1, d > 64, lda < n, ell <= 0. */
gpch_status gpch_se_matrix(gpch_ctx *ctx, int64_t n, int d, const double *X,
                           double sf2, double ell, double sn2,
                           double *A, int64_t lda, void *stream);

/* --------------------------------------- A2-A4: blocked Cholesky, FP64 */

/* In-place blocked right-looking Cholesky, Algorithm 1 (right): for each
 * block column j of width `tile`:
 *   step 1  A_jj = chol(A_jj)                 (diagonal tile, FP64)
 *   step 2  A_ij = A_ij A_jj^{-T}, i > j      (panel triangular solve)
 *   step 3  A_ik -= A_ij A_kj^T, j < k <= i   (SYRK on k == i, GEMM below)
 * A: device, n x n, lda >= n; on return its lower triangle holds L with
 * L L^T = A (Sec. 2.2).  The strict upper triangle is not touched.
 * tile: 64..1024, multiple of 64 (the paper's block size, Sec. 4.4).
 * info (host): 0 on success, else the 1-based column whose pivot was not
 * positive (LAPACK convention); the call then returns GPCH_NOT_SPD and the
 * lower triangle holds a partial factor.  Synchronizes `stream`.
 * Errors: INVALID_ARG (n < 0, lda < n, bad tile, info NULL). */
gpch_status gpch_chol_factor(gpch_ctx *ctx, int64_t n, int tile, double *A,
                             int64_t lda, void *stream, int64_t *info);

/* ------------------------------------------- A5: substitution with L */

/* Solve L L^T X = B in place: forward substitution L Y = B, then back
 * substitution L^T X = Y (Sec. 2.2).  L: device, lower triangle of an
 * n x n factor (as left by gpch_chol_factor), ldl >= n.  B: device,
 * n x nrhs, ldb >= n, overwritten with X.  Asynchronous on `stream`.
 * Errors: INVALID_ARG (n < 0, nrhs < 0, ldl < n, ldb < n). */
gpch_status gpch_chol_solve(gpch_ctx *ctx, int64_t n, const double *L,
                            int64_t ldl, double *B, int64_t ldb, int nrhs,
                            void *stream);

/* The same solve with an FP32 factor, e.g. the low-precision factor of
 * gpch_chol_factor_mixed (the preconditioner application of the refined
 * solve, z = (L L^T)^-1 r): block products in FP32, partial sums and the
 * right-hand sides FP64.  With one or two right-hand sides, a 16-byte
 * aligned L and ldl a multiple of 4, each sweep walks 128-row blocks and
 * keeps one 128 x 128 product per block on its serial chain (coupling
 * blocks inv(L_II) L_{I,I-1} and L_{I+1,I} inv(L_II), formed once per
 * call); otherwise 64-row blocks.  L: device, lower triangle (the strict
 * upper triangle is not read), ldl >= n.  B: device FP64, n x nrhs,
 * ldb >= n, overwritten with X.  Synchronizes the stream.  Extra
 * workspace: about 24 n * 128 + 16 n * 64 bytes.  Errors: INVALID_ARG,
 * TIMEOUT (a bounded wait of a sweep gave up). */
gpch_status gpch_chol_solve_f32(gpch_ctx *ctx, int64_t n, const float *L,
                                int64_t ldl, double *B, int64_t ldb,
                                int nrhs, void *stream);

/* Arithmetic of step 3 in gpch_chol_factor_ex. */
typedef enum gpch_update {
    GPCH_UPDATE_FP64 = 0,           /* FP64 FMAs (gpch_chol_factor)              */
    GPCH_UPDATE_FP64_EMULATED = 1   /* FP64-accurate products on the tensor cores
                                       (gpch_gemm_fp64_emulated)                  */
} gpch_update;

/* gpch_chol_factor with a choice of step-3 arithmetic: GPCH_UPDATE_FP64 is
 * gpch_chol_factor itself; GPCH_UPDATE_FP64_EMULATED computes every
 * trailing update A_ik -= A_ij A_kj^T of Algorithm 1 (right) with the
 * tensor-core product of gpch_gemm_fp64_emulated (per entry and block
 * column an error below about tile 2^-48 times the product of the two
 * rows' largest panel entries, one FP64 rounding), steps 1 and 2 in FP64 as
 * before.  Extra workspace: 8 n * 1024 bytes.  Returns GPCH_TIMEOUT if a
 * bounded tensor-core wait gave up; otherwise as gpch_chol_factor. */
gpch_status gpch_chol_factor_ex(gpch_ctx *ctx, int64_t n, int tile, double *A, int64_t lda, int32_t update,
                                void *stream, int64_t *info);

/* --------------------------------------------------- A6-A7: CG solve */

typedef struct gpch_cg_stats {
    int32_t iterations;   /* max over right-hand sides                       */
    int32_t converged;    /* number of right-hand sides that met rtol         */
    double relres_max;    /* max over RHS of sqrt(u/u0) at exit (recurrence)  */
} gpch_cg_stats;

/* Conjugate gradients, Algorithm 1 (left), per right-hand side:
 *   s = r = b - A x;  u = u0 = r^T r
 *   while u > rtol^2 u0:  t = A s;  alpha = u / s^T t;  x += alpha s;
 *       r -= alpha t  (or r = b - A x on every replace_every-th iteration,
 *       Sec. 2.1);  beta = r^T r / u;  u = r^T r;  s = r + beta s
 * A: device, full symmetric n x n (both triangles stored), lda >= n, of
 * storage type dtype (F32 values are widened exactly to FP64; all vectors,
 * dot products and recurrences are FP64).  B: device n x nrhs (ldb); X:
 * device n x nrhs (ldx), read as the start vector and overwritten with the
 * solution.  The nrhs columns run independent recurrences that share one
 * pass over A per iteration; a converged column is frozen.
 * maxit: iteration cap (> 0).  replace_every: R > 0 replaces the residual
 * on iterations R, 2R, ...; 0 never.  stats (host, may be NULL) is filled
 * after the call synchronizes `stream`.
 * Returns GPCH_NOT_CONVERGED if some column missed rtol within maxit. */
gpch_status gpch_cg_solve(gpch_ctx *ctx, int64_t n, const void *A,
                          gpch_dtype dtype, int64_t lda, const double *B,
                          int64_t ldb, double *X, int64_t ldx, int nrhs,
                          double rtol, int maxit, int replace_every,
                          void *stream, gpch_cg_stats *stats);

/* Options of gpch_cg_solve_ex. */
typedef enum gpch_cg_variant {
    GPCH_CG_CLASSIC = 0,           /* Algorithm 1 (left) as above                     */
    GPCH_CG_SINGLE_REDUCTION = 1   /* Chronopoulos-Gear rearrangement (below)         */
} gpch_cg_variant;

typedef enum gpch_cg_products {
    GPCH_CG_PRODUCTS_FP64 = 0,         /* one FP64 FMA per entry and right-hand side  */
    GPCH_CG_PRODUCTS_DOUBLE_FLOAT = 1, /* double-float products on the FP32 pipe      */
    GPCH_CG_PRODUCTS_TENSOR = 2        /* FP64-accurate products on the tensor cores  */
} gpch_cg_products;

typedef struct gpch_cg_opts {
    int32_t variant;    /* gpch_cg_variant  */
    int32_t products;   /* gpch_cg_products */
} gpch_cg_opts;

/* gpch_cg_solve with a choice of iteration form and product arithmetic
 * (opts NULL = classic, FP64 products: exactly gpch_cg_solve).
 *
 * GPCH_CG_SINGLE_REDUCTION: the same iterates as Algorithm 1 (left) in exact
 * arithmetic, rearranged so that one product w = A r is followed by both
 * inner products together (the single-reduction / pipelined CG variants of
 * the paper's related work, Sec. 1):
 *   r = b - A x; w = A r; gamma = r^T r; delta = w^T r; alpha = gamma/delta
 *   loop: p = r + beta p; s = w + beta s; x += alpha p; r -= alpha s;
 *         w = A r; gamma' = r^T r; delta = w^T r; beta = gamma'/gamma;
 *         alpha = gamma'/(delta - beta gamma'/alpha); gamma = gamma'
 * One reduction point per iteration instead of two; one extra product
 * with A at the start.  On replacement iterations r = b - A x and
 * s = A p are both recomputed (two extra products).  Stop rule
 * gamma <= rtol^2 gamma_0 per column.
 *
 * GPCH_CG_PRODUCTS_DOUBLE_FLOAT: the products A_ij s_i are formed on the
 * FP32 pipe from a float head and tail of each operand (FP64 entries of A
 * are cut by integer operations, the vector once per product with A),
 * head*head exactly plus the two cross terms, summed in an error-free
 * double-float accumulator and reduced across threads in FP64.  Each
 * product carries a relative error below about 2^-45 (FP32 A: below about
 * 2^-47), so the computed A s differs from the FP64 one by about
 * 1e-14 sum_j |A_ij||s_j| per entry.  A's largest diagonal entry and each
 * column's largest |b| set power-of-two scales first, so entries of A
 * within 2^-126 of the largest diagonal entry and vectors within FP32's
 * range of that scale lose nothing more; an entry of A at or above 2^128
 * times the largest diagonal entry makes the product non-finite (the
 * solve then reports NOT_CONVERGED).  The true residuals b - A x (at the
 * start and on replacement iterations) always use FP64 products, so the
 * accuracy the iteration reaches is that of FP64 CG.  The vector
 * recurrences, inner products and scalars stay FP64 in both forms.
 *
 * GPCH_CG_PRODUCTS_TENSOR: the iteration products on the bf16 tensor cores
 * by an error-free splitting (as gpch_gemm_fp64_emulated): A is cut once
 * per solve (and per group of 16 right-hand sides) into 8 base-128 digits
 * per entry with a power-of-two scale per column of A and 512-entry pass,
 * each vector once per product likewise; the 28 digit pairs of weight
 * class p + d <= 6 are summed exactly per pass and rounded once, passes
 * added in FP64.  The dropped pairs weigh at most 2^-44 of the two pass
 * scales per term (each scale is the power of two just above the pass's
 * largest magnitude), so per entry of A s the error is at most about
 * n 2^-42 max_j |A_ij| max |s|.  A must
 * be symmetric (its columns serve as rows).  Extra workspace: 16 np kp
 * bytes for A's digits (np = n rounded up to 128, kp = n rounded up to
 * 512) plus 4 np kp / 512 bytes of exponents.  True residuals take the
 * same tensor-core product with the 8 pairs of weight class 7 kept too, so
 * the dropped pairs weigh at most about 2^-51 of the pass scales per term
 * (FP64-level products).  Errors as above, plus INVALID_ARG when np kp / 8 does not fit
 * 31 bits (n above about 131000) and TIMEOUT when a bounded tensor-core
 * wait gave up. */
gpch_status gpch_cg_solve_ex(gpch_ctx *ctx, int64_t n, const void *A, gpch_dtype dtype, int64_t lda,
                             const double *B, int64_t ldb, double *X, int64_t ldx, int nrhs, double rtol,
                             int maxit, int replace_every, const gpch_cg_opts *opts, void *stream,
                             gpch_cg_stats *stats);

/* ------------------------- row-split CG across ranks: local steps (f4) */

/* A CG solve whose rows are split over ranks (one GPU each): the paper's
 * horizontal split of the matrix between CPU and GPU (Sec. 3.1), carried
 * to several GPUs.  Rank k owns rows r0 .. r0+m-1 of the symmetric A,
 * stored as the n x m column block A[:, r0 : r0+m] (by symmetry the same
 * numbers), and the matching m rows of x, b and every CG vector.  The
 * single-reduction form of gpch_cg_solve_ex runs as:
 *   setup  allgather x0 -> v;  t = Ablk^T v;  r = b - t          (residual, all = 1)
 *          allgather r -> v;  w = Ablk^T v;  partials(r, w) -> sums;
 *          allreduce(sums);  scalars(first = 1)
 *   loop   vectors(replace);
 *          on replacement iterations: allgather x -> v; t = Ablk^T v;
 *              r = b - t (residual, all = 0); allgather p -> v; s = Ablk^T v
 *          allgather r -> v;  w = Ablk^T v;  partials(r, w) -> sums;
 *          allreduce(sums);  scalars(first = 0);  stop when state.done
 * The caller moves the data between ranks (the allgather of one n x nrhs
 * vector and the allreduce of 2 nrhs doubles per iteration, e.g. over
 * NCCL); these calls make every arithmetic step on the rank's rows.  Every
 * rank's scalar state evolves identically because it is computed from the
 * same reduced sums.  All pointers are device memory; asynchronous on
 * `stream`; nrhs <= 16. */

/* Device-resident scalar state of one rank's solve (caller-allocated,
 * sizeof(gpch_cgsr_state) bytes of device memory, 8-byte aligned). */
typedef struct gpch_cgsr_state {
    double gamma[16], gamma0[16], alpha[16], beta[16];
    int32_t active[16], iters[16];
    int32_t done, pad_;
} gpch_cgsr_state;

/* T = Ablk^T V: rows r0 .. r0+m-1 of A V for the symmetric n x n A whose
 * columns r0 .. r0+m-1 are the n x m block Ablk (lda >= n; its diagonal
 * entries are Ablk[r0 + j + j lda]).  V: n x nrhs (ldv >= n); T: m x nrhs
 * (ldt >= m).  products: gpch_cg_products (FP64 or double-float, as in
 * gpch_cg_solve_ex; the double-float scales come from the block's diagonal
 * entries and V's columns).  With m = n and r0 = 0 this is A V.
 * Workspace from the context arena.  Errors: INVALID_ARG. */
gpch_status gpch_block_matvec(gpch_ctx *ctx, int64_t n, int64_t m, int64_t r0, const void *Ablk,
                              gpch_dtype dtype, int64_t lda, const double *V, int64_t ldv, double *T,
                              int64_t ldt, int nrhs, int32_t products, void *stream);

/* sums[c] = sum_i R_ic^2 and sums[nrhs + c] = sum_i W_ic R_ic over the m
 * local rows (fixed-order reduction).  sums: device, 2 nrhs doubles. */
gpch_status gpch_cgsr_partials(gpch_ctx *ctx, int64_t m, int nrhs, const double *R, int64_t ldr,
                               const double *W, int64_t ldw, double *sums, void *stream);

/* Scalar step from the ranks' summed partials (gamma' = sums[c],
 * delta = sums[nrhs + c]).  first = 1: gamma_0 = gamma = gamma',
 * alpha = gamma'/delta, beta = 0, iters = 0, active = gamma' > 0.
 * Otherwise, on active columns: iters += 1, beta = gamma'/gamma,
 * alpha = gamma'/(delta - beta gamma'/alpha), gamma = gamma', and the
 * column retires when gamma' <= rtol^2 gamma_0 or iters >= maxit.  done is
 * set when no column is active. */
gpch_status gpch_cgsr_scalars(gpch_ctx *ctx, int nrhs, const double *sums, gpch_cgsr_state *state,
                              int first, double rtol, int maxit, void *stream);

/* On active columns: p = r + beta p; s = w + beta s; x += alpha p; and,
 * unless `replace`, r -= alpha s.  R, W, P, S: m x nrhs with leading
 * dimension ld; X: m x nrhs (ldx).  P and S start at zero. */
gpch_status gpch_cgsr_vectors(gpch_ctx *ctx, int64_t m, int nrhs, gpch_cgsr_state *state, double *X,
                              int64_t ldx, double *R, const double *W, double *P, double *S, int64_t ld,
                              int replace, void *stream);

/* r = b - t on the active columns (on every column with all = 1).  B:
 * m x nrhs (ldb); T and R: m x nrhs (ld). */
gpch_status gpch_cgsr_residual(gpch_ctx *ctx, int64_t m, int nrhs, gpch_cgsr_state *state, const double *B,
                               int64_t ldb, const double *T, double *R, int64_t ld, int all, void *stream);

/* ------------------------------------- allocation-free CG (no paper
 * counterpart: the paper has no allocation-free variant; this is a
 * service to callers of the library) */

/* Largest n * nrhs gpch_cg_solve_noalloc accepts. */
#define GPCH_NOALLOC_CG_MAX_ELEMS 262144

/* The same conjugate-gradient solve as gpch_cg_solve, for callers that
 * cannot allocate device memory: code that must not call cudaMalloc or
 * cudaFree because it runs where the allocator is off limits (a host
 * application or framework that owns the GPU's memory budget and forbids
 * plugins from allocating, a real-time loop that cannot afford the
 * allocator's implicit synchronization, or a caller without a context of
 * this library, whose creation pins host memory).  It allocates nothing:
 * its scratch (the CG vectors r, s, t, the device scalars and the partial
 * sums) lives in one fixed 12 MiB file-scope device array, and its host
 * staging is on the stack.  The caller still passes A, B and X.
 *   - When the array is reserved: the CUDA driver reserves it on a device
 *     when it loads this library's CG module there.  With lazy module
 *     loading (CUDA's default since 12.2) that happens at the first use of
 *     the module on that device, which may be the first call of this entry
 *     point; the 12 MiB are then taken at that moment and kept until the
 *     process exits.  A caller that may not allocate later makes one call
 *     with n = 0 (or nrhs = 0) on each device at set-up time, with the device
 *     current and before any stream capture: it loads the module, makes
 *     sure the array and the code of every kernel the solve launches are on
 *     the device, and solves nothing.  Calls after it allocate nothing.
 *   - Runs on the caller's current device and looks up the array's device
 *     address on every call (a device reset is therefore harmless).
 *   - Limits: 0 <= nrhs <= 16 and n * nrhs <= GPCH_NOALLOC_CG_MAX_ELEMS;
 *     larger problems return GPCH_INVALID_ARG before any device work.
 *   - Every call shares the one array and leaves its contents behind; the
 *     call clears what must start at zero.  Calls whose GPU work overlaps
 *     (other streams, other host threads) race on the array: serialize them.
 *   - Arguments, convergence rule and return codes as gpch_cg_solve; it
 *     synchronizes `stream`.  No error message is kept (there is no context). */
gpch_status gpch_cg_solve_noalloc(int64_t n, const void *A, gpch_dtype dtype, int64_t lda, const double *B,
                                  int64_t ldb, double *X, int64_t ldx, int nrhs, double rtol, int maxit,
                                  int replace_every, void *stream, gpch_cg_stats *stats);

/* ---------------------------------------------- A10: batched solve */

/* One system of a batch: A (device, FP64, n x n, lda >= n; its lower
 * triangle is overwritten by the factor L) and B (device, n x nrhs,
 * ldb >= n; overwritten by the solution X). */
typedef struct gpch_system {
    int64_t n;
    double *A;
    int64_t lda;
    double *B;
    int64_t ldb;
    int32_t nrhs;
} gpch_system;

/* Factor and solve `count` independent SPD systems A_s X_s = B_s in FP64:
 * Algorithm 1 (right) with 64-wide blocks on every system, then forward
 * and back substitution.  Step k of all systems runs in one grouped launch
 * per kernel kind, and the whole launch sequence of a batch is captured
 * once as a CUDA graph that later calls with the same systems (same sizes
 * and pointers) replay as one graph launch.  Each system is tiled by its
 * own size only, so its result does not depend on its batch-mates.
 * systems: host array of count descriptors.  info: host array of count
 * entries, 0 or the 1-based failing column of that system (the call then
 * returns GPCH_NOT_SPD; the other systems are still solved).  The context
 * keeps up to 8 captured batches (device tables and per-system workspace,
 * counted against the HBM budget) until gpch_destroy.  Synchronizes
 * `stream`. */
gpch_status gpch_batched_solve(gpch_ctx *ctx, int count, const gpch_system *systems, void *stream,
                               int64_t *info);

/* One system of a mixed-precision batch: A (device, FP64, n x n, both
 * triangles, lda >= n) and B (device, n x nrhs, ldb >= n) are read only;
 * X (device, n x nrhs, ldx >= n) receives the solution.  nrhs <= 16. */
typedef struct gpch_msystem {
    int64_t n;
    const double *A;
    int64_t lda;
    const double *B;
    int64_t ldb;
    double *X;
    int64_t ldx;
    int32_t nrhs;
} gpch_msystem;

typedef struct gpch_batch_stats {
    int32_t iterations;          /* refinement corrections, max over systems  */
    int32_t steps;               /* refinement steps the batch ran            */
    double backward_error_max;   /* max over systems and columns at exit      */
} gpch_batch_stats;

/* Mixed-precision batched solve of `count` independent SPD systems: per
 * system an FP32 Cholesky factor, Algorithm 1 (right) with 64-wide blocks
 * (step 1 in FP64 on the widened 64 x 64 diagonal block, its FP64 inverse
 * kept; step 2 as the product with that inverse; step 3 in FP32), then
 * iterative refinement in FP64 until every column's normwise backward
 * error ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf) <= bwd_tol:
 * x_0 = L^-T L^-1 b, then r = b - A x (FP64 products, A intact) and
 * x += L^-T L^-1 r.  Step k of all systems runs as one grouped launch per
 * kernel kind, each system tiled by its own size only (a system's result
 * does not depend on its batch-mates), and the launch sequence (set-up,
 * factor, first solve, 4 refinement steps) is captured once as a CUDA graph
 * per set of systems (same sizes and pointers), replayed by later calls; a
 * batch that needs more steps replays a captured single step (at most
 * maxit steps, maxit >= 4).  The context keeps up to 8 captured batches
 * (their FP32 factors and work vectors, about 4 n^2 + 32 n nrhs bytes per
 * system) until gpch_destroy.
 * info (host, count entries): 0; the 1-based column where the FP32 factor
 * broke down (returns GPCH_NOT_SPD); or -1 if refinement stopped improving
 * (its error no longer halving per step) or reached maxit before bwd_tol
 * (returns GPCH_NOT_CONVERGED).  stats (host, may be NULL).  Synchronizes
 * `stream`. */
gpch_status gpch_batched_solve_mixed(gpch_ctx *ctx, int count, const gpch_msystem *systems, double bwd_tol,
                                     int maxit, void *stream, int64_t *info, gpch_batch_stats *stats);

/* -------------------------------------------------- A11: serving loop */

typedef struct gpch_server gpch_server;

typedef struct gpch_server_opts {
    size_t hbm_budget;       /* device bytes that admitted, unfinished requests
                                may hold (0 = no cap)                              */
    int32_t lanes;           /* GPU lanes: host threads, each with its own
                                context and CUDA stream (1..32)                    */
    int32_t batch_max_count; /* at most this many requests per batched launch      */
    int64_t batch_max_n;     /* requests with n <= batch_max_n go through the
                                batched FP64 path (gpch_batched_solve's kernels)   */
    gpch_prec solo_prec;     /* larger requests: GPCH_PREC_FP64 (factor + solve)
                                or a mixed precision (gpch_solve_refined)          */
    double bwd_tol;          /* backward-error target of the refined path          */
} gpch_server_opts;

/* One GP solve request; every pointer is HOST memory that the caller keeps
 * alive (and Xout untouched) until the request completes. */
typedef struct gpch_request {
    int64_t n;
    int32_t d;               /* point dimension, 1..64                             */
    int32_t nrhs;
    const double *X;         /* n x d points, row-major                            */
    double sf2, ell, sn2;    /* squared-exponential hyper-parameters               */
    const double *B;         /* n x nrhs right-hand sides, column-major            */
    double *Xout;            /* n x nrhs solution, column-major (written on completion) */
} gpch_request;

typedef struct gpch_result {
    gpch_status status;
    int32_t path;            /* 1 batched FP64, 2 solo mixed refined, 3 solo FP64  */
    int32_t iterations;      /* refinement iterations (path 2)                     */
    double backward_error;   /* final backward error reported by the path 2 solve  */
    double latency_ms;       /* completion minus submission                        */
    double queue_ms;         /* start of GPU work minus submission                 */
} gpch_result;

typedef struct gpch_server_stats {
    int64_t completed, failed, batches, batched_requests;
    size_t peak_reserved_bytes;
    double p50_ms, p99_ms, max_ms;   /* latency percentiles of completed requests */
    double solves_per_s;             /* completed / (last completion - first submit) */
} gpch_server_stats;

/* Serving loop with continuous batching (the scope's serving pattern; the
 * paper has no serving layer).  Each request builds its SE matrix (A1) on
 * the device and is solved there.  A dispatcher admits queued requests in
 * arrival order, first fit against hbm_budget, whenever a lane is free:
 * up to batch_max_count small requests (n <= batch_max_n) are solved
 * together by one batched FP64 launch sequence, a larger request runs alone
 * on its lane.  Lanes run concurrently on their own streams, so requests
 * that arrive while others are on the GPU start as soon as a lane and
 * memory are free and their work overlaps.  A request's arithmetic depends
 * only on its own data and the path its n selects.  Each lane keeps its
 * largest device buffers and workspace until gpch_server_destroy. */
gpch_status gpch_server_create(int device, const gpch_server_opts *opts, gpch_server **out);

/* Queue a request (copied; its host buffers are not).  Returns
 * GPCH_OOM_BUDGET if it could never fit the budget. */
gpch_status gpch_server_submit(gpch_server *srv, const gpch_request *req, uint64_t *ticket);

/* Wait up to timeout_s for a request; on completion fills *res (may be NULL),
 * forgets the ticket and returns the request's status (GPCH_TIMEOUT if it
 * is still running; the ticket stays valid). */
gpch_status gpch_server_wait(gpch_server *srv, uint64_t ticket, double timeout_s, gpch_result *res);

/* Non-blocking: *done = 1 and *res filled once the request completed. */
gpch_status gpch_server_poll(gpch_server *srv, uint64_t ticket, int *done, gpch_result *res);

gpch_status gpch_server_get_stats(gpch_server *srv, gpch_server_stats *out);

/* Stop the lanes after their current work; queued requests are dropped.
 * No other call on `srv` may be in progress. */
gpch_status gpch_server_destroy(gpch_server *srv);

/* --------------------------- A4 (mixed): tensor-core trailing update */

/* C -= P P^T on the lower triangle of the m x m FP32 matrix C (ldc), with
 * P the m x k FP32 panel (ldp): the operation of Algorithm 1 step 3 for a
 * whole trailing matrix, computed on the tensor cores from a bfloat16 copy
 * of P (prec = GPCH_PREC_BF16), from a bfloat16 head and tail of P with
 * head*head^T + head*tail^T + tail*head^T (GPCH_PREC_SPLIT_BF16), or from a
 * binary16 head and tail of 2^e P, e chosen so that the largest |entry|
 * lands in [2^14, 2^15), with the three products scaled back by 2^-2e
 * (GPCH_PREC_SPLIT_F16); FP32 accumulation.  The strict upper triangle of
 * C is not touched.  k <= 4096.
 * Synchronizes `stream` (returns GPCH_TIMEOUT if a bounded pipeline wait
 * gave up).  Mixed precision is the paper's future work (Sec. 5). */
gpch_status gpch_syrk_lowprec(gpch_ctx *ctx, int64_t m, int64_t k, const float *P, int64_t ldp, float *C,
                              int64_t ldc, gpch_prec prec, void *stream);

/* ------------------------------------- A8: low-precision factor */

/* Low-precision Cholesky factor of A + shift I: Algorithm 1 (right) on an
 * FP32 copy with step 1 in FP64, step 2 in FP32 (for GPCH_PREC_SPLIT_F16
 * the tensor-core product of the panel with L_jj^-T, split-f16 operands,
 * L_jj^-1 from an FP32 substitution) and step 3 on the tensor cores as in
 * gpch_syrk_lowprec.  A: device FP64 n x n (lower triangle
 * read, not modified).  L: device FP32 n x n (ldl), receives the factor in
 * its lower triangle.  prec: GPCH_PREC_BF16, GPCH_PREC_SPLIT_BF16 or
 * GPCH_PREC_SPLIT_F16 (one power-of-two scale for the whole factor, from
 * |L_ij| <= sqrt(max_i (A_ii + shift))).  Step 3 is applied left-looking:
 * each block column receives the products of all earlier panels just
 * before its diagonal tile is factored.  Workspace: about 4 n^2 bytes for
 * the 16-bit panel copies.
 * info (host): 0, or the 1-based column of a non-positive pivot (returns
 * GPCH_NOT_SPD).  Synchronizes `stream`. */
gpch_status gpch_chol_factor_mixed(gpch_ctx *ctx, int64_t n, int tile, const double *A, int64_t lda,
                                   gpch_prec prec, double shift, float *L, int64_t ldl, void *stream,
                                   int64_t *info);

/* --------------------------------------------- A9: refined solve */

typedef struct gpch_refine_stats {
    int32_t iterations;          /* PCG iterations (max over RHS groups)       */
    int32_t factor_attempts;     /* low-precision factorizations run           */
    double shift;                /* diagonal shift of the accepted factor      */
    double backward_error_max;   /* max over RHS of the final true backward error */
} gpch_refine_stats;

/* Solve A X = B to a normwise backward error
 *     ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf) <= bwd_tol
 * per column: low-precision factor Lt of A + delta I (gpch_chol_factor_mixed
 * with the shift schedule delta_0 = 0 for SPLIT_BF16 and SPLIT_F16 and
 * 2^-7 max_i A_ii for BF16, then delta <- max(4 delta, 2 u max_i A_ii) after
 * each breakdown, u = 2^-8, 2^-16, 2^-22 for BF16, SPLIT_BF16, SPLIT_F16; at
 * most 9 attempts), then preconditioned CG with M = Lt Lt^T in FP64 (A, x,
 * r and all dot products FP64; Algorithm 1 (left) with a preconditioner),
 * from x_0 = 0 (the products A s and the true residuals b - A x formed as
 * double-float products: with one or two right-hand sides per group of 16
 * as gpch_symv_lower, from A's lower triangle, else as gpch_cg_solve_ex's
 * GPCH_CG_PRODUCTS_DOUBLE_FLOAT over all of A; each entry of a true
 * residual is then within about 2^-44 sum_j |A_ij| |x_j| of the exact one,
 * at most 2^-44 of the backward error's denominator), replacing the recurrence residual by b - A x every 50
 * iterations and whenever an estimate of the backward error from the
 * recurrence residual (its ||r||_inf in place of the true residual's,
 * scaled by the truth-to-estimate ratio seen at the previous check)
 * reaches bwd_tol.
 * A: device FP64 symmetric n x n (lda); the factor, ||A||_inf and, with
 * at most two right-hand sides, the products read its lower triangle only
 * (with more, the products read all of it).  B: device n x nrhs
 * (ldb).  X: device n x nrhs (ldx), overwritten.  Workspace (context
 * arena): about 8 n^2 bytes, the FP32 factor and the 16-bit copies of its
 * panels (plus gpch_symv_lower's partial sums); with one or two right-hand
 * sides 4 n^2 bytes more for the products' packed copy of A's lower
 * triangle.
 * tile: the factor's block size, a multiple of 64 in [64, 1024], or 0 for
 * the autotuned tile of n's size bucket (gpch_autotune; defaults 256 for
 * n <= 4096, else 512, until the device is tuned).
 * stats (host, may be NULL).  Synchronizes `stream`.  Returns GPCH_NOT_SPD
 * if every shifted factorization broke down, GPCH_NOT_CONVERGED if some
 * column missed bwd_tol within maxit iterations. */
gpch_status gpch_solve_refined(gpch_ctx *ctx, int64_t n, const double *A, int64_t lda, const double *B,
                               int64_t ldb, double *X, int64_t ldx, int nrhs, gpch_prec prec, int tile,
                               double bwd_tol, int maxit, void *stream, gpch_refine_stats *stats);

/* Y = A X for a symmetric A of which only the lower triangle (i >= j)
 * affects the result: the product of the refined solve's CG iteration
 * (Algorithm 1 (left), its A s and its true residuals b - A x).  Each
 * stored entry serves twice, A_ij x_j in y_i and A_ij x_i in y_j, so the
 * product reads about half of A's bytes.  The products are double-float
 * products on the FP32 pipe (as gpch_cg_solve_ex's
 * GPCH_CG_PRODUCTS_DOUBLE_FLOAT): each carries a relative error below about
 * 2^-44, summed without further loss in double-float and added in FP64 in
 * a fixed order, so y_i is within about 2^-44 sum_j |A_ij| |x_j| of the
 * exact product and the result does not depend on scheduling.  Power-of-two
 * scales come from A's largest diagonal entry and each column's largest
 * |x|: entries of A at or above 2^127 times the largest diagonal entry make
 * the product non-finite, entries below 2^-126 times it count as zero.
 * A: device FP64, n x n column-major (lda); entries above the diagonal may
 * be read but never change the result.  X: device n x nrhs (ldx).  Y:
 * device n x nrhs (ldy), overwritten; it must not overlap X.  Work space
 * from the context arena: about n^2 / 16 bytes per column of a pair (the
 * partial sums of 256 x 256 units).  Enqueued
 * on `stream` (no synchronization); the context's arena is in use until it
 * completes.  Errors: INVALID_ARG (n >= 2^24, ld < n, null pointers),
 * OUT_OF_MEMORY, CUDA_ERROR. */
gpch_status gpch_symv_lower(gpch_ctx *ctx, int64_t n, const double *A, int64_t lda, const double *X, int64_t ldx,
                            double *Y, int64_t ldy, int nrhs, void *stream);

/* ------------------------------ GP quantities on a solved system (f3) */

/* log det A of the SPD matrix A = L L^T from its FP64 Cholesky factor:
 * det A = prod_i L_ii^2, so log det A = 2 sum_i log L_ii.  This is the
 * log-determinant term of the GP's log marginal likelihood; the paper's
 * systems are GP covariance matrices used for behaviour prediction
 * (Sec. 4.1).  L: device, lower triangle of an n x n factor as left by
 * gpch_chol_factor (only the diagonal is read), ldl >= n.  logdet: HOST
 * pointer, written after the call synchronizes `stream` (0 for n = 0).
 * The sum is reduced in a fixed order, so the value is reproducible.
 * Errors: INVALID_ARG (n < 0, ldl < n, NULL pointers); NOT_SPD if some
 * L_ii is not positive or not finite (*logdet is then NaN). */
gpch_status gpch_logdet(gpch_ctx *ctx, int64_t n, const double *L, int64_t ldl, double *logdet,
                        void *stream);

/* GP predictive mean at m new points:
 *     mean_kr = sum_i sf2 exp(-||xs_k - x_i||^2 / (2 ell^2)) alpha_ir
 * the noise-free squared-exponential cross covariance between the test
 * points Xs and the training points X times alpha = (K + sn2 I)^-1 Y, the
 * solution of the GP system (behaviour prediction with a GP, Sec. 4.1).
 * The cross covariance is formed on the fly and never stored.
 * Xs: device, m x d row-major; X: device, n x d row-major (the points the
 * system's matrix was built from, 1 <= d <= 64).  alpha: device n x nrhs
 * (lda >= n), mean: device m x nrhs (ldm >= m), column-major,
 * 0 <= nrhs <= 16.  Asynchronous on `stream`.  Workspace: 128 bytes per
 * (test point, slice) pair, slices chosen to fill the GPU.  Partial sums
 * are added in a fixed order (reproducible).
 * Errors: INVALID_ARG (negative sizes, d out of range, nrhs > 16, ld too
 * small, ell <= 0, NULL pointers); OOM_BUDGET if the workspace does not
 * fit the context's budget. */
gpch_status gpch_predict_mean(gpch_ctx *ctx, int64_t m, int64_t n, int d, const double *Xs, const double *X,
                              double sf2, double ell, const double *alpha, int64_t lda, int nrhs,
                              double *mean, int64_t ldm, void *stream);

/* ------------------------- FP64-accurate products on tensor cores (f1) */

/* C -= A B^T for FP64 A (m x k, lda >= m), B (n x k, ldb >= n) and C
 * (m x n, ldc >= m), column-major, computed on the bf16 tensor cores by an
 * error-free splitting in the manner of the Ozaki scheme (the paper names
 * faster mixed/emulated arithmetic as future work, Sec. 5; the operation is
 * Algorithm 1 step 3 at any size):
 *   - each row of A (and of B) is scaled by a power of two from its
 *     largest |entry| and rounded to a 54-bit integer, written as 8
 *     balanced base-128 digits, each exact in bf16;
 *   - the 36 digit pairs of weight 128^-(p+q), p + q <= 7, are multiplied
 *     on the tensor cores; pairs of equal weight share one FP32 accumulator,
 *     whose sums stay exact (integers below 2^24) over K passes of at most
 *     512 columns;
 *   - the 8 weighted sums are combined exactly and rounded once per pass
 *     into C in FP64.
 * Per entry and pass the error is below about k 2^-48 2^(e_i + f_j), with
 * 2^e_i and 2^f_j the row scales (|A_ic| < 2^e_i): the size of FP64 GEMM's
 * worst-case bound when a row's largest entries set its scale, though
 * larger than FP64's for rows whose entries span many binades.
 * lower != 0: C is square (m == n) and only its lower triangle (row >=
 * column) is written.  A and B may be the same matrix (the SYRK case).
 * Workspace (context arena): about 16 (m + n) * 512 bytes.
 * Synchronizes `stream`; returns GPCH_TIMEOUT if a bounded pipeline wait
 * gave up.  Errors: INVALID_ARG. */
gpch_status gpch_gemm_fp64_emulated(gpch_ctx *ctx, int64_t m, int64_t n, int64_t k, const double *A, int64_t lda,
                                    const double *B, int64_t ldb, double *C, int64_t ldc, int lower, void *stream);

/* ------------------------------------------------------- autotuner */

/* Tile choices per problem-size bucket: bucket b holds n <= 512 * 2^b
 * (b = 0..7), bucket 8 larger n. */
#define GPCH_TUNE_BUCKETS 9

typedef struct gpch_tune_info {
    int32_t source;                              /* 0 defaults, 1 measured, 2 loaded */
    int32_t refined_tile[GPCH_TUNE_BUCKETS];     /* gpch_solve_refined with tile = 0 */
    int32_t batch_tile_fp64[GPCH_TUNE_BUCKETS];  /* trailing-update tile, FP64 batch  */
    int32_t batch_tile_mixed[GPCH_TUNE_BUCKETS]; /* trailing-update tile, mixed batch */
    char gpu[96];                                /* device name the table belongs to */
} gpch_tune_info;

/* Tile choices for the context's device (the block size is a paper
 * parameter: Sec. 4 studies it per system size; no autotuner is in the
 * paper).  Unless `force` is set, the table is loaded from cache_path
 * (JSON, keyed by the GPU's name) when the file holds an entry for this
 * device; otherwise every candidate is timed with CUDA events on synthetic
 * squared-exponential systems generated on the device and the fastest
 * kept:
 *   - refined solve (split-f16): tiles 256, 384, 512 at n = 1024 ... nmax
 *     (powers of two; nmax <= 65536, default 32768 when 0);
 *   - batched FP64 and mixed solves: trailing-update tile 32 or 64, batches
 *     of one size at n = 256 ... 4096 (the batched result does not depend
 *     on it).
 * Buckets not measured take the nearest measured one.  The table then
 * applies to every context on this device in this process and, when
 * cache_path is not NULL, is written there (other GPUs' entries kept).
 * Measurement allocates its own device memory (about 17 n^2 bytes at the
 * largest n) and takes a few seconds.  out (host, may be NULL) receives the
 * table.  Synchronizes the device.  Errors: INVALID_ARG (nmax), CUDA_ERROR,
 * OOM_BUDGET (allocation failed). */
gpch_status gpch_autotune(gpch_ctx *ctx, const char *cache_path, int force, int64_t nmax, gpch_tune_info *out);

/* The table in effect for the context's device (defaults, measured or
 * loaded). */
gpch_status gpch_tune_get(gpch_ctx *ctx, gpch_tune_info *out);

#ifdef __cplusplus
}
#endif

#endif /* GPCHOL_H */
