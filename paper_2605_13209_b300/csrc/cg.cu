// cg.cu -- A6/A7: conjugate gradients, Algorithm 1 (left), with residual
// replacement every R iterations (Sec. 2.1), for up to 16 right-hand sides
// that share one pass over the matrix per iteration.
//
// Per iteration three kernels run:
//   matvec  t = A s and the partial sums of s^T t; the last CTA to finish
//           reduces the partials in a fixed order and sets alpha = u / s^T t
//   update  x += alpha s, r -= alpha t, partial sums of r^T r; the last CTA
//           sets beta = u_new / u, u = u_new and retires converged columns
//   dir     s = r + beta s
// On a replacement iteration `update` is split into x += alpha s, a matvec
// of x, and r = b - A x.  All scalars stay on the device; the host reads
// one "all done" word every few iterations.  Reductions are two-phase with
// a fixed order, so results do not depend on CTA scheduling.
//
// The matvec uses A = A^T: t_j = sum_i A_ij s_i is a dot product down column
// j, which is contiguous in column-major storage.  A CTA owns W consecutive
// columns and walks all rows; each thread keeps the s values of its rows in
// registers and reuses them across the W columns and NR right-hand sides.

#include "dense_fp64.cuh"

namespace {

constexpr int THREADS = 256;
constexpr int ROWS_PER_THREAD = 2;
constexpr int MAXRHS = 16;

struct CGState {
    double *u, *u0, *alpha, *beta;   // [MAXRHS]
    int *active, *iters;            // [MAXRHS]
    int *done;                      // [1]
    unsigned *counter;              // [2]: matvec, update
    double *part;                   // per-CTA partials, part_doubles(n, nrhs)
};

__device__ inline double warp_sum(double v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Last-CTA election for a two-phase reduction: every CTA has written its
// partials; returns true in exactly one CTA, after which all partials are
// visible to it.
__device__ inline bool last_cta(unsigned *counter)
{
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned ticket = atomicAdd(counter, 1u);
        is_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (is_last) __threadfence();
    return is_last;
}

template <typename TA, int W, int NR>
__global__ void __launch_bounds__(THREADS) cg_matvec_kernel(int64_t n, int nrhs, const TA *__restrict__ A,
                                                            int64_t lda, const double *__restrict__ S,
                                                            int64_t lds, double *T, int64_t ldt, CGState st,
                                                            int mode)
{
    // mode 0: t = A s, then alpha; mode 1: t = A s only (s is x here)
    __shared__ double red[THREADS / 32][W * NR];
    __shared__ double tcol[W * NR];
    if (*st.done) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t j0 = (int64_t)blockIdx.x * W;
    const int wcols = (int)((n - j0 < W) ? n - j0 : W);
    double acc[W][NR];
#pragma unroll
    for (int c = 0; c < W; ++c)
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[c][r] = 0.0;

    for (int64_t base = 0; base < n; base += (int64_t)THREADS * ROWS_PER_THREAD) {
        double sv[ROWS_PER_THREAD][NR];
        int64_t rows[ROWS_PER_THREAD];
#pragma unroll
        for (int q = 0; q < ROWS_PER_THREAD; ++q) {
            rows[q] = base + tid + (int64_t)q * THREADS;
#pragma unroll
            for (int r = 0; r < NR; ++r)
                sv[q][r] = (rows[q] < n && r < nrhs) ? S[rows[q] + r * lds] : 0.0;
        }
#pragma unroll
        for (int c = 0; c < W; ++c) {
            if (c < wcols) {
#pragma unroll
                for (int q = 0; q < ROWS_PER_THREAD; ++q) {
                    if (rows[q] < n) {
                        const double a = (double)A[rows[q] + (j0 + c) * lda];
#pragma unroll
                        for (int r = 0; r < NR; ++r) acc[c][r] = fma(a, sv[q][r], acc[c][r]);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int c = 0; c < W; ++c)
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            double v = warp_sum(acc[c][r]);
            if (lane == 0) red[warp][c * NR + r] = v;
        }
    __syncthreads();
    if (tid < W * NR) {
        double v = 0.0;
#pragma unroll
        for (int w = 0; w < THREADS / 32; ++w) v += red[w][tid];
        tcol[tid] = v;
        const int c = tid / NR, r = tid % NR;
        if (c < wcols && r < nrhs) T[(j0 + c) + r * ldt] = v;
    }
    if (mode != 0) return;
    __syncthreads();
    if (tid < NR) {
        double p = 0.0;
        for (int c = 0; c < wcols; ++c)
            if (tid < nrhs) p = fma(S[(j0 + c) + tid * lds], tcol[c * NR + tid], p);
        st.part[(size_t)blockIdx.x * NR + tid] = p;
    }
    if (last_cta(&st.counter[0])) {
        // every thread sums a fixed strided subset of the CTA partials, then
        // one block reduction (a fixed order, so the result is reproducible)
        for (int r = 0; r < nrhs; ++r) {
            double p = 0.0;
            for (unsigned b = tid; b < gridDim.x; b += THREADS) p += __ldcg(&st.part[(size_t)b * NR + r]);
            p = warp_sum(p);
            if (lane == 0) red[warp][0] = p;
            __syncthreads();
            if (tid == 0) {
                double q = 0.0;
                for (int w = 0; w < THREADS / 32; ++w) q += red[w][0];
                st.alpha[r] = st.active[r] ? st.u[r] / q : 0.0;
            }
            __syncthreads();
        }
        if (tid == 0) st.counter[0] = 0;
    }
}

// Tail of update/replace: reduce r^T r partials, set beta, retire columns.
__device__ inline void finish_rr(CGState st, int nrhs, double rtol2, int maxit, bool count_iter)
{
    const int tid = threadIdx.x;
    if (last_cta(&st.counter[1])) {
        __shared__ int any_active;
        if (tid == 0) any_active = 0;
        __syncthreads();
        if (tid < nrhs && st.active[tid]) {
            double un = 0.0;
            for (unsigned b = 0; b < gridDim.x; ++b) un += __ldcg(&st.part[(size_t)b * MAXRHS + tid]);
            st.beta[tid] = un / st.u[tid];
            st.u[tid] = un;
            int it = st.iters[tid] + (count_iter ? 1 : 0);
            st.iters[tid] = it;
            if (un <= rtol2 * st.u0[tid] || it >= maxit) st.active[tid] = 0;
            else atomicOr(&any_active, 1);
        }
        __syncthreads();
        if (tid == 0) {
            if (!any_active) *st.done = 1;
            st.counter[1] = 0;
        }
    }
}

// x += alpha s; r -= alpha t (or, with replace, r = b - t where t = A x and
// x was already updated); partial r^T r per CTA.
__global__ void __launch_bounds__(THREADS) cg_update_kernel(int64_t n, int nrhs, double *X, int64_t ldx,
                                                            double *R, const double *S, const double *T,
                                                            const double *B, int64_t ldb, int64_t ldv,
                                                            CGState st, double rtol2, int maxit, int replace)
{
    __shared__ double red[THREADS / 32][MAXRHS];
    if (*st.done) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t i = (int64_t)blockIdx.x * THREADS + tid;
    for (int r = 0; r < nrhs; ++r) {
        double rr = 0.0;
        if (st.active[r] && i < n) {
            double ri;
            if (replace) {
                ri = B[i + r * ldb] - T[i + r * ldv];
            } else {
                const double a = st.alpha[r];
                X[i + r * ldx] = fma(a, S[i + r * ldv], X[i + r * ldx]);
                ri = fma(-a, T[i + r * ldv], R[i + r * ldv]);
            }
            R[i + r * ldv] = ri;
            rr = ri * ri;
        }
        rr = warp_sum(rr);
        if (lane == 0) red[warp][r] = rr;
    }
    __syncthreads();
    if (tid < nrhs) {
        double v = 0.0;
        for (int w = 0; w < THREADS / 32; ++w) v += red[w][tid];
        st.part[(size_t)blockIdx.x * MAXRHS + tid] = v;
    }
    finish_rr(st, nrhs, rtol2, maxit, true);
}

// x += alpha s only (first half of a replacement iteration).
__global__ void __launch_bounds__(THREADS) cg_xupdate_kernel(int64_t n, int nrhs, double *X, int64_t ldx,
                                                             const double *S, int64_t ldv, CGState st)
{
    if (*st.done) return;
    const int64_t i = (int64_t)blockIdx.x * THREADS + threadIdx.x;
    if (i >= n) return;
    for (int r = 0; r < nrhs; ++r)
        if (st.active[r]) X[i + r * ldx] = fma(st.alpha[r], S[i + r * ldv], X[i + r * ldx]);
}

__global__ void __launch_bounds__(THREADS) cg_dir_kernel(int64_t n, int nrhs, const double *R, double *S,
                                                         int64_t ldv, CGState st)
{
    if (*st.done) return;
    const int64_t i = (int64_t)blockIdx.x * THREADS + threadIdx.x;
    if (i >= n) return;
    for (int r = 0; r < nrhs; ++r)
        if (st.active[r]) S[i + r * ldv] = fma(st.beta[r], S[i + r * ldv], R[i + r * ldv]);
}

// r = b - t (t = A x0), s = r, partial r^T r; last CTA sets u = u0 and the
// initial active flags.
__global__ void __launch_bounds__(THREADS) cg_init_kernel(int64_t n, int nrhs, double *R, double *S,
                                                          const double *T, const double *B, int64_t ldb,
                                                          int64_t ldv, CGState st)
{
    __shared__ double red[THREADS / 32][MAXRHS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t i = (int64_t)blockIdx.x * THREADS + tid;
    for (int r = 0; r < nrhs; ++r) {
        double rr = 0.0;
        if (i < n) {
            double ri = B[i + r * ldb] - T[i + r * ldv];
            R[i + r * ldv] = ri;
            S[i + r * ldv] = ri;
            rr = ri * ri;
        }
        rr = warp_sum(rr);
        if (lane == 0) red[warp][r] = rr;
    }
    __syncthreads();
    if (tid < nrhs) {
        double v = 0.0;
        for (int w = 0; w < THREADS / 32; ++w) v += red[w][tid];
        st.part[(size_t)blockIdx.x * MAXRHS + tid] = v;
    }
    if (last_cta(&st.counter[1])) {
        __shared__ int any_active;
        if (tid == 0) any_active = 0;
        __syncthreads();
        if (tid < nrhs) {
            double u = 0.0;
            for (unsigned b = 0; b < gridDim.x; ++b) u += __ldcg(&st.part[(size_t)b * MAXRHS + tid]);
            st.u[tid] = u;
            st.u0[tid] = u;
            st.iters[tid] = 0;
            st.active[tid] = u > 0.0 ? 1 : 0;
            if (u > 0.0) atomicOr(&any_active, 1);
        }
        __syncthreads();
        if (tid == 0) {
            *st.done = any_active ? 0 : 1;
            st.counter[1] = 0;
        }
    }
}

template <typename TA>
gpch_status launch_matvec(gpch_ctx *ctx, int64_t n, int nrhs, const TA *A, int64_t lda, const double *S,
                          int64_t lds, double *T, int64_t ldt, const CGState &st, int mode, cudaStream_t s)
{
    gpch::PhaseScope ph(ctx, GPCH_PHASE_CG_MATVEC, s,
                        (double)n * n * sizeof(TA) + 2.0 * (double)n * nrhs * sizeof(double));
#define GPCH_MV(Wc, NRc)                                                                         \
    cg_matvec_kernel<TA, Wc, NRc><<<(unsigned)((n + Wc - 1) / Wc), THREADS, 0, s>>>(n, nrhs, A, lda, S, \
                                                                                    lds, T, ldt, st, mode)
    // narrow column blocks make many CTAs (n / 4 for one right-hand side), so
    // the last partial wave of CTAs is a small share of the launch
    if (nrhs <= 1) GPCH_MV(4, 1);
    else if (nrhs <= 2) GPCH_MV(8, 2);
    else if (nrhs <= 4) GPCH_MV(4, 4);
    else if (nrhs <= 8) GPCH_MV(2, 8);
    else GPCH_MV(2, 16);
#undef GPCH_MV
    GPCH_LAUNCH_CHECK(ctx);
    return GPCH_OK;
}

inline int mv_width(int nrhs) { return nrhs <= 1 ? 4 : nrhs <= 2 ? 8 : nrhs <= 4 ? 4 : 2; }
inline int mv_nr(int nrhs) { return nrhs <= 1 ? 1 : nrhs <= 2 ? 2 : nrhs <= 4 ? 4 : nrhs <= 8 ? 8 : 16; }

// Loads every kernel cg_run may launch on the current device.  Under lazy
// module loading a kernel's code is placed in device memory at its first
// launch; asking for its attributes loads it ahead of time.
template <typename TA>
cudaError_t cg_kernels_load()
{
    cudaFuncAttributes a;
    const void *fns[] = {(const void *)cg_matvec_kernel<TA, 4, 1>, (const void *)cg_matvec_kernel<TA, 8, 2>,
                         (const void *)cg_matvec_kernel<TA, 4, 4>, (const void *)cg_matvec_kernel<TA, 2, 8>,
                         (const void *)cg_matvec_kernel<TA, 2, 16>, (const void *)cg_init_kernel,
                         (const void *)cg_update_kernel,           (const void *)cg_xupdate_kernel,
                         (const void *)cg_dir_kernel};
    for (const void *f : fns) {
        cudaError_t e = cudaFuncGetAttributes(&a, f);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Doubles of per-CTA partials: the matvec stores mv_nr per CTA, the vector
// kernels (one CTA per THREADS rows) up to 2 * MAXRHS.
inline size_t part_doubles(int64_t n, int nrhs)
{
    const size_t mv = (size_t)((n + mv_width(nrhs) - 1) / mv_width(nrhs)) * mv_nr(nrhs);
    const size_t vec = (size_t)((n + THREADS - 1) / THREADS) * 3 * MAXRHS;
    return mv > vec ? mv : vec;
}

// Bytes of scratch one CG group of nrhs (<= 16) columns needs.
size_t cg_scratch_bytes(int64_t n, int nrhs)
{
    gpch::Carver dry(nullptr);
    dry.take<double>((size_t)3 * n * nrhs);
    dry.take<double>(4 * MAXRHS);
    dry.take<int>(2 * MAXRHS + 1);
    dry.take<unsigned>(2);
    dry.take<double>(part_doubles(n, nrhs));
    return dry.off;
}

// One CG group on caller-provided scratch (cg_scratch_bytes(n, nrhs) bytes
// of device memory at `scratch`) and a host staging block `hbuf` of at
// least 64 + 4*16*8 + 33*4 bytes (pinned or pageable).
template <typename TA>
gpch_status cg_run(gpch_ctx *ctx, int64_t n, const TA *A, int64_t lda, const double *B, int64_t ldb, double *X,
                   int64_t ldx, int nrhs, double rtol, int maxit, int R, cudaStream_t s, void *scratch, void *hbuf,
                   int *h_iters, double *h_relres)
{
    const int64_t ldv = n;
    const unsigned vec_ctas = (unsigned)((n + THREADS - 1) / THREADS);
    gpch::Carver cv(scratch);
    double *Rv = cv.take<double>((size_t)n * nrhs);
    double *Sv = cv.take<double>((size_t)n * nrhs);
    double *Tv = cv.take<double>((size_t)n * nrhs);
    CGState st;
    double *sc = cv.take<double>(4 * MAXRHS);
    st.u = sc;
    st.u0 = sc + MAXRHS;
    st.alpha = sc + 2 * MAXRHS;
    st.beta = sc + 3 * MAXRHS;
    int *ic = cv.take<int>(2 * MAXRHS + 1);
    st.active = ic;
    st.iters = ic + MAXRHS;
    st.done = ic + 2 * MAXRHS;
    st.counter = cv.take<unsigned>(2);
    st.part = cv.take<double>(part_doubles(n, nrhs));
    GPCH_CUDA(ctx, cudaMemsetAsync(st.counter, 0, 2 * sizeof(unsigned), s));
    GPCH_CUDA(ctx, cudaMemsetAsync(ic, 0, (2 * MAXRHS + 1) * sizeof(int), s));

    // line 1: s = r = b - A x
    GPCH_CHECK(launch_matvec<TA>(ctx, n, nrhs, A, lda, X, ldx, Tv, ldv, st, 1, s));
    cg_init_kernel<<<vec_ctas, THREADS, 0, s>>>(n, nrhs, Rv, Sv, Tv, B, ldb, ldv, st);
    GPCH_LAUNCH_CHECK(ctx);

    int *h_done = static_cast<int *>(hbuf);
    const double rtol2 = rtol * rtol;
    const int chunk = 16;
    int it = 0;
    while (it < maxit) {
        const int k = (maxit - it < chunk) ? maxit - it : chunk;
        for (int q = 0; q < k; ++q) {
            const int iter = it + q + 1;   // 1-based number of the iteration being run
            GPCH_CHECK(launch_matvec<TA>(ctx, n, nrhs, A, lda, Sv, ldv, Tv, ldv, st, 0, s));
            gpch::PhaseScope phv(ctx, GPCH_PHASE_CG_VECTOR, s, 9.0 * (double)n * nrhs * sizeof(double));
            if (R > 0 && iter % R == 0) {
                cg_xupdate_kernel<<<vec_ctas, THREADS, 0, s>>>(n, nrhs, X, ldx, Sv, ldv, st);
                GPCH_LAUNCH_CHECK(ctx);
                GPCH_CHECK(launch_matvec<TA>(ctx, n, nrhs, A, lda, X, ldx, Tv, ldv, st, 1, s));
                cg_update_kernel<<<vec_ctas, THREADS, 0, s>>>(n, nrhs, X, ldx, Rv, Sv, Tv, B, ldb, ldv, st, rtol2,
                                                              maxit, 1);
            } else {
                cg_update_kernel<<<vec_ctas, THREADS, 0, s>>>(n, nrhs, X, ldx, Rv, Sv, Tv, B, ldb, ldv, st, rtol2,
                                                              maxit, 0);
            }
            GPCH_LAUNCH_CHECK(ctx);
            cg_dir_kernel<<<vec_ctas, THREADS, 0, s>>>(n, nrhs, Rv, Sv, ldv, st);
            GPCH_LAUNCH_CHECK(ctx);
        }
        it += k;
        GPCH_CUDA(ctx, cudaMemcpyAsync(h_done, st.done, sizeof(int), cudaMemcpyDeviceToHost, s));
        GPCH_CUDA(ctx, cudaStreamSynchronize(s));
        if (*h_done) break;
    }
    // statistics
    double *h_sc = reinterpret_cast<double *>(static_cast<char *>(hbuf) + 64);
    int *h_ic = reinterpret_cast<int *>(static_cast<char *>(hbuf) + 64 + 4 * MAXRHS * sizeof(double));
    GPCH_CUDA(ctx, cudaMemcpyAsync(h_sc, sc, 4 * MAXRHS * sizeof(double), cudaMemcpyDeviceToHost, s));
    GPCH_CUDA(ctx, cudaMemcpyAsync(h_ic, ic, (2 * MAXRHS + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
    GPCH_CUDA(ctx, cudaStreamSynchronize(s));
    for (int r = 0; r < nrhs; ++r) {
        h_iters[r] = h_ic[MAXRHS + r];
        const double u = h_sc[r], u0 = h_sc[MAXRHS + r];
        h_relres[r] = u0 > 0.0 ? sqrt(u / u0) : 0.0;
    }
    return GPCH_OK;
}

// One CG group on the context's workspace arena and pinned block.
template <typename TA>
gpch_status cg_group(gpch_ctx *ctx, int64_t n, const TA *A, int64_t lda, const double *B, int64_t ldb,
                     double *X, int64_t ldx, int nrhs, double rtol, int maxit, int R, cudaStream_t s,
                     int *h_iters, double *h_relres)
{
    GPCH_CHECK(gpch::ws_reserve(ctx, cg_scratch_bytes(n, nrhs)));
    return cg_run<TA>(ctx, n, A, lda, B, ldb, X, ldx, nrhs, rtol, maxit, R, s, ctx->ws, ctx->pinned, h_iters,
                      h_relres);
}

// ------------------------------------------------------------ PCG (A9)
//
// Refined solve: preconditioned CG with M = Lt Lt^T, Lt the low-precision
// factor (FP32 storage), applied by the forward/back substitution of
// solve.cu.  A, x, r, dot products and recurrences stay in FP64.  The host
// reads a few scalars per iteration (an iteration already costs two
// substitution sweeps), decides when to replace the recurrence residual by
// the true one, and stops each column when its true backward error
// ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf) meets the tolerance.

// x += alpha s, r -= alpha t on active columns; per-CTA sum of r^2 and max
// |x|; the last CTA stores rr[c] and xinf[c].
__global__ void __launch_bounds__(THREADS) pcg_update_kernel(int64_t n, int nrhs, double *X, int64_t ldx, double *R,
                                                             const double *S, const double *T, int64_t ldv,
                                                             CGState st, double *rr_out, double *xinf_out,
                                                             double *rinf_out)
{
    __shared__ double red[THREADS / 32][3 * MAXRHS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t i = (int64_t)blockIdx.x * THREADS + tid;
    for (int r = 0; r < nrhs; ++r) {
        double rr = 0.0, xm = 0.0, rm = 0.0;
        if (st.active[r] && i < n) {
            const double a = st.alpha[r];
            const double xi = fma(a, S[i + r * ldv], X[i + r * ldx]);
            X[i + r * ldx] = xi;
            const double ri = fma(-a, T[i + r * ldv], R[i + r * ldv]);
            R[i + r * ldv] = ri;
            rr = ri * ri;
            xm = fabs(xi);
            rm = fabs(ri);
        }
        rr = warp_sum(rr);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            xm = fmax(xm, __shfl_xor_sync(0xffffffffu, xm, off));
            rm = fmax(rm, __shfl_xor_sync(0xffffffffu, rm, off));
        }
        if (lane == 0) {
            red[warp][r] = rr;
            red[warp][MAXRHS + r] = xm;
            red[warp][2 * MAXRHS + r] = rm;
        }
    }
    __syncthreads();
    if (tid < nrhs) {
        double v = 0.0, m = 0.0, q = 0.0;
        for (int w = 0; w < THREADS / 32; ++w) {
            v += red[w][tid];
            m = fmax(m, red[w][MAXRHS + tid]);
            q = fmax(q, red[w][2 * MAXRHS + tid]);
        }
        st.part[(size_t)blockIdx.x * 3 * MAXRHS + tid] = v;
        st.part[(size_t)blockIdx.x * 3 * MAXRHS + MAXRHS + tid] = m;
        st.part[(size_t)blockIdx.x * 3 * MAXRHS + 2 * MAXRHS + tid] = q;
    }
    if (last_cta(&st.counter[1])) {
        if (tid < nrhs) {
            double v = 0.0, m = 0.0, q = 0.0;
            for (unsigned b = 0; b < gridDim.x; ++b) {
                v += __ldcg(&st.part[(size_t)b * 3 * MAXRHS + tid]);
                m = fmax(m, __ldcg(&st.part[(size_t)b * 3 * MAXRHS + MAXRHS + tid]));
                q = fmax(q, __ldcg(&st.part[(size_t)b * 3 * MAXRHS + 2 * MAXRHS + tid]));
            }
            rr_out[tid] = v;
            xinf_out[tid] = m;
            rinf_out[tid] = q;
        }
        if (tid == 0) st.counter[1] = 0;
    }
}

// r = b - t (t = A x) on active columns; per-column max |r| and max |x|.
__global__ void __launch_bounds__(THREADS) pcg_replace_kernel(int64_t n, int nrhs, const double *X, int64_t ldx,
                                                              double *R, const double *T, const double *B,
                                                              int64_t ldb, int64_t ldv, CGState st, double *rinf,
                                                              double *xinf)
{
    __shared__ double red[THREADS / 32][2 * MAXRHS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t i = (int64_t)blockIdx.x * THREADS + tid;
    for (int r = 0; r < nrhs; ++r) {
        double rm = 0.0, xm = 0.0;
        if (st.active[r] && i < n) {
            const double ri = B[i + r * ldb] - T[i + r * ldv];
            R[i + r * ldv] = ri;
            rm = fabs(ri);
            xm = fabs(X[i + r * ldx]);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            rm = fmax(rm, __shfl_xor_sync(0xffffffffu, rm, off));
            xm = fmax(xm, __shfl_xor_sync(0xffffffffu, xm, off));
        }
        if (lane == 0) {
            red[warp][r] = rm;
            red[warp][MAXRHS + r] = xm;
        }
    }
    __syncthreads();
    if (tid < nrhs) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < THREADS / 32; ++w) {
            a = fmax(a, red[w][tid]);
            b = fmax(b, red[w][MAXRHS + tid]);
        }
        st.part[(size_t)blockIdx.x * 2 * MAXRHS + tid] = a;
        st.part[(size_t)blockIdx.x * 2 * MAXRHS + MAXRHS + tid] = b;
    }
    if (last_cta(&st.counter[1])) {
        if (tid < nrhs) {
            double a = 0.0, b = 0.0;
            for (unsigned blk = 0; blk < gridDim.x; ++blk) {
                a = fmax(a, __ldcg(&st.part[(size_t)blk * 2 * MAXRHS + tid]));
                b = fmax(b, __ldcg(&st.part[(size_t)blk * 2 * MAXRHS + MAXRHS + tid]));
            }
            rinf[tid] = a;
            xinf[tid] = b;
        }
        if (tid == 0) st.counter[1] = 0;
    }
}

// out[c] = U_c^T V_c for every column; with set_beta, beta = out / u and
// u = out on active columns (u starts as out when init is set).
__global__ void __launch_bounds__(THREADS) pcg_dot_kernel(int64_t n, int nrhs, const double *U, int64_t ldu,
                                                          const double *V, int64_t ldv, CGState st, double *out,
                                                          int mode)
{
    // mode 0: store only; 1: u = out (init); 2: beta = out / u, u = out
    __shared__ double red[THREADS / 32][MAXRHS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t i = (int64_t)blockIdx.x * THREADS + tid;
    for (int r = 0; r < nrhs; ++r) {
        double p = (i < n) ? U[i + r * ldu] * V[i + r * ldv] : 0.0;
        p = warp_sum(p);
        if (lane == 0) red[warp][r] = p;
    }
    __syncthreads();
    if (tid < nrhs) {
        double v = 0.0;
        for (int w = 0; w < THREADS / 32; ++w) v += red[w][tid];
        st.part[(size_t)blockIdx.x * 2 * MAXRHS + tid] = v;
    }
    if (last_cta(&st.counter[1])) {
        if (tid < nrhs) {
            double v = 0.0;
            for (unsigned b = 0; b < gridDim.x; ++b) v += __ldcg(&st.part[(size_t)b * 2 * MAXRHS + tid]);
            out[tid] = v;
            if (mode == 1) st.u[tid] = v;
            if (mode == 2 && st.active[tid]) {
                st.beta[tid] = v / st.u[tid];
                st.u[tid] = v;
            }
        }
        if (tid == 0) st.counter[1] = 0;
    }
}

// Order-independent maxima of non-negative doubles through their bit
// patterns (which order like the values).
__device__ inline void atomic_max_nonneg(double *addr, double v)
{
    atomicMax(reinterpret_cast<unsigned long long *>(addr), (unsigned long long)__double_as_longlong(v));
}

// *out = max(0, max_i A_ii).
__global__ void __launch_bounds__(THREADS) diag_max_kernel(int64_t n, const double *__restrict__ A, int64_t lda,
                                                           double *out)
{
    double m = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * THREADS)
        m = fmax(m, A[i + i * lda]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(out, m);
}

// out[c] = max_i |V_ic|.
__global__ void __launch_bounds__(THREADS) absmax_cols_kernel(int64_t n, int nrhs, const double *V, int64_t ldv,
                                                              double *out)
{
    const int64_t i = (int64_t)blockIdx.x * THREADS + threadIdx.x;
    for (int r = 0; r < nrhs; ++r) {
        double m = (i < n) ? fabs(V[i + r * ldv]) : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
        if ((threadIdx.x & 31) == 0) atomic_max_nonneg(&out[r], m);
    }
}

struct RefineResult {
    int iterations = 0;
    double bwd[MAXRHS] = {0};
};

// PCG on one group of <= 16 right-hand sides.  L: FP32 factor (ldl);
// anorm_dev: ||A||_inf on the device (from mixed_init_enqueue).
gpch_status pcg_group(gpch_ctx *ctx, int64_t n, const double *A, int64_t lda, const float *L, int64_t ldl,
                      const double *B, int64_t ldb, double *X, int64_t ldx, int nrhs, double bwd_tol, int maxit,
                      int R, char *wsbase, cudaStream_t s, RefineResult &res, const double *anorm_dev)
{
    const int64_t ldv = n;
    const unsigned vec_ctas = (unsigned)((n + THREADS - 1) / THREADS);
    gpch::Carver cv(wsbase);
    double *Rv = cv.take<double>((size_t)n * nrhs);
    double *Zv = cv.take<double>((size_t)n * nrhs);
    double *Sv = cv.take<double>((size_t)n * nrhs);
    double *Tv = cv.take<double>((size_t)n * nrhs);
    char *solve_base = cv.take<char>(gpch::solve_ws_bytes(n, nrhs));
    gpch::SolveWs sw = gpch::carve_solve(solve_base, n, nrhs);
    CGState st;
    double *sc = cv.take<double>(4 * MAXRHS);
    st.u = sc;
    st.u0 = sc + MAXRHS;
    st.alpha = sc + 2 * MAXRHS;
    st.beta = sc + 3 * MAXRHS;
    int *ic = cv.take<int>(2 * MAXRHS + 1);
    st.active = ic;
    st.iters = ic + MAXRHS;
    st.done = ic + 2 * MAXRHS;
    st.counter = cv.take<unsigned>(2);
    st.part = cv.take<double>(part_doubles(n, nrhs));
    // ex: rr[16] xinf[16] rinf[16] binf[16] bb[16] norms[2] dots[16]
    double *ex = cv.take<double>(6 * MAXRHS + 2);
    double *d_rr = ex, *d_xinf = ex + MAXRHS, *d_rinf = ex + 2 * MAXRHS, *d_binf = ex + 3 * MAXRHS;
    double *d_bb = ex + 4 * MAXRHS, *d_norms = ex + 5 * MAXRHS, *d_dots = ex + 5 * MAXRHS + 2;

    // host mirror in the pinned block: [0, 6*16+2) doubles, then ints
    double *h = static_cast<double *>(ctx->pinned);
    int *h_active = reinterpret_cast<int *>(h + 6 * MAXRHS + 2);

    GPCH_CUDA(ctx, cudaMemsetAsync(st.counter, 0, 2 * sizeof(unsigned), s));
    GPCH_CUDA(ctx, cudaMemsetAsync(ic, 0, (2 * MAXRHS + 1) * sizeof(int), s));
    GPCH_CUDA(ctx, cudaMemsetAsync(ex, 0, (6 * MAXRHS + 2) * sizeof(double), s));
    for (int c = 0; c < MAXRHS; ++c) h_active[c] = c < nrhs ? 1 : 0;
    GPCH_CUDA(ctx, cudaMemcpyAsync(st.active, h_active, MAXRHS * sizeof(int), cudaMemcpyHostToDevice, s));
    // x0 = 0, r = b, z = M^-1 r, s = z, u = r^T z
    for (int c = 0; c < nrhs; ++c) {
        GPCH_CUDA(ctx, cudaMemsetAsync(X + c * ldx, 0, n * sizeof(double), s));
        GPCH_CUDA(ctx, cudaMemcpyAsync(Rv + c * ldv, B + c * ldb, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    // ||A||_inf, made by the pass that built the factor's copy of A
    GPCH_CUDA(ctx, cudaMemcpyAsync(d_norms, anorm_dev, sizeof(double), cudaMemcpyDeviceToDevice, s));
    absmax_cols_kernel<<<vec_ctas, THREADS, 0, s>>>(n, nrhs, B, ldb, d_binf);
    GPCH_LAUNCH_CHECK(ctx);
    pcg_dot_kernel<<<vec_ctas, THREADS, 0, s>>>(n, nrhs, Rv, ldv, Rv, ldv, st, d_bb, 0);
    GPCH_LAUNCH_CHECK(ctx);
    GPCH_CHECK(gpch::solve_prepare_f32(ctx, n, L, ldl, sw, s));
    GPCH_CUDA(ctx, cudaMemcpyAsync(Zv, Rv, (size_t)n * nrhs * sizeof(double), cudaMemcpyDeviceToDevice, s));
    GPCH_CHECK(gpch::solve_apply_f32(ctx, n, L, ldl, Zv, ldv, nrhs, sw, s));
    GPCH_CUDA(ctx, cudaMemcpyAsync(Sv, Zv, (size_t)n * nrhs * sizeof(double), cudaMemcpyDeviceToDevice, s));
    pcg_dot_kernel<<<vec_ctas, THREADS, 0, s>>>(n, nrhs, Rv, ldv, Zv, ldv, st, d_dots, 1);
    GPCH_LAUNCH_CHECK(ctx);
    GPCH_CUDA(ctx, cudaMemcpyAsync(h, ex, (6 * MAXRHS + 2) * sizeof(double), cudaMemcpyDeviceToHost, s));
    GPCH_CUDA(ctx, cudaStreamSynchronize(s));
    const double anorm = h[5 * MAXRHS];
    double binf[MAXRHS], bb[MAXRHS];
    for (int c = 0; c < MAXRHS; ++c) {
        binf[c] = h[3 * MAXRHS + c];
        bb[c] = h[4 * MAXRHS + c];
        res.bwd[c] = c < nrhs ? (binf[c] > 0.0 ? 1.0 : 0.0) : 0.0;
        if (c < nrhs && binf[c] == 0.0) h_active[c] = 0;   // b = 0: x = 0 is exact
    }
    GPCH_CUDA(ctx, cudaMemcpyAsync(st.active, h_active, MAXRHS * sizeof(int), cudaMemcpyHostToDevice, s));
    int nactive = 0;
    for (int c = 0; c < nrhs; ++c) nactive += h_active[c];
    const double eps2 = 1e-30;
    // The recurrence residual's ||r||_inf gives the backward-error estimate;
    // the true residual b - A x is computed once that estimate, scaled by the
    // ratio of truth to estimate seen at the last failed check, meets tol.
    double ratio[MAXRHS];
    for (int c = 0; c < MAXRHS; ++c) ratio[c] = 1.0;
    double est_at_check[MAXRHS] = {0};
    int it = 0;
    while (nactive > 0 && it < maxit) {
        GPCH_CHECK(launch_matvec<double>(ctx, n, nrhs, A, lda, Sv, ldv, Tv, ldv, st, 0, s));
        pcg_update_kernel<<<vec_ctas, THREADS, 0, s>>>(n, nrhs, X, ldx, Rv, Sv, Tv, ldv, st, d_rr, d_xinf, d_rinf);
        GPCH_LAUNCH_CHECK(ctx);
        ++it;
        GPCH_CUDA(ctx, cudaMemcpyAsync(h, ex, 3 * MAXRHS * sizeof(double), cudaMemcpyDeviceToHost, s));
        GPCH_CUDA(ctx, cudaStreamSynchronize(s));
        bool replace = (R > 0 && it % R == 0);
        for (int c = 0; c < nrhs; ++c) {
            if (!h_active[c]) continue;
            const double est = h[2 * MAXRHS + c] / (anorm * h[MAXRHS + c] + binf[c]);
            est_at_check[c] = est;
            if (est * ratio[c] <= bwd_tol || h[c] <= eps2 * bb[c]) replace = true;
        }
        if (replace) {
            GPCH_CHECK(launch_matvec<double>(ctx, n, nrhs, A, lda, X, ldx, Tv, ldv, st, 1, s));
            pcg_replace_kernel<<<vec_ctas, THREADS, 0, s>>>(n, nrhs, X, ldx, Rv, Tv, B, ldb, ldv, st, d_rinf,
                                                            d_xinf);
            GPCH_LAUNCH_CHECK(ctx);
            GPCH_CUDA(ctx, cudaMemcpyAsync(h, ex, 3 * MAXRHS * sizeof(double), cudaMemcpyDeviceToHost, s));
            GPCH_CUDA(ctx, cudaStreamSynchronize(s));
            nactive = 0;
            for (int c = 0; c < nrhs; ++c) {
                if (!h_active[c]) continue;
                const double den = anorm * h[MAXRHS + c] + binf[c];
                res.bwd[c] = den > 0.0 ? h[2 * MAXRHS + c] / den : 0.0;
                if (res.bwd[c] <= bwd_tol) h_active[c] = 0;
                else if (est_at_check[c] > 0.0 && res.bwd[c] / est_at_check[c] > ratio[c])
                    ratio[c] = res.bwd[c] / est_at_check[c];
                nactive += h_active[c];
            }
            GPCH_CUDA(ctx, cudaMemcpyAsync(st.active, h_active, MAXRHS * sizeof(int), cudaMemcpyHostToDevice, s));
            if (nactive == 0) break;
        }
        GPCH_CUDA(ctx, cudaMemcpyAsync(Zv, Rv, (size_t)n * nrhs * sizeof(double), cudaMemcpyDeviceToDevice, s));
        GPCH_CHECK(gpch::solve_apply_f32(ctx, n, L, ldl, Zv, ldv, nrhs, sw, s));
        pcg_dot_kernel<<<vec_ctas, THREADS, 0, s>>>(n, nrhs, Rv, ldv, Zv, ldv, st, d_dots, 2);
        GPCH_LAUNCH_CHECK(ctx);
        cg_dir_kernel<<<vec_ctas, THREADS, 0, s>>>(n, nrhs, Zv, Sv, ldv, st);
        GPCH_LAUNCH_CHECK(ctx);
    }
    res.iterations = it;
    int *h_err = reinterpret_cast<int *>(h_active + MAXRHS);
    GPCH_CUDA(ctx, cudaMemcpyAsync(h_err, sw.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    GPCH_CUDA(ctx, cudaStreamSynchronize(s));
    if (*h_err != 0) return gpch::fail(ctx, GPCH_TIMEOUT, "substitution sweep wait gave up");
    return GPCH_OK;
}

size_t pcg_ws_bytes(int64_t n, int nrhs)
{
    gpch::Carver dry(nullptr);
    for (int i = 0; i < 4; ++i) dry.take<double>((size_t)n * nrhs);
    dry.take<char>(gpch::solve_ws_bytes(n, nrhs));
    dry.take<double>(4 * MAXRHS);
    dry.take<int>(2 * MAXRHS + 1);
    dry.take<unsigned>(2);
    dry.take<double>(part_doubles(n, nrhs));
    dry.take<double>(6 * MAXRHS + 2);
    return dry.off;
}

// max_i A_ii (for the shift schedule), synchronously.
gpch_status diag_max(gpch_ctx *ctx, int64_t n, const double *A, int64_t lda, double *dev2, cudaStream_t s,
                     double *out)
{
    GPCH_CUDA(ctx, cudaMemsetAsync(dev2, 0, 2 * sizeof(double), s));
    diag_max_kernel<<<(unsigned)((n + THREADS - 1) / THREADS < 148 ? (n + THREADS - 1) / THREADS : 148), THREADS, 0,
                      s>>>(n, A, lda, dev2 + 1);
    GPCH_LAUNCH_CHECK(ctx);
    double *h = static_cast<double *>(ctx->pinned);
    GPCH_CUDA(ctx, cudaMemcpyAsync(h, dev2, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    GPCH_CUDA(ctx, cudaStreamSynchronize(s));
    *out = h[1];
    return GPCH_OK;
}

}  // namespace

extern "C" gpch_status gpch_cg_solve(gpch_ctx *ctx, int64_t n, const void *A, gpch_dtype dtype, int64_t lda,
                                     const double *B, int64_t ldb, double *X, int64_t ldx, int nrhs, double rtol,
                                     int maxit, int replace_every, void *stream, gpch_cg_stats *stats)
{
    GPCH_ARG(ctx, ctx != nullptr, "null context");
    if (stats) *stats = gpch_cg_stats{0, 0, 0.0};
    GPCH_ARG(ctx, n >= 0 && nrhs >= 0, "n < 0 or nrhs < 0");
    GPCH_ARG(ctx, lda >= (n > 0 ? n : 1) && ldb >= (n > 0 ? n : 1) && ldx >= (n > 0 ? n : 1), "ld < n");
    GPCH_ARG(ctx, dtype == GPCH_F64 || dtype == GPCH_F32, "bad dtype");
    GPCH_ARG(ctx, maxit > 0 && replace_every >= 0 && rtol >= 0.0, "bad maxit / replace_every / rtol");
    if (n == 0 || nrhs == 0) return GPCH_OK;
    GPCH_ARG(ctx, A && B && X, "null pointer");
    GPCH_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    int max_it = 0, conv = 0;
    double rel_max = 0.0;
    for (int r0 = 0; r0 < nrhs; r0 += MAXRHS) {
        const int g = (nrhs - r0 < MAXRHS) ? nrhs - r0 : MAXRHS;
        int iters[MAXRHS];
        double rel[MAXRHS];
        gpch_status st;
        if (dtype == GPCH_F64)
            st = cg_group<double>(ctx, n, static_cast<const double *>(A), lda, B + r0 * ldb, ldb, X + r0 * ldx,
                                  ldx, g, rtol, maxit, replace_every, s, iters, rel);
        else
            st = cg_group<float>(ctx, n, static_cast<const float *>(A), lda, B + r0 * ldb, ldb, X + r0 * ldx,
                                 ldx, g, rtol, maxit, replace_every, s, iters, rel);
        if (st != GPCH_OK) return st;
        for (int r = 0; r < g; ++r) {
            if (iters[r] > max_it) max_it = iters[r];
            if (rel[r] > rel_max) rel_max = rel[r];
            if (rel[r] <= rtol) ++conv;
        }
    }
    if (stats) *stats = gpch_cg_stats{max_it, conv, rel_max};
    if (conv < nrhs)
        return gpch::fail(ctx, GPCH_NOT_CONVERGED, "%d of %d right-hand sides missed rtol within %d iterations",
                          nrhs - conv, nrhs, maxit);
    return GPCH_OK;
}

extern "C" gpch_status gpch_solve_refined(gpch_ctx *ctx, int64_t n, const double *A, int64_t lda, const double *B,
                                          int64_t ldb, double *X, int64_t ldx, int nrhs, gpch_prec prec, int tile,
                                          double bwd_tol, int maxit, void *stream, gpch_refine_stats *stats)
{
    GPCH_ARG(ctx, ctx != nullptr, "null context");
    if (stats) *stats = gpch_refine_stats{0, 0, 0.0, 0.0};
    GPCH_ARG(ctx, n >= 0 && nrhs >= 0, "n < 0 or nrhs < 0");
    GPCH_ARG(ctx, lda >= (n > 0 ? n : 1) && ldb >= (n > 0 ? n : 1) && ldx >= (n > 0 ? n : 1), "ld < n");
    GPCH_ARG(ctx, prec == GPCH_PREC_BF16 || prec == GPCH_PREC_SPLIT_BF16 || prec == GPCH_PREC_SPLIT_F16,
             "prec must be BF16, SPLIT_BF16 or SPLIT_F16");
    GPCH_ARG(ctx, tile >= 64 && tile <= 1024 && tile % 64 == 0, "tile must be a multiple of 64 in [64, 1024]");
    GPCH_ARG(ctx, bwd_tol > 0.0 && maxit > 0, "bad bwd_tol / maxit");
    GPCH_ARG(ctx, n < (int64_t)1 << 31, "n too large");
    if (n == 0 || nrhs == 0) return GPCH_OK;
    GPCH_ARG(ctx, A && B && X, "null pointer");
    GPCH_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t ldw = (n + 31) / 32 * 32;
    const int g = nrhs < MAXRHS ? nrhs : MAXRHS;
    gpch::Carver dry(nullptr);
    dry.take<float>((size_t)ldw * n);
    dry.take<double>(3);
    dry.take<float>(gpch::anorm_ws_floats(n));
    const size_t fixed = dry.off;
    const size_t mix = gpch::mixed_ws_bytes(n, tile), pcg = pcg_ws_bytes(n, g);
    GPCH_CHECK(gpch::ws_reserve(ctx, fixed + 256 + (mix > pcg ? mix : pcg)));
    gpch::Carver cv(ctx->ws);
    float *W = cv.take<float>((size_t)ldw * n);
    double *dev2 = cv.take<double>(3);   // [0, 2): diag_max, [2]: ||A||_inf
    float *norm_ws = cv.take<float>(gpch::anorm_ws_floats(n));
    char *rest = static_cast<char *>(ctx->ws) + ((cv.off + 255) & ~size_t(255));

    double dmax = 0.0;
    GPCH_CHECK(diag_max(ctx, n, A, lda, dev2, s, &dmax));
    // unit roundoff of the step-3 operands: bf16 8 bits, split bf16 ~16 bits,
    // scaled split binary16 ~22 bits
    const double ulow = (prec == GPCH_PREC_BF16) ? 1.0 / 256.0
                        : (prec == GPCH_PREC_SPLIT_BF16) ? 1.0 / 65536.0
                                                         : 1.0 / 4194304.0;
    double shift = (prec == GPCH_PREC_BF16) ? 2.0 * ulow * dmax : 0.0;
    int attempts = 0;
    int64_t info = 1;
    for (; attempts < 9; ++attempts) {
        GPCH_CHECK(gpch::mixed_init_enqueue(ctx, n, A, lda, W, ldw, shift, s, dev2 + 2, norm_ws));
        int64_t *d_info;
        int *d_err;
        GPCH_CHECK(gpch::mixed_factor_enqueue(ctx, n, tile, W, ldw, (int)prec, rest, &d_info, &d_err, s));
        int64_t *h = static_cast<int64_t *>(ctx->pinned);
        GPCH_CUDA(ctx, cudaMemcpyAsync(h, d_info, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        GPCH_CUDA(ctx, cudaMemcpyAsync(h + 1, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
        GPCH_CUDA(ctx, cudaStreamSynchronize(s));
        if (reinterpret_cast<int *>(h + 1)[0] != 0)
            return gpch::fail(ctx, GPCH_TIMEOUT, "tensor-core pipeline wait gave up");
        info = h[0];
        if (info == 0) break;
        const double floor_shift = 2.0 * ulow * dmax;
        shift = (4.0 * shift > floor_shift) ? 4.0 * shift : floor_shift;
    }
    if (stats) {
        stats->factor_attempts = attempts + (info == 0 ? 1 : 0);
        stats->shift = shift;
    }
    if (info != 0)
        return gpch::fail(ctx, GPCH_NOT_SPD, "low-precision factor broke down after %d shifted attempts", attempts);

    int it_max = 0;
    double bwd_max = 0.0;
    bool all_ok = true;
    for (int r0 = 0; r0 < nrhs; r0 += MAXRHS) {
        const int gg = (nrhs - r0 < MAXRHS) ? nrhs - r0 : MAXRHS;
        RefineResult rr;
        GPCH_CHECK(pcg_group(ctx, n, A, lda, W, ldw, B + r0 * ldb, ldb, X + r0 * ldx, ldx, gg, bwd_tol, maxit, 50,
                             rest, s, rr, dev2 + 2));
        if (rr.iterations > it_max) it_max = rr.iterations;
        for (int c = 0; c < gg; ++c) {
            if (rr.bwd[c] > bwd_max) bwd_max = rr.bwd[c];
            if (rr.bwd[c] > bwd_tol) all_ok = false;
        }
    }
    if (stats) {
        stats->iterations = it_max;
        stats->backward_error_max = bwd_max;
    }
    if (!all_ok)
        return gpch::fail(ctx, GPCH_NOT_CONVERGED, "refinement missed the backward error %.1e within %d iterations",
                          bwd_tol, maxit);
    return GPCH_OK;
}

// ------------------------------------------- allocation-free CG entry point

namespace {

// Scratch of gpch_cg_solve_noalloc: a fixed file-scope device array.  Every
// GPU that loads this library holds it until the process exits.
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(12) << 20;
static __device__ __align__(256) unsigned char g_cg_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is asked
// for, with the device current, on every call: the lookup is cheap, and a
// reset of the device (which may move the array) leaves no stale address.
// The first lookup on a device also loads this file's module there if lazy
// module loading has not loaded it yet, and that load reserves the array.
gpch_status noalloc_scratch(void **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_cg_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return GPCH_CUDA_ERROR;
    }
    *out = p;
    return GPCH_OK;
}

// The set-up call: the array's address and the code of every kernel the
// solve launches, so that later calls make the driver place nothing new.
gpch_status noalloc_setup(void **out)
{
    GPCH_CHECK(noalloc_scratch(out));
    if (cg_kernels_load<double>() != cudaSuccess || cg_kernels_load<float>() != cudaSuccess) {
        cudaGetLastError();
        return GPCH_CUDA_ERROR;
    }
    return GPCH_OK;
}

}  // namespace

extern "C" gpch_status gpch_cg_solve_noalloc(int64_t n, const void *A, gpch_dtype dtype, int64_t lda,
                                             const double *B, int64_t ldb, double *X, int64_t ldx, int nrhs,
                                             double rtol, int maxit, int replace_every, void *stream,
                                             gpch_cg_stats *stats)
{
    // Status plumbing only: this context owns no workspace and no pinned
    // memory, and nothing in this call allocates.
    thread_local gpch_ctx plumbing;
    gpch_ctx *ctx = &plumbing;
    if (stats) *stats = gpch_cg_stats{0, 0, 0.0};
    GPCH_ARG(ctx, n >= 0 && nrhs >= 0 && nrhs <= MAXRHS, "need n >= 0 and 0 <= nrhs <= 16");
    GPCH_ARG(ctx, n * (int64_t)nrhs <= GPCH_NOALLOC_CG_MAX_ELEMS, "n * nrhs exceeds GPCH_NOALLOC_CG_MAX_ELEMS");
    GPCH_ARG(ctx, lda >= (n > 0 ? n : 1) && ldb >= (n > 0 ? n : 1) && ldx >= (n > 0 ? n : 1), "ld < n");
    GPCH_ARG(ctx, dtype == GPCH_F64 || dtype == GPCH_F32, "bad dtype");
    GPCH_ARG(ctx, maxit > 0 && replace_every >= 0 && rtol >= 0.0, "bad maxit / replace_every / rtol");
    GPCH_ARG(ctx, cg_scratch_bytes(n, nrhs) <= NOALLOC_SCRATCH_BYTES, "problem needs more than the fixed scratch");
    // An empty problem is the set-up call: it makes sure the array and the
    // solve's kernels exist on the current device and solves nothing.
    void *scratch = nullptr;
    if (n == 0 || nrhs == 0) return noalloc_setup(&scratch);
    GPCH_CHECK(noalloc_scratch(&scratch));
    GPCH_ARG(ctx, A && B && X, "null pointer");
    alignas(64) unsigned char hbuf[1024];   // host staging for a few scalars (pageable, on the stack)
    int iters[MAXRHS];
    double rel[MAXRHS];
    cudaStream_t s = (cudaStream_t)stream;
    gpch_status st;
    if (dtype == GPCH_F64)
        st = cg_run<double>(ctx, n, static_cast<const double *>(A), lda, B, ldb, X, ldx, nrhs, rtol, maxit,
                            replace_every, s, scratch, hbuf, iters, rel);
    else
        st = cg_run<float>(ctx, n, static_cast<const float *>(A), lda, B, ldb, X, ldx, nrhs, rtol, maxit,
                           replace_every, s, scratch, hbuf, iters, rel);
    if (st != GPCH_OK) return st;
    int max_it = 0, conv = 0;
    double rel_max = 0.0;
    for (int r = 0; r < nrhs; ++r) {
        if (iters[r] > max_it) max_it = iters[r];
        if (rel[r] > rel_max) rel_max = rel[r];
        if (rel[r] <= rtol) ++conv;
    }
    if (stats) *stats = gpch_cg_stats{max_it, conv, rel_max};
    return conv < nrhs ? GPCH_NOT_CONVERGED : GPCH_OK;
}
