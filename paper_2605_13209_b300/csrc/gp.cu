// gp.cu -- GP quantities computed on a solved system: the log-determinant
// from the Cholesky factor and the predictive mean at new points.  The
// paper's systems are GP covariance matrices used for behaviour prediction
// (Sec. 4.1): the prediction is the cross covariance times the solution of
// the system, and the log-determinant is the other term of the GP's log
// marginal likelihood next to y^T alpha.
//
// logdet  one CTA; every thread takes log L_ii of a strided subset of the
//         diagonal, then a fixed-order block reduction (reproducible).
// mean    the cross covariance K(Xs, X) is never stored: a CTA takes TM
//         test points and one slice of the training points, stages the
//         slice's points and alpha rows in shared memory TN at a time, and
//         each thread accumulates exp terms times alpha for one test point
//         over a strided subset of every staged chunk.  The slices' partial
//         sums land in workspace and a second kernel adds them in slice
//         order, so the result does not depend on scheduling.  Work per
//         (test, training) pair: d differences and FMAs, one FP64 exp and
//         nrhs FMAs -- FP64-pipe bound on this part.
#include "internal.cuh"

namespace {

constexpr int LD_THREADS = 1024;

__global__ void __launch_bounds__(LD_THREADS) logdet_kernel(int64_t n, const double *__restrict__ L, int64_t ldl,
                                                           double *out, long long *bad)
{
    __shared__ double red[LD_THREADS / 32];
    __shared__ unsigned long long first_bad;   // smallest 1-based index of a non-positive L_ii
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) first_bad = ~0ull;
    __syncthreads();
    double s = 0.0;
    for (int64_t i = tid; i < n; i += LD_THREADS) {
        const double lii = L[i + i * ldl];
        if (lii > 0.0 && isfinite(lii)) s += log(lii);
        else atomicMin(&first_bad, (unsigned long long)(i + 1));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < LD_THREADS / 32; ++w) t += red[w];
        *out = 2.0 * t;
        *bad = first_bad == ~0ull ? 0 : (long long)first_bad;
    }
}

constexpr int PM_THREADS = 256;
constexpr int TM = 16;                       // test points per CTA
constexpr int G = PM_THREADS / TM;           // training-point groups per CTA
constexpr int TN = 32;                       // training points staged per chunk
constexpr int MAXD = 64;
constexpr int MAXRHS = 16;

template <int NR>
__global__ void __launch_bounds__(PM_THREADS) predict_partial_kernel(int64_t m, int64_t n, int d,
                                                                     const double *__restrict__ Xs,
                                                                     const double *__restrict__ X, double sf2,
                                                                     double inv2l2, const double *__restrict__ alpha,
                                                                     int64_t lda, int nrhs, int64_t slice,
                                                                     double *__restrict__ part)
{
    __shared__ double xs[TM][MAXD + 1];
    __shared__ double xc[TN][MAXD + 1];
    __shared__ double ac[TN][NR];
    __shared__ double red[PM_THREADS / 32][TM][NR];
    const int tid = threadIdx.x;
    const int k = tid % TM, g = tid / TM;
    const int64_t k0 = (int64_t)blockIdx.x * TM;
    const int64_t i_begin = (int64_t)blockIdx.y * slice;
    const int64_t i_end = (i_begin + slice < n) ? i_begin + slice : n;

    for (int e = tid; e < TM * d; e += PM_THREADS) {
        const int r = e / d, c = e % d;
        xs[r][c] = (k0 + r < m) ? Xs[(k0 + r) * d + c] : 0.0;
    }
    double acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = 0.0;

    for (int64_t c0 = i_begin; c0 < i_end; c0 += TN) {
        const int cnt = (int)((i_end - c0 < TN) ? i_end - c0 : TN);
        __syncthreads();
        for (int e = tid; e < cnt * d; e += PM_THREADS) {
            const int r = e / d, c = e % d;
            xc[r][c] = X[(c0 + r) * d + c];
        }
        for (int e = tid; e < cnt * NR; e += PM_THREADS) {
            const int r = e / NR, q = e % NR;
            ac[r][q] = (q < nrhs) ? alpha[(c0 + r) + q * lda] : 0.0;
        }
        __syncthreads();
        for (int i = g; i < cnt; i += G) {
            double d2 = 0.0;
            for (int c = 0; c < d; ++c) {
                const double diff = xs[k][c] - xc[i][c];
                d2 = fma(diff, diff, d2);
            }
            const double kv = sf2 * exp(-d2 * inv2l2);
#pragma unroll
            for (int r = 0; r < NR; ++r) acc[r] = fma(kv, ac[i][r], acc[r]);
        }
    }
    // threads tid and tid + TM share a test point and sit in one warp: add
    // them with a shuffle, then the warps' sums in warp order
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], TM);
        if (lane < TM) red[warp][k][r] = acc[r];
    }
    __syncthreads();
    if (tid < TM * NR) {
        const int kk = tid / NR, r = tid % NR;
        double v = 0.0;
        for (int q = 0; q < PM_THREADS / 32; ++q) v += red[q][kk][r];
        if (k0 + kk < m && r < nrhs) part[((size_t)blockIdx.y * m + (k0 + kk)) * MAXRHS + r] = v;
    }
}

__global__ void predict_reduce_kernel(int64_t m, int nrhs, int slices, const double *__restrict__ part,
                                      double *__restrict__ mean, int64_t ldm)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m * nrhs) return;
    const int64_t k = e % m;
    const int r = (int)(e / m);
    double v = 0.0;
    for (int s = 0; s < slices; ++s) v += part[((size_t)s * m + k) * MAXRHS + r];
    mean[k + r * ldm] = v;
}

int sm_count(int device)
{
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        v = 148;
    }
    return v;
}

}  // namespace

extern "C" gpch_status gpch_logdet(gpch_ctx *ctx, int64_t n, const double *L, int64_t ldl, double *logdet,
                                   void *stream)
{
    GPCH_ARG(ctx, ctx != nullptr, "null context");
    GPCH_ARG(ctx, logdet != nullptr, "null output");
    GPCH_ARG(ctx, n >= 0 && ldl >= (n > 0 ? n : 1), "need n >= 0 and ldl >= n");
    if (n == 0) {
        *logdet = 0.0;
        return GPCH_OK;
    }
    GPCH_ARG(ctx, L != nullptr, "null factor");
    GPCH_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    GPCH_CHECK(gpch::ws_reserve(ctx, 256));
    double *dout = static_cast<double *>(ctx->ws);
    long long *dbad = reinterpret_cast<long long *>(static_cast<char *>(ctx->ws) + 64);
    logdet_kernel<<<1, LD_THREADS, 0, s>>>(n, L, ldl, dout, dbad);
    GPCH_LAUNCH_CHECK(ctx);
    double *h = static_cast<double *>(ctx->pinned);
    GPCH_CUDA(ctx, cudaMemcpyAsync(h, ctx->ws, 128, cudaMemcpyDeviceToHost, s));
    GPCH_CUDA(ctx, cudaStreamSynchronize(s));
    const long long bad = *reinterpret_cast<long long *>(reinterpret_cast<char *>(h) + 64);
    if (bad != 0) {
        *logdet = NAN;
        return gpch::fail(ctx, GPCH_NOT_SPD, "factor diagonal entry %lld is not positive", bad);
    }
    *logdet = h[0];
    return GPCH_OK;
}

extern "C" gpch_status gpch_predict_mean(gpch_ctx *ctx, int64_t m, int64_t n, int d, const double *Xs,
                                         const double *X, double sf2, double ell, const double *alpha,
                                         int64_t lda, int nrhs, double *mean, int64_t ldm, void *stream)
{
    GPCH_ARG(ctx, ctx != nullptr, "null context");
    GPCH_ARG(ctx, m >= 0 && n >= 0 && d >= 1 && d <= MAXD, "need m, n >= 0 and 1 <= d <= 64");
    GPCH_ARG(ctx, nrhs >= 0 && nrhs <= MAXRHS, "need 0 <= nrhs <= 16");
    GPCH_ARG(ctx, lda >= (n > 0 ? n : 1) && ldm >= (m > 0 ? m : 1), "leading dimension too small");
    GPCH_ARG(ctx, ell > 0.0, "ell must be positive");
    if (m == 0 || nrhs == 0) return GPCH_OK;
    GPCH_ARG(ctx, Xs != nullptr && mean != nullptr && (n == 0 || (X != nullptr && alpha != nullptr)),
             "null pointer");
    GPCH_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t mt = (m + TM - 1) / TM;
    GPCH_ARG(ctx, mt < (int64_t)0x7fffffff, "m too large");
    // enough training-point slices for four CTAs per SM, each slice at
    // least 4 chunks long
    const int64_t want = (4LL * sm_count(ctx->device) + mt - 1) / mt;
    const int64_t most = (n + 4 * TN - 1) / (4 * TN);
    int64_t slices = want < most ? want : most;
    if (slices < 1) slices = 1;
    if (slices > 65535) slices = 65535;
    const int64_t slice = (n + slices - 1) / slices;
    slices = n > 0 ? (n + slice - 1) / slice : 1;
    GPCH_CHECK(gpch::ws_reserve(ctx, (size_t)slices * m * MAXRHS * sizeof(double)));
    double *part = static_cast<double *>(ctx->ws);
    const double inv2l2 = 1.0 / (2.0 * ell * ell);
    dim3 grid((unsigned)mt, (unsigned)slices);
    if (n == 0) {
        GPCH_CUDA(ctx, cudaMemsetAsync(part, 0, (size_t)m * MAXRHS * sizeof(double), s));
    } else if (nrhs <= 1) {
        predict_partial_kernel<1><<<grid, PM_THREADS, 0, s>>>(m, n, d, Xs, X, sf2, inv2l2, alpha, lda, nrhs, slice,
                                                              part);
    } else if (nrhs <= 4) {
        predict_partial_kernel<4><<<grid, PM_THREADS, 0, s>>>(m, n, d, Xs, X, sf2, inv2l2, alpha, lda, nrhs, slice,
                                                              part);
    } else {
        predict_partial_kernel<16><<<grid, PM_THREADS, 0, s>>>(m, n, d, Xs, X, sf2, inv2l2, alpha, lda, nrhs,
                                                               slice, part);
    }
    if (n > 0) GPCH_LAUNCH_CHECK(ctx);
    const int64_t total = m * nrhs;
    predict_reduce_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(m, nrhs, (int)slices, part, mean, ldm);
    GPCH_LAUNCH_CHECK(ctx);
    return GPCH_OK;
}
