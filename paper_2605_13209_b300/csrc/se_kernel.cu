// se_kernel.cu -- A1: squared-exponential GP covariance matrix on the device.
//
// A_ij = sf2 * exp(-sum_k (x_ik - x_jk)^2 / (2 ell^2)) + sn2 [i == j]
// (the GP covariance matrices of Sec. 4.1, synthetic SE stand-in).
// One CTA computes a 32 x 32 tile (I, J) with I >= J and writes it twice:
// at (I, J) and, transposed through shared memory, at (J, I).  Both writes
// are coalesced down the columns of the column-major output.
#include "internal.cuh"

namespace {

constexpr int TS = 32;
constexpr int MAXD = 64;

__global__ void __launch_bounds__(256) se_tile_kernel(int64_t n, int d, const double *__restrict__ X,
                                                      double sf2, double inv2l2, double sn2,
                                                      double *__restrict__ A, int64_t lda)
{
    __shared__ double xi[TS][MAXD + 1];
    __shared__ double xj[TS][MAXD + 1];
    __shared__ double V[TS][TS + 1];

    // lower-triangular tile index -> (I, J), I >= J
    int64_t t = blockIdx.x;
    int64_t I = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((I + 1) * (I + 2) / 2 <= t) ++I;
    while (I * (I + 1) / 2 > t) --I;
    int64_t J = t - I * (I + 1) / 2;

    int64_t i0 = I * TS, j0 = J * TS;
    for (int e = threadIdx.x; e < TS * d; e += blockDim.x) {
        int r = e / d, k = e % d;
        xi[r][k] = (i0 + r < n) ? X[(i0 + r) * d + k] : 0.0;
        xj[r][k] = (j0 + r < n) ? X[(j0 + r) * d + k] : 0.0;
    }
    __syncthreads();

    int r = threadIdx.x % TS;
    for (int c = threadIdx.x / TS; c < TS; c += blockDim.x / TS) {
        double d2 = 0.0;
        for (int k = 0; k < d; ++k) {
            double diff = xi[r][k] - xj[c][k];
            d2 += diff * diff;
        }
        double v = sf2 * exp(-d2 * inv2l2);
        if (i0 + r == j0 + c) v += sn2;
        V[r][c] = v;
    }
    __syncthreads();

    for (int c = threadIdx.x / TS; c < TS; c += blockDim.x / TS) {
        if (i0 + r < n && j0 + c < n) A[(i0 + r) + (j0 + c) * lda] = V[r][c];
        if (I != J && j0 + r < n && i0 + c < n) A[(j0 + r) + (i0 + c) * lda] = V[c][r];
    }
}

}  // namespace

extern "C" gpch_status gpch_se_matrix(gpch_ctx *ctx, int64_t n, int d, const double *X, double sf2,
                                      double ell, double sn2, double *A, int64_t lda, void *stream)
{
    GPCH_ARG(ctx, ctx != nullptr, "null context");
    GPCH_ARG(ctx, n >= 0 && d >= 1 && d <= MAXD, "need n >= 0 and 1 <= d <= 64");
    GPCH_ARG(ctx, lda >= (n > 0 ? n : 1), "lda < n");
    GPCH_ARG(ctx, ell > 0.0, "ell must be positive");
    if (n == 0) return GPCH_OK;
    GPCH_ARG(ctx, X != nullptr && A != nullptr, "null pointer");
    GPCH_CUDA(ctx, cudaSetDevice(ctx->device));
    int64_t T = (n + TS - 1) / TS;
    int64_t tiles = T * (T + 1) / 2;
    GPCH_ARG(ctx, tiles < (int64_t)0x7fffffff, "n too large");
    gpch::PhaseScope ph(ctx, GPCH_PHASE_SE, (cudaStream_t)stream, 8.0 * (double)n * n);
    se_tile_kernel<<<(unsigned)tiles, 256, 0, (cudaStream_t)stream>>>(n, d, X, sf2, 1.0 / (2.0 * ell * ell),
                                                                       sn2, A, lda);
    GPCH_LAUNCH_CHECK(ctx);
    return GPCH_OK;
}
