// solve.cu -- A5: forward and back substitution with the Cholesky factor,
// L Y = B then L^T X = Y (Sec. 2.2), FP64, blocked by 64.
//
// All 64 x 64 diagonal blocks of L are inverted first, in one launch.  Each
// sweep then takes one launch per block row:
//   forward, block J:  y_J = inv(L_JJ) b_J;  b_I -= L_IJ y_J  for I > J
//   back,    block J:  x_J = inv(L_JJ)^T w_J;  w_K -= L_JK^T x_J  for K < J
// Every CTA of a step recomputes the 64-entry y_J (x_J) itself, so no
// launch waits on another CTA; the step's output goes to a second buffer so
// that no CTA reads what another CTA of the same launch writes.
#include "dense_fp64.cuh"

namespace {

using gpch::LEAF;

template <typename TL>
__global__ void __launch_bounds__(256) inv_diag_blocks_kernel(int64_t n, const TL *__restrict__ L,
                                                              int64_t ldl, double *Linv)
{
    extern __shared__ double inv_smem[];
    double (*S)[LEAF + 1] = reinterpret_cast<double (*)[LEAF + 1]>(inv_smem);
    double (*Vi)[LEAF + 1] = reinterpret_cast<double (*)[LEAF + 1]>(inv_smem + LEAF * (LEAF + 1));
    const int64_t J = blockIdx.x, o = J * LEAF;
    const int nb = (int)((n - o < LEAF) ? n - o : LEAF);
    for (int e = threadIdx.x; e < LEAF * LEAF; e += blockDim.x) {
        int r = e % LEAF, c = e / LEAF;
        double v = 0.0;
        if (r < nb && c < nb) {
            if (r >= c) v = (double)L[(o + r) + (o + c) * ldl];
        } else if (r == c) {
            v = 1.0;
        }
        S[r][c] = v;
    }
    __syncthreads();
    gpch::invert_lower_64(S, Vi);
    __syncthreads();
    double *dst = Linv + J * LEAF * LEAF;
    for (int e = threadIdx.x; e < LEAF * LEAF; e += blockDim.x) {
        int r = e % LEAF, c = e / LEAF;
        dst[r + c * LEAF] = Vi[r][c];
    }
}

// Forward step J.  W: working right-hand sides (rows > J updated here);
// Y: output (rows of block J written by CTA 0).  Rows below the block are
// split over CTAs, one row per thread.
template <typename TL>
__global__ void __launch_bounds__(256) fwd_step_kernel(int64_t n, int64_t J, const TL *__restrict__ L,
                                                       int64_t ldl, const double *__restrict__ LinvJ,
                                                       double *W, int64_t ldw, double *Y, int64_t ldy,
                                                       int nrhs)
{
    __shared__ double bj[LEAF];
    __shared__ double yj[LEAF];
    const int tid = threadIdx.x;
    const int64_t o = J * LEAF;
    const int nb = (int)((n - o < LEAF) ? n - o : LEAF);
    const int64_t row = o + nb + (int64_t)blockIdx.x * blockDim.x + tid;
    for (int r = 0; r < nrhs; ++r) {
        if (tid < LEAF) bj[tid] = (tid < nb) ? W[o + tid + r * ldw] : 0.0;
        __syncthreads();
        if (tid < LEAF) {
            double s = 0.0;
            for (int k = 0; k <= tid; ++k) s = fma(LinvJ[tid + k * LEAF], bj[k], s);
            yj[tid] = s;
            if (blockIdx.x == 0 && tid < nb) Y[o + tid + r * ldy] = s;
        }
        __syncthreads();
        if (row < n) {
            double s = W[row + r * ldw];
            for (int k = 0; k < nb; ++k) s = fma(-(double)L[row + (o + k) * ldl], yj[k], s);
            W[row + r * ldw] = s;
        }
        __syncthreads();
    }
}

// Back step J.  W: working vectors (entries of blocks K < J updated here);
// X: output (block J written by CTA 0).  Columns c < o are split over CTAs,
// one warp per column, lanes over the 64 rows of block J.
template <typename TL>
__global__ void __launch_bounds__(256) bwd_step_kernel(int64_t n, int64_t J, const TL *__restrict__ L,
                                                       int64_t ldl, const double *__restrict__ LinvJ,
                                                       double *W, int64_t ldw, double *X, int64_t ldx,
                                                       int nrhs)
{
    __shared__ double wj[LEAF];
    __shared__ double xj[LEAF];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t o = J * LEAF;
    const int nb = (int)((n - o < LEAF) ? n - o : LEAF);
    for (int r = 0; r < nrhs; ++r) {
        if (tid < LEAF) wj[tid] = (tid < nb) ? W[o + tid + r * ldw] : 0.0;
        __syncthreads();
        if (tid < LEAF) {
            // x = inv(L_JJ)^T w: x[t] = sum_{k >= t} inv(L)[k][t] w[k]
            double s = 0.0;
            for (int k = tid; k < LEAF; ++k) s = fma(LinvJ[k + tid * LEAF], wj[k], s);
            xj[tid] = s;
            if (blockIdx.x == 0 && tid < nb) X[o + tid + r * ldx] = s;
        }
        __syncthreads();
        const int64_t cbase = (int64_t)blockIdx.x * LEAF;
        for (int cc = warp; cc < LEAF; cc += 8) {
            const int64_t c = cbase + cc;
            if (c >= o) break;
            double s = 0.0;
            if (lane < nb) s = (double)L[(o + lane) + c * ldl] * xj[lane];
            if (lane + 32 < nb) s = fma((double)L[(o + lane + 32) + c * ldl], xj[lane + 32], s);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            if (lane == 0) W[c + r * ldw] -= s;
        }
        __syncthreads();
    }
}

}  // namespace

namespace gpch {

// Enqueue the two sweeps on B (n x nrhs, in place).  Linv: n_blocks*64*64
// doubles of workspace; Y: n x nrhs doubles of workspace (ld n).  TL is the
// storage type of L (FP64 factor, or the FP32 low-precision factor); the
// arithmetic is FP64 either way.
template <typename TL>
gpch_status chol_solve_enqueue_t(gpch_ctx *ctx, int64_t n, const TL *L, int64_t ldl, double *B, int64_t ldb,
                                 int nrhs, double *Linv, double *Y, cudaStream_t st)
{
    gpch::PhaseScope ph(ctx, GPCH_PHASE_SOLVE, st, 2.0 * (double)n * n * nrhs);
    const int64_t NBk = (n + LEAF - 1) / LEAF;
    constexpr size_t INV_SMEM = 2 * LEAF * (LEAF + 1) * sizeof(double);
    static bool attr_done = false;
    if (!attr_done) {
        GPCH_CUDA(ctx, cudaFuncSetAttribute(inv_diag_blocks_kernel<TL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)INV_SMEM));
        attr_done = true;
    }
    inv_diag_blocks_kernel<<<(unsigned)NBk, 256, INV_SMEM, st>>>(n, L, ldl, Linv);
    GPCH_LAUNCH_CHECK(ctx);
    for (int64_t J = 0; J < NBk; ++J) {
        const int64_t below = n - (J + 1) * LEAF;
        const unsigned grid = below > 0 ? (unsigned)((below + 255) / 256) : 1u;
        fwd_step_kernel<<<grid, 256, 0, st>>>(n, J, L, ldl, Linv + J * LEAF * LEAF, B, ldb, Y, n, nrhs);
        GPCH_LAUNCH_CHECK(ctx);
    }
    for (int64_t J = NBk - 1; J >= 0; --J) {
        const int64_t above = J * LEAF;
        const unsigned grid = above > 0 ? (unsigned)((above + LEAF - 1) / LEAF) : 1u;
        bwd_step_kernel<<<grid, 256, 0, st>>>(n, J, L, ldl, Linv + J * LEAF * LEAF, Y, n, B, ldb, nrhs);
        GPCH_LAUNCH_CHECK(ctx);
    }
    return GPCH_OK;
}

gpch_status chol_solve_enqueue(gpch_ctx *ctx, int64_t n, const double *L, int64_t ldl, double *B, int64_t ldb,
                               int nrhs, double *Linv, double *Y, cudaStream_t st)
{
    return chol_solve_enqueue_t<double>(ctx, n, L, ldl, B, ldb, nrhs, Linv, Y, st);
}

gpch_status chol_solve_enqueue_f32(gpch_ctx *ctx, int64_t n, const float *L, int64_t ldl, double *B, int64_t ldb,
                                   int nrhs, double *Linv, double *Y, cudaStream_t st)
{
    return chol_solve_enqueue_t<float>(ctx, n, L, ldl, B, ldb, nrhs, Linv, Y, st);
}

}  // namespace gpch

extern "C" gpch_status gpch_chol_solve(gpch_ctx *ctx, int64_t n, const double *L, int64_t ldl, double *B,
                                       int64_t ldb, int nrhs, void *stream)
{
    GPCH_ARG(ctx, ctx != nullptr, "null context");
    GPCH_ARG(ctx, n >= 0 && nrhs >= 0, "n < 0 or nrhs < 0");
    GPCH_ARG(ctx, ldl >= (n > 0 ? n : 1) && ldb >= (n > 0 ? n : 1), "ldl or ldb < n");
    if (n == 0 || nrhs == 0) return GPCH_OK;
    GPCH_ARG(ctx, L != nullptr && B != nullptr, "null pointer");
    GPCH_CUDA(ctx, cudaSetDevice(ctx->device));
    const int64_t NBk = (n + LEAF - 1) / LEAF;
    gpch::Carver dry(nullptr);
    dry.take<double>((size_t)NBk * LEAF * LEAF);
    dry.take<double>((size_t)n * nrhs);
    GPCH_CHECK(gpch::ws_reserve(ctx, dry.off));
    gpch::Carver cv(ctx->ws);
    double *Linv = cv.take<double>((size_t)NBk * LEAF * LEAF);
    double *Y = cv.take<double>((size_t)n * nrhs);
    return gpch::chol_solve_enqueue(ctx, n, L, ldl, B, ldb, nrhs, Linv, Y, (cudaStream_t)stream);
}
