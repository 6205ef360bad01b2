// dense_fp64.cuh -- SIMT building blocks of the blocked Cholesky (Algorithm 1,
// right) and of the triangular solves, for FP64 storage (the direct path)
// and FP32 storage (the panel of the mixed-precision factor).
//
// Leaf size is 64: a 64 x 64 FP64 block (32 KB) fits one CTA's shared
// memory, so a diagonal tile of any size is factored as a nest of 64-wide
// leaf steps.  On this GPU one SM retires two FP64 FMAs per clock, so the
// FP64 kernels are bound by the FP64 pipe, not by memory; they keep that
// pipe busy with 4 x 4 register tiles per thread and several CTAs per SM.
#pragma once

#include "internal.cuh"

namespace gpch {

constexpr int LEAF = 64;

// Inverse of the unit-padded lower-triangular 64 x 64 block S (S[r][c],
// row r, column c) into Vi (same layout), by forward substitution on the
// columns of the identity: Vi[c][c] = 1/S[c][c],
// Vi[i][c] = -(sum_{k=c}^{i-1} S[i][k] Vi[k][c]) / S[i][i] for i > c.
// 256 threads: four lanes share one column and split the sum over k.
// Entries above the diagonal are set to zero.
__device__ inline void invert_lower_64(const double (*S)[LEAF + 1], double (*Vi)[LEAF + 1])
{
    const int tid = threadIdx.x;
    const int c = tid >> 2, q = tid & 3;
    for (int i = 0; i < LEAF; ++i) {
        double part = 0.0;
        if (i > c)
            for (int k = c + q; k < i; k += 4) part = fma(S[i][k], Vi[k][c], part);
        part += __shfl_xor_sync(0xffffffffu, part, 1);
        part += __shfl_xor_sync(0xffffffffu, part, 2);
        if (q == 0) {
            if (i < c) Vi[i][c] = 0.0;
            else if (i == c) Vi[c][c] = 1.0 / S[c][c];
            else Vi[i][c] = -part / S[i][i];
        }
        __syncwarp();
    }
}

}  // namespace gpch

// Kernels and their launchers have internal linkage: every translation unit
// that uses them compiles and registers its own copies.
namespace {

using gpch::LEAF;

// Panel leaf solve: X = B inv(L)^T in place on the m x nc panel B (nc <=
// 64), inv(L) given as a 64 x 64 FP64 block (column-major, ld 64).  Every
// CTA owns 64 whole rows, so reading B and writing X never overlap across
// CTAs.  T is the storage and arithmetic type of B.
template <typename T>
__global__ void __launch_bounds__(256) trsm_inv_kernel(T *B, int64_t ldb, int64_t m, int nc,
                                                       const double *__restrict__ Linv, const int64_t *info)
{
    extern __shared__ __align__(16) unsigned char trsm_smem[];
    T *Bs = reinterpret_cast<T *>(trsm_smem);   // Bs[k * 64 + r]
    T *Ls = Bs + LEAF * LEAF;                   // Ls[k * 64 + c] = inv(L)[c][k]
    if (info && *info != 0) return;
    const int tid = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * LEAF;
    for (int e = tid; e < LEAF * LEAF; e += blockDim.x) {
        int r = e % LEAF, k = e / LEAF;
        Bs[k * LEAF + r] = (r0 + r < m && k < nc) ? B[(r0 + r) + k * ldb] : T(0);
        Ls[k * LEAF + r] = (T)Linv[r + k * LEAF];
    }
    __syncthreads();
    const int tx = tid % 16, ty = tid / 16;
    T acc[4][4] = {};
    for (int k = 0; k < LEAF; ++k) {
        T a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = Bs[k * LEAF + tx + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Ls[k * LEAF + ty + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int64_t r = r0 + tx + 16 * i;
            int c = ty + 16 * j;
            if (r < m && c < nc) B[r + c * ldb] = acc[i][j];
        }
}

// C[m x nn] -= A[m x k] B[nn x k]^T.  LOWER: C is square and only its lower
// triangle is updated; the grid enumerates the lower 64 x 64 tiles.
template <typename T, bool LOWER>
__global__ void __launch_bounds__(256, 3) gemm_nt_minus_kernel(int64_t m, int64_t nn, int k,
                                                               const T *__restrict__ A, int64_t lda,
                                                               const T *__restrict__ B, int64_t ldb, T *C,
                                                               int64_t ldc, const int64_t *info)
{
    constexpr int KC = 32;
    __shared__ T As[KC][LEAF];
    __shared__ T Bs[KC][LEAF];
    if (info && *info != 0) return;
    int64_t ti, tj;
    if (LOWER) {
        int64_t t = blockIdx.x;
        ti = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
        while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
        while (ti * (ti + 1) / 2 > t) --ti;
        tj = t - ti * (ti + 1) / 2;
    } else {
        ti = blockIdx.x;
        tj = blockIdx.y;
    }
    const int64_t r0 = ti * LEAF, c0 = tj * LEAF;
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    T acc[4][4] = {};
    for (int k0 = 0; k0 < k; k0 += KC) {
        for (int e = tid; e < KC * LEAF; e += blockDim.x) {
            int r = e % LEAF, kk = e / LEAF;
            bool kin = k0 + kk < k;
            As[kk][r] = (kin && r0 + r < m) ? A[(r0 + r) + (int64_t)(k0 + kk) * lda] : T(0);
            Bs[kk][r] = (kin && c0 + r < nn) ? B[(c0 + r) + (int64_t)(k0 + kk) * ldb] : T(0);
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < KC; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int64_t r = r0 + tx + 16 * i, c = c0 + ty + 16 * j;
            if (r < m && c < nn && (!LOWER || r >= c)) C[r + c * ldc] -= acc[i][j];
        }
}

template <typename T>
constexpr size_t trsm_smem_bytes()
{
    return 2 * LEAF * LEAF * sizeof(T);
}

template <typename T>
inline gpch_status launch_gemm(gpch_ctx *ctx, bool lower, int64_t m, int64_t nn, int k, const T *A, int64_t lda,
                               const T *B, int64_t ldb, T *C, int64_t ldc, const int64_t *info, cudaStream_t st)
{
    if (m <= 0 || nn <= 0 || k <= 0) return GPCH_OK;
    if (lower) {
        int64_t Tn = (m + LEAF - 1) / LEAF;
        gemm_nt_minus_kernel<T, true><<<(unsigned)(Tn * (Tn + 1) / 2), 256, 0, st>>>(m, nn, k, A, lda, B, ldb, C,
                                                                                      ldc, info);
    } else {
        dim3 grid((unsigned)((m + LEAF - 1) / LEAF), (unsigned)((nn + LEAF - 1) / LEAF));
        gemm_nt_minus_kernel<T, false><<<grid, 256, 0, st>>>(m, nn, k, A, lda, B, ldb, C, ldc, info);
    }
    GPCH_LAUNCH_CHECK(ctx);
    return GPCH_OK;
}

template <typename T>
inline gpch_status launch_trsm(gpch_ctx *ctx, T *B, int64_t ldb, int64_t m, int nc, const double *Linv,
                               const int64_t *info, cudaStream_t st)
{
    if (m <= 0) return GPCH_OK;
    static bool attr_done = false;
    if (!attr_done) {
        GPCH_CUDA(ctx, cudaFuncSetAttribute(trsm_inv_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)trsm_smem_bytes<T>()));
        attr_done = true;
    }
    trsm_inv_kernel<T><<<(unsigned)((m + LEAF - 1) / LEAF), 256, trsm_smem_bytes<T>(), st>>>(B, ldb, m, nc, Linv,
                                                                                          info);
    GPCH_LAUNCH_CHECK(ctx);
    return GPCH_OK;
}

}  // namespace

namespace gpch {

// Enqueue the FP64 blocked factorization (chol_fp64.cu).  A failed pivot
// at local column c sets *info = col_offset + c + 1.
gpch_status chol_fp64_enqueue(gpch_ctx *ctx, int64_t n, int tile, double *A, int64_t lda, double *Linv,
                              int64_t *info, cudaStream_t st, int64_t col_offset);

// Enqueue L L^T X = B (solve.cu); Linv (n_blocks*64*64 doubles) and Y
// (n*nrhs doubles) are workspace.  The _f32 form takes an FP32 factor.
gpch_status chol_solve_enqueue(gpch_ctx *ctx, int64_t n, const double *L, int64_t ldl, double *B, int64_t ldb,
                               int nrhs, double *Linv, double *Y, cudaStream_t st);
gpch_status chol_solve_enqueue_f32(gpch_ctx *ctx, int64_t n, const float *L, int64_t ldl, double *B, int64_t ldb,
                                   int nrhs, double *Linv, double *Y, cudaStream_t st);

// Low-precision factor (mixed.cu): workspace size, W = A + shift I, and the
// factorization of W in place (info / err device words returned).
size_t mixed_ws_bytes(int64_t n, int tile);
gpch_status mixed_init_enqueue(gpch_ctx *ctx, int64_t n, const double *A, int64_t lda, float *W, int64_t ldw,
                               double shift, cudaStream_t st);
gpch_status mixed_factor_enqueue(gpch_ctx *ctx, int64_t n, int tile, float *W, int64_t ldw, int prec, void *wsbase,
                                 int64_t **info_out, int **err_out, cudaStream_t st);

}  // namespace gpch
