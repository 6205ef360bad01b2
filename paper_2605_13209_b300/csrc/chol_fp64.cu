// chol_fp64.cu -- A2-A4: FP64 blocked right-looking Cholesky, Algorithm 1
// (right) of the paper, in place on the lower triangle of a column-major
// matrix.
//
// Per block column j of width `tile`:
//   step 1  the diagonal tile is factored as a nest of 32-wide leaf steps
//           (potrf_leaf -> inverse-apply TRSM below it -> SYRK inside it);
//   step 2  the panel below is solved against L_jj^T one 64-column chunk at
//           a time: X_c = B_c inv(L_cc)^T, then B_{>c} -= X_c L_{>c,c}^T;
//   step 3  one launch updates every 64 x 64 tile of the trailing lower
//           triangle, A_ik -= A_ij A_kj^T with K = tile (SYRK on the
//           diagonal tiles, GEMM below them).
// A device-side info word stops all later kernels after a failed pivot.
#include "dense_fp64.cuh"

namespace {

using gpch::LEAF;

// Step 1 leaf (see potrf_leaf_pipe): factor of an nb x nb block, nb <= W.
template <int W>
__global__ void __launch_bounds__(128) potrf_leaf_kernel(double *A, int64_t lda, int nb, double *rinv, int64_t col0,
                                                         int64_t *info)
{
    gpch::pdl_wait();
    gpch::pdl_trigger();
    potrf_leaf_pipe<W>(A, lda, nb, rinv, col0, info);   // returns at once after an earlier failed pivot
}

// Width of the leaf factorizations inside a diagonal tile.  A leaf runs on
// one SM: its serial pivot chain costs ~5 FP64 instructions per column and
// its bulk update grows with the cube of the width on that SM's FP64 units
// (a 64-wide leaf measured 3.2x a 32-wide one), while every leaf step also
// pays a substitution and an update launch over the rest of the tile.
// 32-wide leaves are the faster of the two.
constexpr int DIAG_LEAF = 32;


}  // namespace

namespace gpch {

// Enqueue the FP64 factorization of the n x n lower triangle at A.
// Linv: workspace of tile/64 * 64*64 doubles; info: device int64 (zeroed by
// the caller).  Used by gpch_chol_factor and by the refined solve.
gpch_status chol_fp64_enqueue(gpch_ctx *ctx, int64_t n, int tile, double *A, int64_t lda, double *rinv,
                              int64_t *info, cudaStream_t st, int64_t col_offset, void *oz_ws, int **oz_err)
{
    for (int64_t j0 = 0; j0 < n; j0 += tile) {
        const int64_t nj = (n - j0 < tile) ? n - j0 : tile;
        double *Ajj = A + j0 + j0 * lda;
        // step 1: the diagonal tile, as a nest of DIAG_LEAF-wide leaf steps
        {
            gpch::PhaseScope ph1(ctx, GPCH_PHASE_DIAG, st, (double)nj * nj * nj / 3.0);
            for (int64_t c0 = 0; c0 < nj; c0 += DIAG_LEAF) {
                const int nc = (int)((nj - c0 < DIAG_LEAF) ? nj - c0 : DIAG_LEAF);
                double *Lcc = Ajj + c0 + c0 * lda;
                // the leaf, substitution and update kernels of this chain
                // are launched as programmatic dependents of their
                // predecessor (each waits for it before reading memory)
                GPCH_CUDA(ctx, gpch::launch_pdl(potrf_leaf_kernel<DIAG_LEAF>, dim3(1), dim3(128), 0, st, Lcc, lda,
                                                nc, rinv + c0, col_offset + j0 + c0, info));
                GPCH_LAUNCH_CHECK(ctx);
                const int64_t mr = nj - c0 - nc;
                if (mr > 0) {
                    double *P = Ajj + (c0 + nc) + c0 * lda;
                    GPCH_CHECK(launch_trsm_sub(ctx, P, lda, mr, nc, Lcc, lda, rinv + c0, info, st, true));
                    GPCH_CHECK(launch_gemm<double>(ctx, true, mr, mr, nc, P, lda, P, lda,
                                                   Ajj + (c0 + nc) * (1 + lda), lda, info, st, true));
                }
            }
        }
        // step 2: panel below the tile, 64-column chunks solved by substitution
        const int64_t m = n - j0 - nj;
        if (m <= 0) continue;
        double *Pan = A + (j0 + nj) + j0 * lda;
        {
            gpch::PhaseScope ph2(ctx, GPCH_PHASE_PANEL, st, (double)m * nj * nj);
            for (int64_t c0 = 0; c0 < nj; c0 += LEAF) {
                const int nc = (int)((nj - c0 < LEAF) ? nj - c0 : LEAF);
                double *Xc = Pan + c0 * lda;
                GPCH_CHECK(launch_trsm_sub(ctx, Xc, lda, m, nc, Ajj + c0 + c0 * lda, lda, rinv + c0, info,
                                                   st));
                const int64_t rest = nj - c0 - nc;
                if (rest > 0)
                    GPCH_CHECK(launch_gemm<double>(ctx, false, m, rest, nc, Xc, lda, Ajj + (c0 + nc) + c0 * lda,
                                                   lda, Pan + (c0 + nc) * lda, lda, info, st));
            }
        }
        // step 3: trailing lower triangle, K = tile: FP64 FMAs, or with
        // oz_ws the FP64-accurate tensor-core product (ozaki.cu)
        gpch::PhaseScope ph3(ctx, GPCH_PHASE_TRAILING, st, (double)nj * m * (m + 1));
        if (oz_ws)
            GPCH_CHECK(oz_gemm_enqueue(ctx, m, m, nj, Pan, lda, Pan, lda, A + (j0 + nj) * (1 + lda), lda, true, oz_ws,
                                       st, oz_err));
        else
            GPCH_CHECK(launch_gemm<double>(ctx, true, m, m, (int)nj, Pan, lda, Pan, lda, A + (j0 + nj) * (1 + lda),
                                           lda, info, st));
    }
    return GPCH_OK;
}

}  // namespace gpch

extern "C" gpch_status gpch_chol_factor_ex(gpch_ctx *ctx, int64_t n, int tile, double *A, int64_t lda,
                                           int32_t update, void *stream, int64_t *info)
{
    GPCH_ARG(ctx, ctx != nullptr, "null context");
    GPCH_ARG(ctx, info != nullptr, "info must not be NULL");
    *info = 0;
    GPCH_ARG(ctx, n >= 0, "n < 0");
    GPCH_ARG(ctx, lda >= (n > 0 ? n : 1), "lda < n");
    GPCH_ARG(ctx, tile >= LEAF && tile <= 1024 && tile % LEAF == 0, "tile must be a multiple of 64 in [64, 1024]");
    GPCH_ARG(ctx, update == GPCH_UPDATE_FP64 || update == GPCH_UPDATE_FP64_EMULATED, "bad update arithmetic");
    if (n == 0) return GPCH_OK;
    GPCH_ARG(ctx, A != nullptr, "null A");
    GPCH_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const bool emu = update == GPCH_UPDATE_FP64_EMULATED;
    gpch::Carver dry(nullptr);
    dry.take<int64_t>(1);
    dry.take<double>((size_t)tile);
    const size_t oz_off = dry.reserve(emu ? gpch::oz_ws_bytes(n, n, true) : 0);
    GPCH_CHECK(gpch::ws_reserve(ctx, dry.off));
    gpch::Carver cv(ctx->ws);
    int64_t *d_info = cv.take<int64_t>(1);
    double *rinv = cv.take<double>((size_t)tile);
    void *oz_ws = emu ? static_cast<char *>(ctx->ws) + oz_off : nullptr;
    int *oz_err = nullptr;
    GPCH_CUDA(ctx, cudaMemsetAsync(d_info, 0, sizeof(int64_t), st));
    GPCH_CHECK(gpch::chol_fp64_enqueue(ctx, n, tile, A, lda, rinv, d_info, st, 0, oz_ws, &oz_err));
    int64_t *h = static_cast<int64_t *>(ctx->pinned);
    GPCH_CUDA(ctx, cudaMemcpyAsync(h, d_info, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    if (oz_err) GPCH_CUDA(ctx, cudaMemcpyAsync(h + 1, oz_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    GPCH_CUDA(ctx, cudaStreamSynchronize(st));
    *info = *h;
    if (oz_err && *reinterpret_cast<int *>(h + 1) != 0)
        return gpch::fail(ctx, GPCH_TIMEOUT, "tensor-core pipeline wait gave up");
    if (*info != 0) return gpch::fail(ctx, GPCH_NOT_SPD, "pivot %lld not positive", (long long)*info);
    return GPCH_OK;
}

extern "C" gpch_status gpch_chol_factor(gpch_ctx *ctx, int64_t n, int tile, double *A, int64_t lda,
                                        void *stream, int64_t *info)
{
    return gpch_chol_factor_ex(ctx, n, tile, A, lda, GPCH_UPDATE_FP64, stream, info);
}
