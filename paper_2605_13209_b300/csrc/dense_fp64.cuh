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

// Inverse X = L^-1 of the unit-padded lower-triangular 64 x 64 block S
// (S[r][c], row r, column c; 256 threads) into Vi (same layout), by forward
// substitution on all columns of the identity at once: row j of X is final
// once scaled by 1/L_jj, and is then eliminated from every row below it,
// X[r][c] -= L[r][j] X[j][c].  Thread (tx, ty) keeps X entries
// (tx + 16i, ty + 16jj) in registers; the finished row j goes through a
// double-buffered shared row so one barrier per step suffices.  Entries
// above the diagonal are zero.
__device__ inline void invert_lower_64(const double (*S)[LEAF + 1], double (*Vi)[LEAF + 1])
{
    __shared__ double dinv[LEAF];
    __shared__ double xrow[2][LEAF];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    double x[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) x[i][jj] = (tx + 16 * i == ty + 16 * jj) ? 1.0 : 0.0;
    if (tid < LEAF) dinv[tid] = 1.0 / S[tid][tid];
    __syncthreads();
    for (int j = 0; j < LEAF; ++j) {
        double *xr = xrow[j & 1];
        if (tx == j % 16) {
            const int i = j / 16;
            const double d = dinv[j];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                const int c = ty + 16 * jj;
                if (c <= j) {
                    x[i][jj] *= d;
                    xr[c] = x[i][jj];
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = tx + 16 * i;
            if (r <= j) continue;
            const double l = S[r][j];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                const int c = ty + 16 * jj;
                if (c <= j) x[i][jj] -= l * xr[c];
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) Vi[tx + 16 * i][ty + 16 * jj] = x[i][jj];
}

// Square root and reciprocal square root of a positive pivot d, by Newton
// iteration on y = 1/sqrt(d) from an FP32 seed: each step
// y <- y (3 - d y^2) / 2 doubles the correct bits (24 -> 48 -> full), then
// s = d y is corrected once by s <- s + y (d - s^2) / 2.  Both results are
// within a few units in the last place; the exact cases (d = 1, perfect
// squares of small integers) come out exact.  Outside the FP32 range the
// division-based form is used.
__device__ inline void pivot_sqrt(double d, double &s, double &y)
{
    if (d > 1e-30 && d < 1e30) {
        y = (double)__frsqrt_rn((float)d);
        y = y * fma(-0.5 * d, y * y, 1.5);
        y = y * fma(-0.5 * d, y * y, 1.5);
        s = d * y;
        s = fma(0.5 * y, fma(-s, s, d), s);
    } else {
        s = sqrt(d);
        y = 1.0 / s;
    }
}

// Reciprocal of a positive pivot d: FP32 seed y0 (rcp.approx), then one
// Newton-Raphson step taken to third order, y = y0 (1 + e + e^2) with
// e = 1 - d y0 (the truncated series of 1 / (1 - e)); with |e| < 2^-21 the
// truncation error is below 2^-63, so the result is within about one unit
// in the last place.  Outside the FP32 range the division is used.
__device__ inline double pivot_rcp(double d)
{
    if (d > 1e-30 && d < 1e30) {
        float yf;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"((float)d));
        const double y0 = (double)yf;
        const double e = fma(-d, y0, 1.0);
        return fma(y0, fma(e, e, e), y0);
    }
    return 1.0 / d;
}

// Pivot test and reciprocal for the critical chain of a leaf, with as few
// FP64-pipe instructions as possible (on this GPU each one occupies the
// sub-partition's FP64 unit for many cycles, so the chain's length is their
// count).  The positivity / range test reads the exponent bits with integer
// instructions.  For 2^-100 <= d <= 2^100 the reciprocal is the hardware
// approximation (rcp.approx.ftz.f64) refined by the truncated series
// y0 (1 + e + e^2 + e^3), e = 1 - d y0, whose error is e^4; other positive
// finite pivots take the division.  Returns false for d <= 0, inf or NaN.
__device__ inline bool pivot_rcp_chain(double d, double &rd)
{
    const long long bits = __double_as_longlong(d);
    const int ex = (int)(bits >> 52);   // exponent field when the sign bit is clear, < 0 otherwise
    if (ex >= 1023 - 100 && ex <= 1023 + 100) {
        double y0;
        asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y0) : "d"(d));
        const double e = fma(-d, y0, 1.0);
        rd = fma(y0, fma(e, fma(e, e, e), e), y0);
        return true;
    }
    if (bits > 0 && ex < 2047) {
        rd = 1.0 / d;
        return true;
    }
    return false;
}

// Programmatic dependent launch.  A kernel of the step-1 chain calls
// pdl_wait() before touching memory (it returns once the preceding kernel
// of the stream has finished and its writes are visible; immediately when
// the launch was an ordinary one) and pdl_trigger() to let the next kernel
// be scheduled while this one runs, which hides the launch latency of the
// chain's many small dependent launches.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch `kern` on `st` allowing it to start before the previous kernel of
// the stream has finished (the kernel must begin with pdl_wait()).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

}  // namespace gpch

// Kernels and their launchers have internal linkage: every translation unit
// that uses them compiles and registers its own copies.
namespace {

using gpch::LEAF;

// Step 1 leaf: factor the nb x nb (nb <= W, W = 32 or 64) lower block at A
// in place.  Thread (tx, ty) keeps the (W/16)^2 entries (tx + 16i, ty + 16j)
// in registers.  The column sweep is square-root free: step j subtracts
// a_rj * (a_cj / d_j) from every entry (r, c) with r >= c > j, which is the
// right-looking Cholesky update l_rj l_cj written with the unscaled column
// (a_rj = l_rj sqrt(d_j)).  The entries of column j are final after step
// j - 1 and are never touched again, so at the end L_rc = a_rc / sqrt(d_c)
// and L_cc = sqrt(d_c), with all square roots taken at once.  Per step one
// barrier: the owner of the next pivot updates it, takes its reciprocal and
// publishes it together with the next column while the other threads finish
// their updates (one-column lookahead).  Outputs: rinv[c] = 1 / L_cc (c < W;
// 1 in the padding) and, when Linv is not null (W = 64 only), inv(L) of the
// unit-padded block (column-major, ld 64).  leaf_smem: 2 * 64 * 65 doubles.
template <int W>
__device__ inline void potrf_leaf_body(double *A, int64_t lda, int nb, double *rinv, double *Linv, int64_t col0,
                                       int64_t *info, double *leaf_smem)
{
    constexpr int RT = W / 16;
    double (*S)[LEAF + 1] = reinterpret_cast<double (*)[LEAF + 1]>(leaf_smem);
    double (*Vi)[LEAF + 1] = reinterpret_cast<double (*)[LEAF + 1]>(leaf_smem + LEAF * (LEAF + 1));
    __shared__ double ucol[2][LEAF];   // column j before scaling, by the parity of j
    __shared__ double rdb[2];          // 1 / d_j, by the parity of j
    __shared__ double dpiv[LEAF];      // pivots d_j
    __shared__ double sqv[LEAF], rsv[LEAF];
    __shared__ int bad;
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    double a[RT][RT];
#pragma unroll
    for (int i = 0; i < RT; ++i)
#pragma unroll
        for (int j = 0; j < RT; ++j) {
            const int r = tx + 16 * i, c = ty + 16 * j;
            double v;
            if (r < nb && c < nb) v = (r >= c) ? A[r + c * lda] : 0.0;
            else v = (r == c) ? 1.0 : 0.0;
            a[i][j] = v;
        }
    if (tid == 0) bad = 0;
    __syncthreads();
    if (ty == 0) {
#pragma unroll
        for (int i = 0; i < RT; ++i) ucol[0][tx + 16 * i] = a[i][0];
    }
    if (tid == 0) {
        const double d = a[0][0];
        dpiv[0] = d;
        if (!(d > 0.0) || !isfinite(d)) bad = 1;
        else rdb[0] = gpch::pivot_rcp(d);
    }
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        if (bad) break;
        const double rd = rdb[j & 1];
        const double *uc = ucol[j & 1];
        const int j1 = j + 1;
        const bool more = j1 < nb;
        const int jq = j1 / 16, jr = j1 % 16;
#pragma unroll
        for (int jj = 0; jj < RT; ++jj) {
            const int c = ty + 16 * jj;
            if (c <= j) continue;
            const double lc = uc[c] * rd;
#pragma unroll
            for (int i = 0; i < RT; ++i) {
                const int r = tx + 16 * i;
                if (r >= c) a[i][jj] = fma(-uc[r], lc, a[i][jj]);
            }
        }
        if (more && ty == jr) {
#pragma unroll
            for (int jj = 0; jj < RT; ++jj) {
                if (jj != jq) continue;
#pragma unroll
                for (int i = 0; i < RT; ++i) {
                    const int r = tx + 16 * i;
                    if (r > j1) ucol[j1 & 1][r] = a[i][jj];
                    if (r == j1) {
                        const double d = a[i][jj];
                        dpiv[j1] = d;
                        if (!(d > 0.0) || !isfinite(d)) bad = j1 + 1;
                        else rdb[j1 & 1] = gpch::pivot_rcp(d);
                    }
                }
            }
        }
        __syncthreads();
    }
    if (bad) {
        if (tid == 0) *info = col0 + bad;
        return;
    }
    if (tid < W) {
        double sq = 1.0, rs = 1.0;
        if (tid < nb) gpch::pivot_sqrt(dpiv[tid], sq, rs);
        sqv[tid] = sq;
        rsv[tid] = rs;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RT; ++i)
#pragma unroll
        for (int j = 0; j < RT; ++j) {
            const int r = tx + 16 * i, c = ty + 16 * j;
            a[i][j] = (r > c) ? a[i][j] * rsv[c] : (r == c ? sqv[c] : 0.0);
            if (r < nb && c < nb && r >= c) A[r + c * lda] = a[i][j];
        }
    if (rinv && tid < W) rinv[tid] = rsv[tid];
    if (Linv == nullptr) return;
    // inverse of the unit-padded 64 x 64 block (W == 64)
#pragma unroll
    for (int i = 0; i < RT; ++i)
#pragma unroll
        for (int j = 0; j < RT; ++j) S[tx + 16 * i][ty + 16 * j] = a[i][j];
    __syncthreads();
    gpch::invert_lower_64(S, Vi);
    __syncthreads();
    for (int e = tid; e < LEAF * LEAF; e += blockDim.x) {
        const int r = e % LEAF, c = e / LEAF;
        Linv[r + c * LEAF] = Vi[r][c];
    }
}

// Step 1 leaf of width W (32 or 64), one CTA of THREADS threads: the same
// square-root-free sweep as potrf_leaf_body, laid out for the FP64 units.
// The W x W block lives in shared memory.  Warp 0 (alone on SM
// sub-partition 0; the other warps there only take part in the barriers)
// owns the serial chain: at step j it applies column j to column j+1 (lane
// l holds rows l, l + 32, ...), takes the reciprocal of the new pivot and
// publishes l_c = a_c,j+1 / d_j+1 for the next step.  The warps on
// sub-partitions 1-3 update every column beyond j+1, PER entries per thread
// taken in column-major order of the lower triangle, so whole warps fall
// idle as the sweep moves right.  One barrier per column.  Outputs as
// potrf_leaf_body: A (lower nb x nb, nb <= W) overwritten by L, rinv[c] =
// 1 / L_cc (1 in the padding), *info = col0 + c + 1 on a failed pivot.
template <int W, int THREADS>
__device__ inline void potrf_leaf_chain(double *A, int64_t lda, int nb, double *rinv, int64_t col0, int64_t *info)
{
    constexpr int RH = W / 32;                                  // rows per lane of warp 0
    constexpr int BULK = THREADS / 4 * 3;                       // threads on sub-partitions 1-3
    constexpr int PER = (W * (W + 1) / 2 + BULK - 1) / BULK;    // lower-triangle entries per bulk thread
    __shared__ double S[W][W + 1];   // S[r][c]
    __shared__ double lcb[2][W];     // l_c of the current step, by parity
    __shared__ double dpiv[W], sqv[W], rsv[W];
    __shared__ int bad;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int e = tid; e < W * W; e += THREADS) {
        const int r = e % W, c = e / W;
        double v;
        if (r < nb && c < nb) v = (r >= c) ? A[r + c * lda] : 0.0;
        else v = (r == c) ? 1.0 : 0.0;
        S[r][c] = v;
    }
    if (tid == 0) bad = 0;
    const int sp = warp & 3;
    const int b = (sp != 0) ? ((warp >> 2) * 3 + (sp - 1)) * 32 + lane : -1;
    int er[PER], ec[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        er[q] = -1;
        ec[q] = W;   // never active
        const int e = PER * b + q;
        if (b >= 0 && e < W * (W + 1) / 2) {
            int c = 0, off = 0;
            while (e >= off + (W - c)) {
                off += W - c;
                ++c;
            }
            er[q] = c + (e - off);
            ec[q] = c;
        }
    }
    __syncthreads();
    if (warp == 0) {
        double rd = 0.0;
        if (lane == 0) {
            dpiv[0] = S[0][0];
            if (!gpch::pivot_rcp_chain(S[0][0], rd)) bad = 1;
        }
        rd = __shfl_sync(0xffffffffu, rd, 0);
#pragma unroll
        for (int h = 0; h < RH; ++h) lcb[0][lane + 32 * h] = S[lane + 32 * h][0] * rd;
    }
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        if (bad) break;
        const double *lc = lcb[j & 1];
        const int j1 = j + 1;
        if (warp == 0) {
            if (j1 < nb) {
                // column j1 <- column j1 - column j * l_j1 (rows above j1 are zero)
                const int hp = j1 / 32, lp = j1 % 32;   // holder of the pivot row
                double a[RH];
#pragma unroll
                for (int h = 0; h < RH; ++h) a[h] = fma(-S[lane + 32 * h][j], lc[j1], S[lane + 32 * h][j1]);
                double rd = 0.0;
                if (lane == lp) {
                    const double d = a[hp];
                    dpiv[j1] = d;
                    if (!gpch::pivot_rcp_chain(d, rd)) bad = j1 + 1;
                }
                rd = __shfl_sync(0xffffffffu, rd, lp);
#pragma unroll
                for (int h = 0; h < RH; ++h) {
                    const int r = lane + 32 * h;
                    if (r >= j1) S[r][j1] = a[h];
                    lcb[j1 & 1][r] = a[h] * rd;
                }
            }
        } else if (b >= 0) {
#pragma unroll
            for (int q = 0; q < PER; ++q)
                if (ec[q] > j1) S[er[q]][ec[q]] = fma(-S[er[q]][j], lc[ec[q]], S[er[q]][ec[q]]);
        }
        __syncthreads();
    }
    if (bad) {
        if (tid == 0) *info = col0 + bad;
        return;
    }
    if (tid < W) {
        double sq = 1.0, rs = 1.0;
        if (tid < nb) gpch::pivot_sqrt(dpiv[tid], sq, rs);
        sqv[tid] = sq;
        rsv[tid] = rs;
    }
    __syncthreads();
    for (int e = tid; e < W * W; e += THREADS) {
        const int r = e % W, c = e / W;
        if (r < nb && c < nb && r >= c) A[r + c * lda] = (r == c) ? sqv[c] : S[r][c] * rsv[c];
    }
    if (rinv && tid < W) rinv[tid] = rsv[tid];
}

// Panel solve by substitution: X = B L^-T in place on the m x nc panel B
// (nc <= 64), with L a lower nc x nc FP64 block (ld ldl) and rinv its
// diagonal reciprocals.  Column-oriented (right-looking): x_c = b_c / L_cc,
// then b_k -= x_c L[k][c] for every k > c.  One warp per RPW rows; lane l
// holds columns l and l + 32 of each of its rows (NARROW, nc <= 32: column
// l only), so a column costs one shuffle and three (NARROW: two) FMA-class
// instructions per row.  The CTA's WARPS * RPW rows are staged through
// shared memory so that global reads and writes stay coalesced.  T is the
// storage and arithmetic type of B.
template <typename T, int RPW, int WARPS = 8, bool NARROW = false>
__global__ void __launch_bounds__(WARPS * 32) trsm_sub_kernel(T *B, int64_t ldb, int64_t m, int nc,
                                                              const double *__restrict__ L, int64_t ldl,
                                                              const double *__restrict__ rinv, const int64_t *info)
{
    constexpr int ROWS = WARPS * RPW;
    constexpr int KR = NARROW ? 32 : LEAF;   // columns held
    __shared__ T Ls[KR][KR + 1];   // Ls[k][c] = L[k][c]
    __shared__ T rs[KR];
    __shared__ T Bs[KR][ROWS + 1];
    gpch::pdl_wait();
    gpch::pdl_trigger();
    if (info && *info != 0) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * ROWS;
    for (int e = tid; e < KR * KR; e += blockDim.x) {
        const int k = e % KR, c = e / KR;   // column-major walk: coalesced
        Ls[k][c] = (k > c && k < nc && c < nc) ? (T)L[k + (int64_t)c * ldl] : T(0);
    }
    if (tid < KR) rs[tid] = tid < nc ? (T)rinv[tid] : T(1);
    for (int e = tid; e < KR * ROWS; e += blockDim.x) {
        const int r = e % ROWS, k = e / ROWS;
        Bs[k][r] = (r0 + r < m && k < nc) ? B[(r0 + r) + (int64_t)k * ldb] : T(0);
    }
    __syncthreads();
    T b0[RPW], b1[RPW];
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
        b0[q] = Bs[lane][warp * RPW + q];
        b1[q] = NARROW ? T(0) : Bs[lane + 32 - (NARROW ? 32 : 0)][warp * RPW + q];
    }
    for (int c = 0; c < nc; ++c) {
        const T l0 = Ls[lane][c];   // zero on and above the diagonal
        const T rc = rs[c];
        const int src = c & 31;
        if (NARROW) {
#pragma unroll
            for (int q = 0; q < RPW; ++q) {
                const T xc = __shfl_sync(0xffffffffu, b0[q], src) * rc;
                if (lane == src) b0[q] = xc;
                b0[q] = fma(-xc, l0, b0[q]);
            }
            continue;
        }
        const T l1 = Ls[lane + 32 - (NARROW ? 32 : 0)][c];
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            const T xc = __shfl_sync(0xffffffffu, c < 32 ? b0[q] : b1[q], src) * rc;
            if (lane == src) {
                if (c < 32) b0[q] = xc;
                else b1[q] = xc;
            }
            b0[q] = fma(-xc, l0, b0[q]);
            b1[q] = fma(-xc, l1, b1[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
        Bs[lane][warp * RPW + q] = b0[q];
        if (!NARROW) Bs[lane + 32 - (NARROW ? 32 : 0)][warp * RPW + q] = b1[q];
    }
    __syncthreads();
    for (int e = tid; e < KR * ROWS; e += blockDim.x) {
        const int r = e % ROWS, k = e / ROWS;
        if (r0 + r < m && k < nc) B[(r0 + r) + (int64_t)k * ldb] = Bs[k][r];
    }
}

template <typename T, int ROWS>
__device__ inline void trsm_inv_body(T *B, int64_t ldb, int64_t m, int nc, const double *__restrict__ Linv,
                                     int64_t r0, unsigned char *trsm_smem)
{
    constexpr int G = 256 / ROWS, NC = LEAF / G;
    T *Bs = reinterpret_cast<T *>(trsm_smem);   // Bs[k * ROWS + r]
    T *Ls = Bs + LEAF * ROWS;                   // Ls[k * 64 + c] = inv(L)[c][k]
    const int tid = threadIdx.x;
    for (int e = tid; e < LEAF * ROWS; e += blockDim.x) {
        const int r = e % ROWS, k = e / ROWS;
        Bs[k * ROWS + r] = (r0 + r < m && k < nc) ? B[(r0 + r) + k * ldb] : T(0);
    }
    for (int e = tid; e < LEAF * LEAF; e += blockDim.x) {
        const int c = e % LEAF, k = e / LEAF;
        Ls[k * LEAF + c] = (T)Linv[c + k * LEAF];
    }
    __syncthreads();
    const int r = tid % ROWS, g = tid / ROWS;
    T acc[NC] = {};
    for (int k = 0; k < LEAF; ++k) {
        const T b = Bs[k * ROWS + r];
#pragma unroll
        for (int u = 0; u < NC; ++u) acc[u] = fma(b, Ls[k * LEAF + g + G * u], acc[u]);
    }
    if (r0 + r < m)
#pragma unroll
        for (int u = 0; u < NC; ++u) {
            const int c = g + G * u;
            if (c < nc) B[(r0 + r) + c * ldb] = acc[u];
        }
}

template <typename T, int ROWS>
__global__ void __launch_bounds__(256) trsm_inv_kernel(T *B, int64_t ldb, int64_t m, int nc,
                                                       const double *__restrict__ Linv, const int64_t *info)
{
    extern __shared__ __align__(16) unsigned char trsm_smem[];
    if (info && *info != 0) return;
    trsm_inv_body<T, ROWS>(B, ldb, m, nc, Linv, (int64_t)blockIdx.x * ROWS, trsm_smem);
}

// Triangular tile index t -> (ti, tj), ti >= tj, t = ti (ti + 1) / 2 + tj.
__device__ inline void tri_index(int64_t t, int64_t &ti, int64_t &tj)
{
    ti = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
    while (ti * (ti + 1) / 2 > t) --ti;
    tj = t - ti * (ti + 1) / 2;
}

// One BT x BT tile (ti, tj) of C[m x nn] -= A[m x k] B[nn x k]^T; LOWER
// keeps only entries on or below the diagonal.  Thread (tx, ty) owns
// entries (tx + 16i, ty + 16j) of the tile.
template <typename T, bool LOWER, int BT>
__device__ inline void gemm_nt_minus_body(int64_t m, int64_t nn, int k, const T *__restrict__ A, int64_t lda,
                                          const T *__restrict__ B, int64_t ldb, T *C, int64_t ldc, int64_t ti,
                                          int64_t tj)
{
    constexpr int KC = 32, RT = BT / 16;
    __shared__ T As[KC][BT];
    __shared__ T Bs[KC][BT];
    const int64_t r0 = ti * BT, c0 = tj * BT;
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    T acc[RT][RT] = {};
    for (int k0 = 0; k0 < k; k0 += KC) {
        for (int e = tid; e < KC * BT; e += blockDim.x) {
            int r = e % BT, kk = e / BT;
            bool kin = k0 + kk < k;
            As[kk][r] = (kin && r0 + r < m) ? A[(r0 + r) + (int64_t)(k0 + kk) * lda] : T(0);
            Bs[kk][r] = (kin && c0 + r < nn) ? B[(c0 + r) + (int64_t)(k0 + kk) * ldb] : T(0);
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < KC; ++kk) {
            T a[RT], b[RT];
#pragma unroll
            for (int i = 0; i < RT; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < RT; ++j) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < RT; ++i)
#pragma unroll
                for (int j = 0; j < RT; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < RT; ++i)
#pragma unroll
        for (int j = 0; j < RT; ++j) {
            int64_t r = r0 + tx + 16 * i, c = c0 + ty + 16 * j;
            if (r < m && c < nn && (!LOWER || r >= c)) C[r + c * ldc] -= acc[i][j];
        }
}

// C[m x nn] -= A[m x k] B[nn x k]^T.  LOWER: C is square and only its lower
// triangle is updated; the grid enumerates the lower BT x BT tiles.
template <typename T, bool LOWER, int BT>
__global__ void __launch_bounds__(256, BT == 16 ? 6 : 3) gemm_nt_minus_kernel(int64_t m, int64_t nn, int k,
                                                               const T *__restrict__ A, int64_t lda,
                                                               const T *__restrict__ B, int64_t ldb, T *C,
                                                               int64_t ldc, const int64_t *info)
{
    gpch::pdl_wait();
    gpch::pdl_trigger();
    if (info && *info != 0) return;
    int64_t ti, tj;
    if (LOWER) {
        tri_index(blockIdx.x, ti, tj);
    } else {
        ti = blockIdx.x;
        tj = blockIdx.y;
    }
    gemm_nt_minus_body<T, LOWER, BT>(m, nn, k, A, lda, B, ldb, C, ldc, ti, tj);
}

template <typename T, int ROWS>
constexpr size_t trsm_smem_bytes()
{
    return (size_t)(LEAF * ROWS + LEAF * LEAF) * sizeof(T);
}

// Below this many 64 x 64 tiles (two per SM) the small-tile variants are
// used, so that small in-tile steps still spread over the whole GPU.
constexpr int64_t SMALL_GRID = 296;

template <typename T>
inline gpch_status launch_gemm(gpch_ctx *ctx, bool lower, int64_t m, int64_t nn, int k, const T *A, int64_t lda,
                               const T *B, int64_t ldb, T *C, int64_t ldc, const int64_t *info, cudaStream_t st,
                               bool pdl = false)
{
    if (m <= 0 || nn <= 0 || k <= 0) return GPCH_OK;
    const int64_t tm = (m + LEAF - 1) / LEAF, tn = (nn + LEAF - 1) / LEAF;
    const bool small = (lower ? tm * (tm + 1) / 2 : tm * tn) < SMALL_GRID;
    const int64_t t32 = (m + 31) / 32;
    if (lower && t32 * (t32 + 1) / 2 < SMALL_GRID / 2) {
        const int64_t Tn = (m + 15) / 16;
        const dim3 grid((unsigned)(Tn * (Tn + 1) / 2));
        if (pdl)
            GPCH_CUDA(ctx, gpch::launch_pdl(gemm_nt_minus_kernel<T, true, 16>, grid, dim3(256), 0, st, m, nn, k, A,
                                            lda, B, ldb, C, ldc, info));
        else
            gemm_nt_minus_kernel<T, true, 16><<<grid, 256, 0, st>>>(m, nn, k, A, lda, B, ldb, C, ldc, info);
    } else if (lower) {
        if (small) {
            const int64_t Tn = (m + 31) / 32;
            gemm_nt_minus_kernel<T, true, 32><<<(unsigned)(Tn * (Tn + 1) / 2), 256, 0, st>>>(m, nn, k, A, lda, B, ldb,
                                                                                           C, ldc, info);
        } else {
            gemm_nt_minus_kernel<T, true, 64><<<(unsigned)(tm * (tm + 1) / 2), 256, 0, st>>>(m, nn, k, A, lda, B, ldb,
                                                                                           C, ldc, info);
        }
    } else {
        if (small) {
            dim3 grid((unsigned)((m + 31) / 32), (unsigned)((nn + 31) / 32));
            gemm_nt_minus_kernel<T, false, 32><<<grid, 256, 0, st>>>(m, nn, k, A, lda, B, ldb, C, ldc, info);
        } else {
            dim3 grid((unsigned)tm, (unsigned)tn);
            gemm_nt_minus_kernel<T, false, 64><<<grid, 256, 0, st>>>(m, nn, k, A, lda, B, ldb, C, ldc, info);
        }
    }
    GPCH_LAUNCH_CHECK(ctx);
    return GPCH_OK;
}

template <typename T, int ROWS>
inline gpch_status launch_trsm_rows(gpch_ctx *ctx, T *B, int64_t ldb, int64_t m, int nc, const double *Linv,
                                    const int64_t *info, cudaStream_t st)
{
    static bool attr_done = false;
    if (!attr_done) {
        GPCH_CUDA(ctx, cudaFuncSetAttribute(trsm_inv_kernel<T, ROWS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)trsm_smem_bytes<T, ROWS>()));
        attr_done = true;
    }
    trsm_inv_kernel<T, ROWS><<<(unsigned)((m + ROWS - 1) / ROWS), 256, trsm_smem_bytes<T, ROWS>(), st>>>(
        B, ldb, m, nc, Linv, info);
    GPCH_LAUNCH_CHECK(ctx);
    return GPCH_OK;
}

// X = B L^-T by substitution (trsm_sub_kernel); FP64 panels take one row
// per warp (their cost is FP64 issue), FP32 panels four.
template <typename T>
inline gpch_status launch_trsm_sub(gpch_ctx *ctx, T *B, int64_t ldb, int64_t m, int nc, const double *L,
                                   int64_t ldl, const double *rinv, const int64_t *info, cudaStream_t st,
                                   bool pdl = false)
{
    if (m <= 0 || nc <= 0) return GPCH_OK;
    constexpr int RPW = sizeof(T) == 4 ? 4 : 1;
    if (sizeof(T) == 8 && nc <= 32) {
        // narrow FP64 blocks: one warp per SM sub-partition, so each row's
        // chain of FP64 instructions is not interleaved with another warp's
        const dim3 grid((unsigned)((m + 3) / 4));
        if (pdl)
            GPCH_CUDA(ctx, gpch::launch_pdl(trsm_sub_kernel<T, 1, 4, true>, grid, dim3(128), 0, st, B, ldb, m, nc, L,
                                            ldl, rinv, info));
        else
            trsm_sub_kernel<T, 1, 4, true><<<grid, 128, 0, st>>>(B, ldb, m, nc, L, ldl, rinv, info);
        GPCH_LAUNCH_CHECK(ctx);
        return GPCH_OK;
    }
    trsm_sub_kernel<T, RPW><<<(unsigned)((m + 8 * RPW - 1) / (8 * RPW)), 256, 0, st>>>(B, ldb, m, nc, L, ldl, rinv,
                                                                                     info);
    GPCH_LAUNCH_CHECK(ctx);
    return GPCH_OK;
}

template <typename T>
inline gpch_status launch_trsm(gpch_ctx *ctx, T *B, int64_t ldb, int64_t m, int nc, const double *Linv,
                               const int64_t *info, cudaStream_t st)
{
    if (m <= 0) return GPCH_OK;
    if ((m + LEAF - 1) / LEAF < SMALL_GRID) return launch_trsm_rows<T, 16>(ctx, B, ldb, m, nc, Linv, info, st);
    return launch_trsm_rows<T, 64>(ctx, B, ldb, m, nc, Linv, info, st);
}

}  // namespace

namespace gpch {

// Enqueue the FP64 blocked factorization (chol_fp64.cu).  rinv: workspace
// of `tile` doubles that receives 1 / L_cc of the last diagonal tile
// factored (a caller that factors one tile reads it afterwards).  A failed
// pivot at local column c sets *info = col_offset + c + 1.
gpch_status chol_fp64_enqueue(gpch_ctx *ctx, int64_t n, int tile, double *A, int64_t lda, double *rinv,
                              int64_t *info, cudaStream_t st, int64_t col_offset);

// Forward/back substitution (solve.cu).  SolveWs is carved from
// solve_ws_bytes(n, nrhs) bytes of workspace; solve_prepare inverts the
// diagonal blocks of L once per factor, solve_apply then overwrites B
// (n x nrhs) with (L L^T)^-1 B.  The _f32 forms take an FP32 factor.
struct SolveWs {
    double *Linv;                   // inverted diagonal blocks (FP32 values for an FP32 factor)
    double *Y;                      // forward-sweep result
    unsigned *flags;                // per-block "solved" flags, FP64 sweeps
    unsigned long long *tagw;       // tagged (value, tag) words, FP32 sweeps
    size_t tagw_words;
    float *Linv128;                 // 128 x 128 diagonal-block inverses, FP32 factor
    int *err;
    unsigned epoch;
};
size_t solve_ws_bytes(int64_t n, int nrhs);
SolveWs carve_solve(void *base, int64_t n, int nrhs);
gpch_status solve_prepare(gpch_ctx *ctx, int64_t n, const double *L, int64_t ldl, SolveWs &w, cudaStream_t st);
gpch_status solve_prepare_f32(gpch_ctx *ctx, int64_t n, const float *L, int64_t ldl, SolveWs &w, cudaStream_t st);
gpch_status solve_apply(gpch_ctx *ctx, int64_t n, const double *L, int64_t ldl, double *B, int64_t ldb, int nrhs,
                        SolveWs &w, cudaStream_t st);
gpch_status solve_apply_f32(gpch_ctx *ctx, int64_t n, const float *L, int64_t ldl, double *B, int64_t ldb, int nrhs,
                            SolveWs &w, cudaStream_t st);

// Low-precision factor (mixed.cu): workspace size, W = A + shift I, and the
// factorization of W in place (info / err device words returned).
size_t mixed_ws_bytes(int64_t n, int tile);
gpch_status mixed_init_enqueue(gpch_ctx *ctx, int64_t n, const double *A, int64_t lda, float *W, int64_t ldw,
                               double shift, cudaStream_t st);
gpch_status mixed_factor_enqueue(gpch_ctx *ctx, int64_t n, int tile, float *W, int64_t ldw, int prec, void *wsbase,
                                 int64_t **info_out, int **err_out, cudaStream_t st);

}  // namespace gpch
