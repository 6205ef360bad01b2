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

// FP64 code that a branch skips still costs its issue time on this GPU when
// the compiler predicates it instead of branching around it (an FP64
// instruction holds its warp for about 64 cycles whether or not any lane
// executes it).  The rare paths of the pivot helpers below are therefore
// kept out of line, behind a branch that is almost never taken.
static __device__ __noinline__ double pivot_div_slow(double d) { return 1.0 / d; }

static __device__ __noinline__ double2 pivot_sqrt_slow(double d)
{
    const double s = sqrt(d);
    return make_double2(s, 1.0 / s);
}

// True when d is positive, finite and within 2^-100 .. 2^101 (exponent bits
// read with integer instructions, no FP64 compare).
__device__ __forceinline__ bool pivot_in_fast_range(double d)
{
    const int ex = (int)(__double_as_longlong(d) >> 52);   // < 0 when the sign bit is set
    return ex >= 1023 - 100 && ex <= 1023 + 100;
}

// Square root and reciprocal square root of a positive pivot d, by Newton
// iteration on y = 1/sqrt(d) from an FP32 seed: each step
// y <- y (3 - d y^2) / 2 doubles the correct bits (24 -> 48 -> full), then
// s = d y is corrected once by s <- s + y (d - s^2) / 2.  Both results are
// within a few units in the last place; the exact cases (d = 1, perfect
// squares of small integers) come out exact.  Outside 2^-100 .. 2^101 the
// division-based form is used.
__device__ inline void pivot_sqrt(double d, double &s, double &y)
{
    if (pivot_in_fast_range(d)) {
        y = (double)__frsqrt_rn((float)d);
        y = y * fma(-0.5 * d, y * y, 1.5);
        y = y * fma(-0.5 * d, y * y, 1.5);
        s = d * y;
        s = fma(0.5 * y, fma(-s, s, d), s);
    } else {
        const double2 r = pivot_sqrt_slow(d);
        s = r.x;
        y = r.y;
    }
}

// Reciprocal of a positive pivot d: FP32 seed y0 (rcp.approx), then one
// Newton-Raphson step taken to third order, y = y0 (1 + e + e^2) with
// e = 1 - d y0 (the truncated series of 1 / (1 - e)); with |e| < 2^-21 the
// truncation error is below 2^-63, so the result is within about one unit
// in the last place.  Outside 2^-100 .. 2^101 the division is used.
__device__ inline double pivot_rcp(double d)
{
    if (pivot_in_fast_range(d)) {
        float yf;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"((float)d));
        const double y0 = (double)yf;
        const double e = fma(-d, y0, 1.0);
        return fma(y0, fma(e, e, e), y0);
    }
    return pivot_div_slow(d);
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

// Pivot test and reciprocal for the critical chain of a leaf, with as few
// FP64 instructions as possible (each one occupies its warp for about 64
// cycles, so the chain's length is their count).  The positivity / range
// test reads the exponent bits with integer instructions.  For
// 2^-100 <= d < 2^101: y0 = rcp.approx.ftz.f64(d), e = 1 - d y0,
// 1/d ~ y0 (1 + e + e^2).  The seed's relative error measured on this GPU is
// below 2^-19.9 (4M samples over 2^-100..2^100), so the truncation term e^3
// is below 2^-59 and the result is within one unit in the last place of the
// correctly rounded quotient.  Other positive finite pivots take the
// out-of-line division.  Returns false for d <= 0, inf or NaN.
__device__ inline bool pivot_rcp_short(double d, double &rd)
{
    if (pivot_in_fast_range(d)) {
        double y0;
        asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y0) : "d"(d));
        const double e = fma(-d, y0, 1.0);
        rd = fma(y0, fma(e, e, e), y0);
        return true;
    }
    const long long bits = __double_as_longlong(d);
    if (bits > 0 && (int)(bits >> 52) < 2047) {
        rd = pivot_div_slow(d);
        return true;
    }
    return false;
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

// Position p of the W-wide leaf's entry order -> (row, column).  The order
// runs over columns W-1, W-2, ..., 0 (column c holds W - c entries) and,
// inside a column, over rows W-1 down to c, so the diagonal entry closes
// its column.  Block k = W - c starts at (k - 1) k / 2.
template <int W>
__device__ __forceinline__ void leaf_entry(int p, int &r, int &c)
{
    const int k = (int)((1.0f + sqrtf((float)(8 * p + 1))) * 0.5f);   // exact: 8p + 1 < 2^24
    const int i = p - (k - 1) * k / 2;
    c = W - k;
    r = W - 1 - i;
}

// One bulk step of potrf_leaf_pipe with NQ live slots in this warp: apply
// column j - 1 to this thread's live entries, S[r][c] -= S[r][j-1] l_c, with
// l_c = S[c][j-1] / D_{j-1} in lw.  Operands are read first and stores come
// last, so the NQ FP64 instructions issue back to back; an entry at or past
// `active` (the diagonal (j, j), finished by the chain) is computed but not
// stored.  rc[q] packs slot q's entry as row | column << 8.
template <int W, int NQ>
__device__ __forceinline__ void leaf_bulk(double (*S)[W + 1], const double *lw, int j, int b, int active,
                                          const int *rc)
{
    double x[NQ], y[NQ], l[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int r = rc[q] & 0xff, c = rc[q] >> 8;
        x[q] = S[r][j - 1];
        y[q] = S[r][c];
        l[q] = lw[c];
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) y[q] = fma(-x[q], l[q], y[q]);
#pragma unroll
    for (int q = 0; q < NQ; ++q)
        if (q * 96 + b < active) S[rc[q] & 0xff][rc[q] >> 8] = y[q];
}

// The bulk warps' steps, one loop per live-slot count: the loop for NQ runs
// while this warp has exactly NQ slots with a live lane (the count only
// falls as j grows), then hands over to NQ - 1.  Every iteration ends with
// the CTA barrier of its step.
template <int W, int NQ>
__device__ __forceinline__ void leaf_bulk_phases(double (*S)[W + 1], double *lw, const double *rdv, const int *rc,
                                                 const int *bad, int &j, int nb, int b, int bw, int lane,
                                                 bool &stop, double *u2v)
{
    for (; !stop && j < nb; ++j) {
        const int live = (W - j) * (W - j + 1) / 2 - 1;
        if ((live - bw + 95) / 96 < NQ) break;
        const double rd = rdv[j - 1];
#pragma unroll
        for (int c = lane; c < W; c += 32) lw[c] = S[c][j - 1] * rd;
        __syncwarp();
        leaf_bulk<W, NQ>(S, lw, j, b, live, rc);
        if (j + 1 < W) {
            // entry (j+1, j) is final now; the warp that updated it squares it
            // for the chain's next pivot (position of the entry in the order
            // of leaf_entry: column j's block, second to last)
            const int p = (W - 1 - j) * (W - j) / 2 + (W - 2 - j);
            if ((p % 96) / 32 == (b >> 5)) {
                __syncwarp();
                if (lane == 0) {
                    const double u = S[j + 1][j];
                    u2v[j + 1] = u * u;
                }
            }
        }
        __syncthreads();
        const int f = *bad;
        stop = (f != 0 && f <= j + 1);
    }
    if constexpr (NQ > 1) leaf_bulk_phases<W, NQ - 1>(S, lw, rdv, rc, bad, j, nb, b, bw, lane, stop, u2v);
}

// Step 1 leaf of width W (32 or 64), one CTA of 128 threads.
// Square-root-free sweep (the block is reduced to L' D L'^T with
// S[r][c] = L_rc sqrt(D_c) below the diagonal; the square roots are taken
// once at the end), pipelined so that the serial pivot chain is as short as
// the FP64 units allow.  On this GPU each SM sub-partition retires one FP64
// warp instruction per ~64 cycles, whatever the number of active lanes (an
// instruction predicated off for every lane costs the same), and warp w
// runs on sub-partition w % 4.  Hence:
//   warp 0 (the chain), step j:  D_j = s_j - u_j (u_j / D_{j-1}) with
//       u_j = S[j][j-1] (final) and s_j = S[j][j] (updated through column
//       j-2), then 1 / D_j (pivot_rcp_short): five FP64 instructions;
//   warps 1-3 (the bulk, one per remaining sub-partition), step j: apply
//       column j-1 to every entry (r, c) with r >= c >= j except (j, j).
// The W(W-1)/2 updatable entries (1 <= c <= r < W) are dealt to the 96
// bulk threads cyclically in the order of leaf_entry, so the entries live
// at step j form a prefix of that order whose last element is (j, j); each
// warp runs a loop per live-slot count, so no FP64 instruction is issued
// for a slot without a live lane.  One barrier per column.  Outputs as
// potrf_leaf_body: A (lower nb x nb, nb <= W) overwritten by L,
// rinv[c] = 1 / L_cc (1 in the padding), *info = col0 + c + 1 on a failed
// pivot (D_c <= 0 or not finite).
template <int W>
__device__ inline void potrf_leaf_pipe(double *A, int64_t lda, int nb, double *rinv, int64_t col0, int64_t *info)
{
    static_assert(W == 32 || W == 64, "leaf width");
    constexpr int THREADS = 128, NBULK = 96;
    constexpr int NE = W * (W - 1) / 2;                  // entries with 1 <= c <= r < W
    constexpr int PER = (NE + NBULK - 1) / NBULK;        // 6 (W = 32) or 21 (W = 64)
    __shared__ double S[W][W + 1];   // S[r][c]
    __shared__ double rdv[W], dpiv[W], sqv[W], rsv[W];
    __shared__ double lws[3][W];     // l_c of the current step, one copy per bulk warp
    __shared__ double u2v[W];        // u2v[j] = S[j][j-1]^2 (final), left by the bulk for the chain
    __shared__ int bad;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // an earlier failed pivot stops the chain; the word is read together
    // with the block and tested once the block is in shared memory
    const int64_t info0 = *info;
    {
        // all loads of a thread in flight at once
        constexpr int NL = W * W / THREADS;
        double v[NL];
#pragma unroll
        for (int i = 0; i < NL; ++i) {
            const int e = tid + i * THREADS, r = e % W, c = e / W;
            v[i] = (r < nb && c < nb && r >= c) ? A[r + c * lda] : 0.0;
        }
#pragma unroll
        for (int i = 0; i < NL; ++i) {
            const int e = tid + i * THREADS, r = e % W, c = e / W;
            S[r][c] = (r < nb && c < nb) ? v[i] : ((r == c) ? 1.0 : 0.0);
        }
    }
    if (info0 != 0) return;   // the same value in every thread
    if (tid == 0) bad = 0;
    __syncthreads();
    if (warp == 0) {
        double rdp = 0.0;   // 1 / D_{j-1}
        for (int j = 0; j < nb; ++j) {
            double d;
            if (j == 0) d = S[0][0];
            else d = fma(-u2v[j], rdp, S[j][j]);
            double rd = 0.0;
            const bool ok = gpch::pivot_rcp_short(d, rd);
            if (lane == 0) {
                if (!ok) bad = j + 1;
                dpiv[j] = d;
                rdv[j] = rd;
            }
            rdp = rd;
            __syncthreads();
            // a failure of step j is seen by every thread after this barrier
            // (the chain warp knows its own outcome)
            if (!ok) break;
        }
    } else {
        const int b = tid - 32;          // bulk index, 0..95
        const int bw = (warp - 1) * 32;  // first bulk index of this warp
        int rc[PER];
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int p = q * NBULK + b;
            int r = 1, c = 1;
            if (p < NE) leaf_entry<W>(p, r, c);
            rc[q] = r | (c << 8);
        }
        bool stop = false;
        // step 0 has no bulk work but the chain's input of step 1
        if (tid == 32) u2v[1] = S[1][0] * S[1][0];
        __syncthreads();
        {
            const int f = bad;
            stop = (f != 0 && f <= 1);
        }
        int j = 1;
        leaf_bulk_phases<W, PER>(S, lws[warp - 1], rdv, rc, &bad, j, nb, b, bw, lane, stop, u2v);
        for (; !stop && j < nb; ++j) {
            __syncthreads();
            const int f = bad;
            stop = (f != 0 && f <= j + 1);
        }
    }
    if (bad) {
        if (tid == 0) *info = col0 + bad;
        return;
    }
    for (int c = tid; c < W; c += THREADS) {
        double sq = 1.0, rs = 1.0;
        if (c < nb) gpch::pivot_sqrt(dpiv[c], sq, rs);
        sqv[c] = sq;
        rsv[c] = rs;
    }
    __syncthreads();
    // the lower triangle including the diagonal: the positions of
    // leaf_entry extended by column 0 (block k = W)
    for (int p = tid; p < W * (W + 1) / 2; p += THREADS) {
        int r, c;
        leaf_entry<W>(p, r, c);
        if (r < nb && c < nb) A[r + c * lda] = (r == c) ? sqv[c] : S[r][c] * rsv[c];
    }
    if (rinv) for (int c = tid; c < W; c += THREADS) rinv[c] = rsv[c];
}

// Panel solve by substitution: X = B L^-T in place on the m x nc FP64 panel
// B (nc <= NC, NC = 32 or 64), with L a lower nc x nc block (ld ldl) and
// rinv its diagonal reciprocals.  Row by row, x L^T = b is solved with the
// unit lower L' = L diag(rinv) (L'_kc = L_kc / L_cc): the running values y
// start as b, column c takes y_c as it stands and subtracts y_c L'_kc from
// every y_k, k > c, and x = y diag(rinv) at the end; the same products as
// the textbook x_c = b_c / L_cc form, without a multiplication on the
// per-column chain.  One warp per RPW rows, four warps (one per SM
// sub-partition, so a row's chain of FP64 instructions is not interleaved
// with another warp's); lane l holds columns l and l + 32.  Columns are
// walked with runtime trip counts, so no FP64 instruction is issued for a
// column that does not exist (on this GPU an FP64 instruction costs its
// issue time even when every lane is predicated off).
template <int NC, int RPW>
__global__ void __launch_bounds__(128) trsm_unit_kernel(double *B, int64_t ldb, int64_t m, int nc,
                                                        const double *__restrict__ L, int64_t ldl,
                                                        const double *__restrict__ rinv, const int64_t *info)
{
    static_assert(NC == 32 || NC == 64, "block width");
    constexpr int WARPS = 4, ROWS = WARPS * RPW, H = NC / 32;
    __shared__ double Ls[NC][NC + 1];   // Ls[k][c] = L'_kc for k > c, else 0
    __shared__ double rs[NC];
    __shared__ double Bs[NC][ROWS + 1];
    gpch::pdl_wait();
    gpch::pdl_trigger();
    // read with the operands, tested before the first barrier
    const int64_t info0 = info ? *info : 0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * ROWS;
#pragma unroll 8
    for (int e = tid; e < NC * NC; e += 128) {
        const int k = e % NC, c = e / NC;   // column-major walk: coalesced
        Ls[k][c] = (k > c && k < nc && c < nc) ? L[k + (int64_t)c * ldl] : 0.0;
    }
    if (tid < NC) rs[tid] = tid < nc ? rinv[tid] : 1.0;
#pragma unroll 4
    for (int e = tid; e < NC * ROWS; e += 128) {
        const int r = e % ROWS, k = e / ROWS;
        Bs[k][r] = (r0 + r < m && k < nc) ? B[(r0 + r) + (int64_t)k * ldb] : 0.0;
    }
    if (info0 != 0) return;   // the same value in every thread
    __syncthreads();
    // L' = L diag(rinv) over the lower triangle (positions of leaf_entry;
    // the diagonal and the padding hold zeros, so every product is issued
    // without a predicate)
#pragma unroll 4
    for (int p = tid; p < NC * (NC + 1) / 2; p += 128) {
        int k, c;
        leaf_entry<NC>(p, k, c);
        Ls[k][c] *= rs[c];
    }
    __syncthreads();
    double y[H][RPW];
#pragma unroll
    for (int h = 0; h < H; ++h)
#pragma unroll
        for (int q = 0; q < RPW; ++q) y[h][q] = Bs[lane + 32 * h][warp * RPW + q];
    const int n0 = nc < 32 ? nc : 32;
    for (int c = 0; c < n0; ++c) {
        double l[H];
#pragma unroll
        for (int h = 0; h < H; ++h) l[h] = Ls[lane + 32 * h][c];
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            const double yc = __shfl_sync(0xffffffffu, y[0][q], c);
#pragma unroll
            for (int h = 0; h < H; ++h) y[h][q] = fma(-yc, l[h], y[h][q]);
        }
    }
    if (H == 2) {
        for (int c = 32; c < nc; ++c) {
            const double l1 = Ls[lane + 32][c];
#pragma unroll
            for (int q = 0; q < RPW; ++q) {
                const double yc = __shfl_sync(0xffffffffu, y[H - 1][q], c - 32);
                y[H - 1][q] = fma(-yc, l1, y[H - 1][q]);
            }
        }
    }
#pragma unroll
    for (int h = 0; h < H; ++h) {
        const double r = rs[lane + 32 * h];
#pragma unroll
        for (int q = 0; q < RPW; ++q) Bs[lane + 32 * h][warp * RPW + q] = y[h][q] * r;
    }
    __syncthreads();
#pragma unroll 4
    for (int e = tid; e < NC * ROWS; e += 128) {
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
                                          int64_t tj, bool stop = false)
{
    constexpr int KC = 32, RT = BT / 16;
    __shared__ T As[KC][BT];
    __shared__ T Bs[KC][BT];
    const int64_t r0 = ti * BT, c0 = tj * BT;
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    T acc[RT][RT] = {};
    // small tiles (the latency-bound steps inside a diagonal tile) load
    // their C entries together with the first operands instead of after
    // the product
    constexpr bool early_c = BT <= 32;
    T cold[early_c ? RT : 1][early_c ? RT : 1];
    if constexpr (early_c) {
#pragma unroll
        for (int i = 0; i < RT; ++i)
#pragma unroll
            for (int j = 0; j < RT; ++j) {
                const int64_t r = r0 + tx + 16 * i, c = c0 + ty + 16 * j;
                cold[i][j] = (r < m && c < nn && (!LOWER || r >= c)) ? C[r + c * ldc] : T(0);
            }
    }
    for (int k0 = 0; k0 < k; k0 += KC) {
        for (int e = tid; e < KC * BT; e += blockDim.x) {
            int r = e % BT, kk = e / BT;
            bool kin = k0 + kk < k;
            As[kk][r] = (kin && r0 + r < m) ? A[(r0 + r) + (int64_t)(k0 + kk) * lda] : T(0);
            Bs[kk][r] = (kin && c0 + r < nn) ? B[(c0 + r) + (int64_t)(k0 + kk) * ldb] : T(0);
        }
        if (stop) return;   // the same value in every thread, before the first barrier
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
            if (r < m && c < nn && (!LOWER || r >= c)) {
                if constexpr (early_c)
                    C[r + c * ldc] = cold[i][j] - acc[i][j];
                else
                    C[r + c * ldc] -= acc[i][j];
            }
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
    // an earlier failed pivot stops the kernel: the word is read here and
    // tested once the first operands are in flight
    const bool stop = info && *info != 0;
    int64_t ti, tj;
    if (LOWER) {
        tri_index(blockIdx.x, ti, tj);
    } else {
        ti = blockIdx.x;
        tj = blockIdx.y;
    }
    gemm_nt_minus_body<T, LOWER, BT>(m, nn, k, A, lda, B, ldb, C, ldc, ti, tj, stop);
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
    static gpch::DeviceOnce attr_once;
    GPCH_CHECK(gpch::once_per_device(ctx, attr_once, [&]() -> gpch_status {
        GPCH_CUDA(ctx, cudaFuncSetAttribute(trsm_inv_kernel<T, ROWS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)trsm_smem_bytes<T, ROWS>()));
        return GPCH_OK;
    }));
    trsm_inv_kernel<T, ROWS><<<(unsigned)((m + ROWS - 1) / ROWS), 256, trsm_smem_bytes<T, ROWS>(), st>>>(
        B, ldb, m, nc, Linv, info);
    GPCH_LAUNCH_CHECK(ctx);
    return GPCH_OK;
}

// X = B L^-T by substitution (trsm_unit_kernel) for an FP64 panel of
// m x nc, nc <= 64.  Short panels (the steps inside a diagonal tile) take
// one row per warp, so the chain of each row starts at once on its own
// sub-partition; long panels take four rows per warp, which spreads the
// shared prologue over more rows.
inline gpch_status launch_trsm_sub(gpch_ctx *ctx, double *B, int64_t ldb, int64_t m, int nc, const double *L,
                                   int64_t ldl, const double *rinv, const int64_t *info, cudaStream_t st,
                                   bool pdl = false)
{
    if (m <= 0 || nc <= 0) return GPCH_OK;
    const bool wide = nc > 32, many = m > 1024;
    auto go = [&](auto kern, int rows) -> gpch_status {
        const dim3 grid((unsigned)((m + rows - 1) / rows));
        if (pdl)
            GPCH_CUDA(ctx, gpch::launch_pdl(kern, grid, dim3(128), 0, st, B, ldb, m, nc, L, ldl, rinv, info));
        else
            kern<<<grid, 128, 0, st>>>(B, ldb, m, nc, L, ldl, rinv, info);
        GPCH_LAUNCH_CHECK(ctx);
        return GPCH_OK;
    };
    if (wide) return many ? go(trsm_unit_kernel<64, 4>, 16) : go(trsm_unit_kernel<64, 1>, 4);
    return many ? go(trsm_unit_kernel<32, 4>, 16) : go(trsm_unit_kernel<32, 1>, 4);
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
// pivot at local column c sets *info = col_offset + c + 1.  With oz_ws
// (oz_ws_bytes(n, n, true) bytes) step 3 takes the FP64-accurate
// tensor-core product; *oz_err (nullptr on entry) then receives its status
// word.
gpch_status chol_fp64_enqueue(gpch_ctx *ctx, int64_t n, int tile, double *A, int64_t lda, double *rinv,
                              int64_t *info, cudaStream_t st, int64_t col_offset, void *oz_ws = nullptr,
                              int **oz_err = nullptr);

// FP64-accurate C -= A B^T on the tensor cores (ozaki.cu): workspace bytes,
// and the enqueue.  *err_out receives the status word's address; it is
// cleared on the stream when *err_out is nullptr on entry (a caller making
// several calls keeps the first call's word, so no failure is lost).
size_t oz_ws_bytes(int64_t m, int64_t n, bool same);
gpch_status oz_gemm_enqueue(gpch_ctx *ctx, int64_t m, int64_t n, int64_t k, const double *A, int64_t lda,
                            const double *B, int64_t ldb, double *C, int64_t ldc, bool lower, void *ws,
                            cudaStream_t st, int **err_out);

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
    float *F128, *G128;             // forward and back coupling blocks of the 128-row FP32 sweeps
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

// Head and tail of 2^-ea a for an FP64 a, from its bit pattern with integer
// operations only (a float conversion would run on the FP64 pipe).  The
// head is the top 24 significand bits (truncated), the tail the next 23,
// so |2^-ea a - head - tail| < 2^-46 |2^-ea a|.  ebias = 896 + ea.  Scaled
// values below 2^-126 give head 0 (and below 2^-103 tail 0); values at or
// above 2^128 give an infinite head, so the product is not finite.
__device__ __forceinline__ void df_split_a(double a, unsigned ebias, float &head, float &tail)
{
    const unsigned long long bits = (unsigned long long)__double_as_longlong(a);
    const unsigned h = (unsigned)(bits >> 32), l = (unsigned)bits;
    const unsigned t = h & 0x7fffffffu;      // exponent field E at bits 20..30
    const unsigned sgn = h & 0x80000000u;
    // (E << 23 | top 23 fraction bits) modulo 2^32, rebiased to E - ebias
    const unsigned hb = __funnelshift_l(l, t, 3) - (ebias << 23);
    const bool small = t < ((ebias + 1u) << 20);
    const bool big = t >= ((ebias + 255u) << 20);
    const unsigned hbits = small ? 0u : (big ? 0x7f800000u : hb);
    head = __uint_as_float(hbits | sgn);
    // tail: fraction bits 6..28 of the low word, weighted 2^(E - ebias - 150)
    // as the difference of two floats with exponent field E - ebias - 23
    const unsigned mb = (hb & 0x7f800000u) - (23u << 23);
    const unsigned fb = mb | ((l >> 6) & 0x007fffffu);
    const bool tail_ok = t >= ((ebias + 24u) << 20) && !big;
    tail = tail_ok ? __uint_as_float(fb | sgn) - __uint_as_float(mb | sgn) : 0.0f;
}

// The packed copy of a symmetric A's lower triangle that the refinement's
// products read (float2 (head, tail) of 2^-ea A_ij per stored entry, as
// df_split_a cuts it): strip J holds columns SYM_STRIP J .. + SYM_STRIP - 1,
// rows SYM_STRIP J .. n2 - 1 (n2 = n rounded up to even), column-major with
// ld n2 - SYM_STRIP J, from float2 offset sy_off(n, J); sy_off(n, strips)
// is its size.
constexpr int SYM_STRIP = 256;
__host__ __device__ inline int64_t sy_off(int64_t n, int64_t J)
{
    const int64_t n2 = (n + 1) & ~int64_t(1);
    return (int64_t)SYM_STRIP * (J * n2 - (int64_t)(SYM_STRIP / 2) * J * (J - 1));
}

// Low-precision factor (mixed.cu): workspace size, W = A + shift I (and,
// with anorm and norm_ws, ||A||_inf of the symmetric A into *anorm), and the
// factorization of W in place (info / err device words returned).
size_t mixed_ws_bytes(int64_t n, int tile);
gpch_status mixed_init_enqueue(gpch_ctx *ctx, int64_t n, const double *A, int64_t lda, float *W, int64_t ldw,
                               double shift, cudaStream_t st, double *anorm = nullptr, float *norm_ws = nullptr);
size_t anorm_ws_floats(int64_t n);   // workspace of the ||A||_inf pieces (floats)
// The input pass W = A + shift I (with ||A||_inf into *anorm through
// norm_ws) run by the factor itself, block column by block column on a
// stream of its own, each part of the factor waiting only for the block
// columns it touches.
struct MixedInit {
    const double *A;
    int64_t lda;
    double shift;
    double *anorm;
    float *norm_ws;
    float2 *packed;      // optional: the refinement's packed copy, written in the same pass
    unsigned ebias;      // its df_split_a exponent offset (896 + ea)
};
gpch_status mixed_factor_enqueue(gpch_ctx *ctx, int64_t n, int tile, float *W, int64_t ldw, int prec, void *wsbase,
                                 int64_t **info_out, int **err_out, cudaStream_t st, const MixedInit *init = nullptr);

}  // namespace gpch
