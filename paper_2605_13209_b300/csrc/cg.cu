// cg.cu -- A6/A7: conjugate gradients, Algorithm 1 (left), with residual
// replacement every R iterations (Sec. 2.1), for up to 16 right-hand sides
// that share one pass over the matrix per iteration; and the
// single-reduction rearrangement of the same iteration (Chronopoulos and
// Gear), one of the pipelined CG variants the paper's related work cites.
//
// Classic CG, per iteration three kernels run:
//   matvec  t = A s and the partial sums of s^T t; the last CTA to finish
//           reduces the partials in a fixed order and sets alpha = u / s^T t
//   update  x += alpha s, r -= alpha t, partial sums of r^T r; the last CTA
//           sets beta = u_new / u, u = u_new and retires converged columns
//   dir     s = r + beta s
// On a replacement iteration `update` is split into x += alpha s, a matvec
// of x, and r = b - A x.
//
// Single-reduction CG, per iteration two kernels run:
//   sr_vec  p = r + beta p, s = w + beta s (s = A p), x += alpha p,
//           r -= alpha s
//   matvec  w = A r and the partial sums of r^T r and w^T r together; the
//           last CTA sets beta = gamma'/gamma and
//           alpha = gamma' / (delta - beta gamma' / alpha), and retires
//           converged columns
// so an iteration has one reduction point instead of two.  On a
// replacement iteration r = b - A x and s = A p are recomputed.
//
// All scalars stay on the device; the host reads one "all done" word every
// few iterations.  Reductions are two-phase with a fixed order, so results
// do not depend on CTA scheduling.
//
// The matvec uses A = A^T: t_j = sum_i A_ij s_i is a dot product down column
// j, which is contiguous in column-major storage.  A CTA owns W consecutive
// columns and walks all rows with 16-byte loads (two FP64 or four FP32 rows
// per thread and step); each thread reuses its rows' vector entries across
// the W columns and NR right-hand sides.
//
// Two product arithmetics:
//   PROD_FP64  one FP64 FMA per element and right-hand side.  This part
//              issues FP64 at 2 FMAs per clock per SM, below the rate at
//              which HBM delivers FP64 elements, so this path is FP64-pipe
//              bound.
//   PROD_DF    double-float products on the FP32 pipe: every FP64 entry of
//              A is cut by integer operations into a float head (its top 24
//              significand bits) and a float tail (the next 23), the
//              vector is pre-split into float head + tail, and
//              (a_h + a_t)(s_h + s_t) is formed as a_h s_h exactly (product
//              and its FMA error term) plus a_h s_t + a_t s_h, summed per
//              thread in an error-free double-float accumulator (two-sum).
//              Per product the relative error is below about 2^-45, the
//              accumulator adds about 2^-48 of the running sum, and the
//              per-thread sums are combined and reduced in FP64.  FP32 A
//              is exact in a float, so only the vector is split.  Powers
//              of two bring A's largest entry and each column of the vector
//              near 1 first, so FP32's exponent range holds them.
//              True residuals b - A x (the start and every replacement)
//              always take FP64 products: they bound the accuracy the
//              iteration can reach, and they are 1/R of the products.
//   PROD_OZ    FP64-accurate products on the bf16 tensor cores, the
//              error-free splitting of ozaki.cu: A (as A^T, its columns)
//              is cut once per solve into 8 base-128 digits per entry with
//              one power-of-two scale per column and 512-row pass, the
//              vectors every matvec likewise per right-hand side; a CTA
//              forms 128 entries of A s for all right-hand sides.  The
//              vectors' digits are stacked along N, so that one MMA takes
//              digit p of A against every kept digit d <= 6 - p of all 16
//              right-hand sides (N = 16 (7 - p)); the 28 kept digit pairs
//              are summed exactly in FP32 per pass, gathered into 7 weight
//              classes p + d in the epilogue, combined and rounded once per
//              pass, and the passes added in FP64.  The dropped classes
//              (p + d >= 7) weigh at most 2^-44 of the pass's scales per
//              term.  The digit copy takes 16 bytes per entry of A.  True
//              residuals take the same product with class 7 kept as well
//              (the dropped classes then weigh at most 2^-51 of the scales
//              per term, FP64-level).

#include <cuda_bf16.h>

#include <cmath>

#include "dense_fp64.cuh"
#include "ozaki.cuh"

namespace {

constexpr int THREADS = 256;
constexpr int MAXRHS = 16;

// PROD_OZ_FULL (internal): PROD_OZ with weight class 7 kept as well, for
// the true residuals of the tensor-core solve
enum Product : int { PROD_FP64 = 0, PROD_DF = 1, PROD_OZ = 2, PROD_OZ_FULL = 3 };
enum Variant : int { VAR_CLASSIC = 0, VAR_SINGLE_REDUCTION = 1 };
enum MvMode : int { MV_ALPHA = 0, MV_PLAIN = 1, MV_SR = 2 };

struct CGState {
    double *u, *u0, *alpha, *beta;   // [MAXRHS]  (u = gamma = r^T r in the single-reduction form)
    int *active, *iters;            // [MAXRHS]
    int *done;                      // [1]
    unsigned *counter;              // [2]: matvec, vector kernels
    double *part;                   // per-CTA partials, part_doubles(n, nrhs)
};

// Buffers of the tensor-core path: the digit copy of A^T, tile-major so
// that a CTA streams contiguous memory: for row tile rt (128 rows, the
// last padded with zeros to npad rows), K stage kc (32 columns) and plane
// b (digits 2b, 2b + 1), a block of 128 rows of 64 positions (128 bytes:
// digit p of column k at (p % 2) 32 + k % 32); its exponents
// EA[t * npad + j] (column j, pass t); the vectors' copy DS, stacked for
// one product per digit of A: for K stage kc, digit d and right-hand side
// r, row (8 kc + d) 16 + r of 32 positions (64 bytes, column k at k % 32),
// and exponents ES[t * 16 + r]; the status word of the bounded waits.  np
// passes of 512, kpt = 512 np.
struct OzArgs {
    __nv_bfloat16 *DA, *DS;
    int *EA, *ES;
    int *err;
    int np;
    int64_t kpt, npad;
};

// Inputs of the double-float path.  SS holds the pre-split vector,
// row-major by row: the (head, tail) of 2^-es_r v_ir at SS[i * NR + r].
// scale[r] = 2^(ea + es_r) restores the product's scale; inv[r] = 2^-es_r;
// *ebias = 896 + ea is the exponent offset that maps A's FP64 exponent field
// to the float exponent of 2^-ea A.
struct DFArgs {
    float2 *SS;
    const double *scale;
    const double *inv;
    const int *ebias;
    OzArgs oz;   // the tensor-core path's buffers (PROD_OZ)
};

struct SRArgs {
    double rtol2;
    int maxit;
    int first;   // the set-up product w = A r0: sets gamma_0, alpha_0, beta_0
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

// Sum of part[b * stride + idx] over the grid's CTAs b in a fixed order
// (strided per thread, then warp and block); the result is valid in thread
// 0.  All threads of the CTA must call it.
__device__ inline double block_sum_partials(const double *part, size_t stride, int idx)
{
    __shared__ double red[THREADS / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double p = 0.0;
    for (unsigned b = tid; b < gridDim.x; b += THREADS) p += __ldcg(&part[(size_t)b * stride + idx]);
    p = warp_sum(p);
    if (lane == 0) red[warp] = p;
    __syncthreads();
    double q = 0.0;
    if (tid == 0)
        for (int w = 0; w < THREADS / 32; ++w) q += red[w];
    __syncthreads();
    return q;
}

// ------------------------------------------------ double-float arithmetic

// hi + lo <- hi + lo + p + e, with hi + p taken exactly (two-sum).
__device__ __forceinline__ void df_add(float &hi, float &lo, float p, float e)
{
    const float s = hi + p;
    const float bp = s - hi;
    const float err = (hi - (s - bp)) + (p - bp);
    hi = s;
    lo += err + e;
}

// (hi, lo) += (h2, l2), two double-float values.
__device__ __forceinline__ void df_add2(float &hi, float &lo, float h2, float l2)
{
    const float s = hi + h2;
    const float bp = s - hi;
    const float err = (hi - (s - bp)) + (h2 - bp);
    hi = s;
    lo = lo + l2 + err;
}

using gpch::df_split_a;

// ------------------------------------------------------------- the matvec

// Tail of a matvec CTA, once tcol[c * NR + r] holds (A s)_(j0 + c), r for
// its W columns: store T, then the mode's partial sums and, in the last
// CTA, the mode's scalar step (see cg_matvec_kernel).
template <int W, int NR>
__device__ __forceinline__ void mv_finish(int64_t j0, int wcols, int nrhs, const double *__restrict__ S, int64_t lds,
                                          double *T, int64_t ldt, const CGState &st, int mode, const SRArgs &sr,
                                          const double *tcol)
{
    const int tid = threadIdx.x;
    __syncthreads();
    for (int e = tid; e < W * NR; e += THREADS) {
        const int c = e / NR, r = e % NR;
        if (c < wcols && r < nrhs) T[(j0 + c) + r * ldt] = tcol[e];
    }
    if (mode == MV_PLAIN) return;
    if (mode == MV_ALPHA) {
        if (tid < NR) {
            double p = 0.0;
            for (int c = 0; c < wcols; ++c)
                if (tid < nrhs) p = fma(S[(j0 + c) + tid * lds], tcol[c * NR + tid], p);
            st.part[(size_t)blockIdx.x * NR + tid] = p;
        }
        if (last_cta(&st.counter[0])) {
            for (int r = 0; r < nrhs; ++r) {
                const double q = block_sum_partials(st.part, NR, r);
                if (tid == 0) st.alpha[r] = st.active[r] ? st.u[r] / q : 0.0;
            }
            if (tid == 0) st.counter[0] = 0;
        }
        return;
    }
    // MV_SR: S is r, T is w
    if (tid < NR) {
        double g = 0.0, d = 0.0;
        for (int c = 0; c < wcols; ++c)
            if (tid < nrhs) {
                const double rj = S[(j0 + c) + tid * lds];
                g = fma(rj, rj, g);
                d = fma(tcol[c * NR + tid], rj, d);
            }
        st.part[(size_t)blockIdx.x * 2 * NR + tid] = g;
        st.part[(size_t)blockIdx.x * 2 * NR + NR + tid] = d;
    }
    if (last_cta(&st.counter[0])) {
        __shared__ int any_active;
        if (tid == 0) any_active = 0;
        for (int r = 0; r < nrhs; ++r) {
            const double g = block_sum_partials(st.part, 2 * NR, r);
            const double d = block_sum_partials(st.part, 2 * NR, NR + r);
            if (tid == 0) {
                if (sr.first) {
                    st.u0[r] = g;
                    st.u[r] = g;
                    st.iters[r] = 0;
                    st.beta[r] = 0.0;
                    st.alpha[r] = g > 0.0 ? g / d : 0.0;
                    st.active[r] = g > 0.0 ? 1 : 0;
                } else if (st.active[r]) {
                    const int it = st.iters[r] + 1;
                    st.iters[r] = it;
                    const double b = g / st.u[r];
                    st.alpha[r] = g / (d - b * g / st.alpha[r]);
                    st.beta[r] = b;
                    st.u[r] = g;
                    if (g <= sr.rtol2 * st.u0[r] || it >= sr.maxit) st.active[r] = 0;
                }
                any_active |= st.active[r];
            }
        }
        if (tid == 0) {
            *st.done = any_active ? 0 : 1;
            st.counter[0] = 0;
        }
    }
}

// T[:, r] = A^T S[:, r] on the CTA's W columns of the n x ncols matrix A
// (ncols = n for a whole symmetric A, where A^T S = A S), then per mode:
//   MV_ALPHA  partial s^T t; the last CTA sets alpha = u / s^T t
//   MV_PLAIN  nothing more (t = A x for a true residual)
//   MV_SR     partial r^T r and w^T r (S = r, T = w); the last CTA runs the
//             single-reduction scalar step (SRArgs)
// With DF the products read the pre-split DFArgs::SS; S itself is read only
// for the CTA's own columns (the partial dot products).
template <typename TA, int W, int NR, bool DF>
__global__ void __launch_bounds__(THREADS) cg_matvec_kernel(int64_t n, int64_t ncols, int nrhs, const TA *__restrict__ A,
                                                            int64_t lda, const double *__restrict__ S,
                                                            int64_t lds, double *T, int64_t ldt, CGState st,
                                                            int mode, SRArgs sr, DFArgs df, int vec)
{
    constexpr int RPT = 16 / sizeof(TA);            // rows per thread and step (one 16-byte load)
    constexpr int STEP = THREADS * RPT;
    constexpr bool SPLIT_A = DF && sizeof(TA) == 8;
    __shared__ double tcol[W * NR];
    if (*st.done) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t j0 = (int64_t)blockIdx.x * W;
    const int wcols = (int)((ncols - j0 < W) ? ncols - j0 : W);

    // FP64 path: acc[c][r]; DF path: head/tail pairs
    double acc[DF ? 1 : W][DF ? 1 : NR];
    float ah[DF ? W : 1][DF ? NR : 1], al[DF ? W : 1][DF ? NR : 1];
    if constexpr (DF) {
#pragma unroll
        for (int c = 0; c < W; ++c)
#pragma unroll
            for (int r = 0; r < NR; ++r) ah[c][r] = al[c][r] = 0.0f;
    } else {
#pragma unroll
        for (int c = 0; c < W; ++c)
#pragma unroll
            for (int r = 0; r < NR; ++r) acc[c][r] = 0.0;
    }
    const unsigned ebias = SPLIT_A ? (unsigned)*df.ebias : 0u;

    for (int64_t base = 0; base < n; base += STEP) {
        const int64_t row0 = base + (int64_t)tid * RPT;
        if (row0 >= n) continue;
        const bool full = vec && row0 + RPT <= n;
        // the rows' vector entries
        double sv[DF ? 1 : RPT][DF ? 1 : NR];
        float sh[DF ? RPT : 1][DF ? NR : 1], sl[DF ? RPT : 1][DF ? NR : 1];
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            const bool ok = row0 + q < n;
            if constexpr (DF) {
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const float2 v = ok ? df.SS[(row0 + q) * NR + r] : make_float2(0.0f, 0.0f);
                    sh[q][r] = v.x;
                    sl[q][r] = v.y;
                }
            } else {
#pragma unroll
                for (int r = 0; r < NR; ++r) sv[q][r] = (ok && r < nrhs) ? S[row0 + q + r * lds] : 0.0;
            }
        }
        // the W columns' entries on these rows, all loads issued first
        TA a[W][RPT];
#pragma unroll
        for (int c = 0; c < W; ++c) {
            const TA *col = A + (j0 + (c < wcols ? c : 0)) * lda + row0;
            if (full) {
                if constexpr (sizeof(TA) == 8) {
                    const double2 v = __ldcs(reinterpret_cast<const double2 *>(col));
                    a[c][0] = v.x;
                    a[c][1] = v.y;
                } else {
                    const float4 v = __ldcs(reinterpret_cast<const float4 *>(col));
                    a[c][0] = v.x;
                    a[c][1] = v.y;
                    a[c][2] = v.z;
                    a[c][3] = v.w;
                }
            } else {
#pragma unroll
                for (int q = 0; q < RPT; ++q) a[c][q] = (row0 + q < n) ? col[q] : (TA)0;
            }
        }
#pragma unroll
        for (int c = 0; c < W; ++c) {
            if (c < wcols) {
#pragma unroll
                for (int q = 0; q < RPT; ++q) {
                    if constexpr (DF) {
                        float h, t = 0.0f;
                        if constexpr (SPLIT_A) df_split_a((double)a[c][q], ebias, h, t);
                        else h = (float)a[c][q];
#pragma unroll
                        for (int r = 0; r < NR; ++r) {
                            const float p = h * sh[q][r];
                            float e = fmaf(h, sh[q][r], -p);
                            e = fmaf(h, sl[q][r], e);
                            if constexpr (SPLIT_A) e = fmaf(t, sh[q][r], e);
                            df_add(ah[c][r], al[c][r], p, e);
                        }
                    } else {
                        const double av = (double)a[c][q];
#pragma unroll
                        for (int r = 0; r < NR; ++r) acc[c][r] = fma(av, sv[q][r], acc[c][r]);
                    }
                }
            }
        }
    }

    // reduce over the CTA: warps by shuffles, then warps in warp order
    if constexpr (DF) {
        __shared__ float2 red2[THREADS / 32][W * NR];
#pragma unroll
        for (int c = 0; c < W; ++c)
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                float h = ah[c][r], l = al[c][r];
#pragma unroll
                for (int off = 16; off > 0; off >>= 1)
                    df_add2(h, l, __shfl_xor_sync(0xffffffffu, h, off), __shfl_xor_sync(0xffffffffu, l, off));
                if (lane == 0) red2[warp][c * NR + r] = make_float2(h, l);
            }
        __syncthreads();
        if (tid < W * NR) {
            float h = red2[0][tid].x, l = red2[0][tid].y;
            for (int w = 1; w < THREADS / 32; ++w) df_add2(h, l, red2[w][tid].x, red2[w][tid].y);
            const int r = tid % NR;
            tcol[tid] = ((double)h + (double)l) * (r < nrhs ? df.scale[r] : 0.0);
        }
    } else {
        __shared__ double red[THREADS / 32][W * NR];
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
        }
    }
    mv_finish<W, NR>(j0, wcols, nrhs, S, lds, T, ldt, st, mode, sr, tcol);
}

// Double-float matvec for several right-hand sides (NR = 4, 8, 16), tiled
// so that the split vector is read from L2 once per 16 columns: a CTA owns
// 16 columns, two per warp, and walks the rows in chunks of 32 * RPL rows
// (RPL = 2 FP64 or 4 FP32 rows per lane, one 16-byte load per column).
// Each chunk of the split vector is staged in shared memory, heads and
// tails in separate arrays padded to NR + 1 floats per row so that the
// lanes' rows fall in distinct banks; the next chunk's vector and matrix
// entries are loaded while the current one is computed.  Every (column,
// right-hand side) sum lives in one warp and is reduced by shuffles.
constexpr int TW = 16;                     // columns per CTA of the tiled kernel

template <typename TA, int NR>
__global__ void __launch_bounds__(THREADS) cg_matvec_df_tiled_kernel(int64_t n, int64_t ncols, int nrhs,
                                                                     const TA *__restrict__ A,
                                                                     int64_t lda, const double *__restrict__ S,
                                                                     int64_t lds, double *T, int64_t ldt,
                                                                     CGState st, int mode, SRArgs sr, DFArgs df,
                                                                     int vec)
{
    constexpr int RPL = 16 / sizeof(TA);           // rows per lane and chunk
    constexpr int KC = 32 * RPL;                   // rows per chunk
    constexpr int SPT = KC * NR / THREADS;         // split-vector pairs each thread stages per chunk
    constexpr bool SPLIT_A = sizeof(TA) == 8;
    static_assert(SPT >= 1 && KC * NR % THREADS == 0, "chunk must split evenly over the CTA");
    __shared__ float sh_s[KC][NR + 1], sl_s[KC][NR + 1];
    __shared__ double tcol[TW * NR];
    if (*st.done) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t j0 = (int64_t)blockIdx.x * TW;
    const int wcols = (int)((ncols - j0 < TW) ? ncols - j0 : TW);
    const int c0 = 2 * warp;                       // this warp's two columns (local)
    const unsigned ebias = SPLIT_A ? (unsigned)*df.ebias : 0u;
    const TA *col[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) col[c] = A + (j0 + (c0 + c < wcols ? c0 + c : 0)) * lda;

    float ah[2][NR], al[2][NR];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int r = 0; r < NR; ++r) ah[c][r] = al[c][r] = 0.0f;

    // staged loads of one chunk: split-vector pairs and this lane's rows of
    // the warp's two columns
    float2 sv[SPT];
    TA av[2][RPL];
    auto load_chunk = [&](int64_t base) {
#pragma unroll
        for (int q = 0; q < SPT; ++q) {
            const int64_t e = base * NR + (int64_t)q * THREADS + tid;   // element of SS, row-major by row
            sv[q] = (e < n * NR) ? df.SS[e] : make_float2(0.0f, 0.0f);
        }
        const int64_t row0 = base + (int64_t)lane * RPL;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            if (vec && row0 + RPL <= n) {
                if constexpr (sizeof(TA) == 8) {
                    const double2 v = __ldcs(reinterpret_cast<const double2 *>(col[c] + row0));
                    av[c][0] = v.x;
                    av[c][1] = v.y;
                } else {
                    const float4 v = __ldcs(reinterpret_cast<const float4 *>(col[c] + row0));
                    av[c][0] = v.x;
                    av[c][1] = v.y;
                    av[c][2] = v.z;
                    av[c][3] = v.w;
                }
            } else {
#pragma unroll
                for (int q = 0; q < RPL; ++q) av[c][q] = (row0 + q < n) ? col[c][row0 + q] : (TA)0;
            }
        }
    };

    load_chunk(0);
    for (int64_t base = 0; base < n; base += KC) {
        __syncthreads();                           // the previous chunk's readers are done
#pragma unroll
        for (int q = 0; q < SPT; ++q) {
            const int e = q * THREADS + tid;
            sh_s[e / NR][e % NR] = sv[q].x;
            sl_s[e / NR][e % NR] = sv[q].y;
        }
        __syncthreads();
        TA cur[2][RPL];
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int q = 0; q < RPL; ++q) cur[c][q] = av[c][q];
        if (base + KC < n) load_chunk(base + KC);
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            const int lr = lane * RPL + q;           // row within the chunk
            float h[2], t[2];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                if constexpr (SPLIT_A) {
                    df_split_a((double)cur[c][q], ebias, h[c], t[c]);
                } else {
                    h[c] = (float)cur[c][q];
                    t[c] = 0.0f;
                }
            }
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const float shv = sh_s[lr][r], slv = sl_s[lr][r];
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const float p = h[c] * shv;
                    float e = fmaf(h[c], shv, -p);
                    e = fmaf(h[c], slv, e);
                    if constexpr (SPLIT_A) e = fmaf(t[c], shv, e);
                    df_add(ah[c][r], al[c][r], p, e);
                }
            }
        }
    }
    // each (column, right-hand side) sum is spread over the warp's lanes
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            float hh = ah[c][r], ll = al[c][r];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1)
                df_add2(hh, ll, __shfl_xor_sync(0xffffffffu, hh, off), __shfl_xor_sync(0xffffffffu, ll, off));
            if (lane == 0)
                tcol[(c0 + c) * NR + r] = ((double)hh + (double)ll) * (r < nrhs ? df.scale[r] : 0.0);
        }
    mv_finish<TW, NR>(j0, wcols, nrhs, S, lds, T, ldt, st, mode, sr, tcol);
}

// ----------------------------------------------- tensor-core products

// N = round(x 2^(54 - e)) for |x| < 2^e from x's bit pattern (integer
// operations only; FP64 or FP32 x).
template <typename TX>
__device__ __forceinline__ long long oz_fixed(TX x, int e)
{
    unsigned long long mant;
    int ebits, bias;
    bool neg;
    if constexpr (sizeof(TX) == 8) {
        const unsigned long long bits = (unsigned long long)__double_as_longlong((double)x);
        const int E11 = (int)((bits >> 52) & 0x7ff);
        mant = bits & 0xfffffffffffffull;
        ebits = E11 == 0 ? 1 : E11;
        if (E11 != 0) mant |= 1ull << 52;
        bias = 1075;
        neg = (bits >> 63) != 0;
    } else {
        const unsigned bits = __float_as_uint((float)x);
        const int E8 = (int)((bits >> 23) & 0xff);
        mant = bits & 0x7fffffu;
        ebits = E8 == 0 ? 1 : E8;
        if (E8 != 0) mant |= 1u << 23;
        bias = 150;
        neg = (bits >> 31) != 0;
    }
    // x = mant 2^(ebits - bias); shift to units of 2^(e - 54)
    const int sh = ebits - bias + 54 - e;
    unsigned long long a;
    if (sh >= 0) a = mant << sh;   // sh <= 1 for FP64 (|x| < 2^e); FP32 mantissas are shorter
    else if (sh > -64) a = (mant + (1ull << (-sh - 1))) >> (-sh);
    else a = 0;
    return neg ? -(long long)a : (long long)a;
}

// Digits of the columns of X (column c: its n entries, ld ldx) for the
// tensor-core products, in the layouts of OzArgs: tiled (A's copy, rows
// 0 .. plane_rows-1) or stacked (the vectors', plane_rows = 16), with
// exponent E[t * plane_rows + c] per pass t of 512 entries (the smallest e
// with every |x| of the pass below 2^e; 0 for a zero pass).  Columns at or
// past ncols (and entries past n) are zero.  One warp per (column, pass).
template <typename TX>
__global__ void __launch_bounds__(256) oz_split_cols_kernel(int64_t n, int np, int64_t kpt, const TX *__restrict__ X,
                                                            int64_t ldx, int64_t ncols, int64_t plane_rows,
                                                            __nv_bfloat16 *__restrict__ D, int *__restrict__ E,
                                                            const int *done, int tiled)
{
    if (done && *done) return;
    const int lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int64_t c = w / np;
    const int t = (int)(w % np);
    if (c >= plane_rows) return;
    const bool valid = c < ncols;
    const int64_t k0 = (int64_t)t * 512;
    const TX *x = X + (valid ? c : 0) * ldx;
    TX v[16];
    TX mx = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int64_t k = k0 + lane + 32 * i;
        v[i] = (valid && k < n) ? x[k] : (TX)0;
        mx = mx > (v[i] < 0 ? -v[i] : v[i]) ? mx : (v[i] < 0 ? -v[i] : v[i]);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const TX o = __shfl_xor_sync(0xffffffffu, mx, off);
        mx = mx > o ? mx : o;
    }
    int e = 0;
    if (mx > (TX)0) {
        if constexpr (sizeof(TX) == 8) frexp((double)mx, &e);
        else frexpf((float)mx, &e);
    }
    if (lane == 0) E[(int64_t)t * plane_rows + c] = e;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int64_t k = k0 + lane + 32 * i;
        long long N = oz_fixed<TX>(v[i], e);
        // balanced base-128 digits, least significant first
#pragma unroll
        for (int p = 7; p >= 0; --p) {
            long long d;
            if (p > 0) {
                d = ((N + 64) & 127) - 64;
                N = (N - d) >> 7;
            } else {
                d = N;   // |N| <= 2^54 / 128^7 + 1 = 33
            }
            const int64_t at = tiled ? ((((c / 128) * (kpt / 32) + k / 32) * 4 + p / 2) * 128 + c % 128) * 64 +
                                           (p & 1) * 32 + k % 32
                                     : (((k / 32) * 8 + p) * plane_rows + c) * 32 + k % 32;
            D[at] = __float2bfloat16_rn((float)d);
        }
    }
}

// T = A s for up to 16 right-hand sides with FP64-accurate tensor-core
// products (PROD_OZ): CTA b forms rows 128 b .. 128 b + 127 of A s for all
// right-hand sides, then the mode's reductions as the other matvecs do.
// tm_a: the digit copy of A^T (tile-major, rows of 64 positions, 128-row
// boxes, 128-byte swizzle); tm_s: the vectors' stacked copy (rows of 32
// positions, 128-row boxes: 8 digits x 16 right-hand sides, 64-byte
// swizzle).  Per 32 K columns and K step of 16, digit p of A (p = 0..6)
// meets digits d = 0 .. 6 - p of all vectors in ONE MMA (M = 128,
// N = 16 (7 - p)), whose columns hold the pair sums S_pd; the 28 pairs with
// p + d <= 6 are kept (the weight classes above 6, at most 2^-44 of the
// scales' product per term, are dropped).  Roles: warp 0 lane 0 TMA (3
// stages of 4 A boxes and 1 vector box), warp 1 the TMEM (448 of 512
// columns) and its lane 0 the MMAs (14 per stage), warps 4-7 the epilogue
// (warp w: rows 32 (w % 4) .., its TMEM lanes), which per pass of 512
// forms the 7 class sums (exact: at most 7 pair sums of magnitude 2^21),
// combines them exactly, rounds once and adds in FP64.  Bounded waits set
// *oz.err.
constexpr int OZM_BM = 128;
constexpr int OZM_N = MAXRHS;
constexpr int OZM_KSTAGE = 32;
constexpr int OZM_SPP = 512 / OZM_KSTAGE;    // stages per pass
constexpr int OZM_STAGES = 3;
constexpr int OZM_CLASSES = 7;               // weight classes D = p + d kept (0..6)
constexpr uint32_t OZM_ABOX = OZM_BM * 128, OZM_SBOX = 8 * OZM_N * 64;
constexpr uint32_t OZM_STAGE = 4 * OZM_ABOX + OZM_SBOX;   // 72 KB
constexpr size_t OZM_SMEM = OZM_STAGES * OZM_STAGE + 1024 + 256;
constexpr uint32_t OZM_TMEM = 512;
constexpr uint32_t OZM_SPIN = 1u << 26;
static_assert((size_t)OZM_BM * OZM_N * sizeof(double) <= OZM_STAGES * OZM_STAGE, "tcol fits the stages");
// first TMEM column of digit p's product: 16 sum_{p' < p} (7 - p')
__host__ __device__ constexpr int ozm_base(int p) { return OZM_N * (7 * p - p * (p - 1) / 2); }

// With FULL, the eight pairs of weight class 7 (p + d = 7) are summed too,
// all into one more 16-column TMEM block (exact in FP32: at most 8 pair
// sums of 2^21), and the pass's total gains one more base-128 place: the
// dropped classes then weigh at most 2^-51 of the scales' product per term,
// FP64-level products for the true residuals.
constexpr uint32_t OZM_C7 = 448;   // TMEM column of the class-7 block
template <bool FULL>
__global__ void __launch_bounds__(THREADS, 1)
    oz_matvec_kernel(const __grid_constant__ CUtensorMap tm_a, const __grid_constant__ CUtensorMap tm_s, int64_t n,
                     int nrhs, const double *S, int64_t lds, double *T, int64_t ldt, CGState st, int mode, SRArgs sr,
                     OzArgs oz)
{
    if (*st.done) return;
    extern __shared__ __align__(1024) uint8_t ozm_smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(ozm_smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + OZM_STAGES * OZM_STAGE);
    uint64_t *empty = full + OZM_STAGES;
    uint64_t *tfull = empty + OZM_STAGES;
    uint64_t *tempty = tfull + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tempty + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i0 = (int64_t)blockIdx.x * OZM_BM;
    const int np = oz.np;
    if (threadIdx.x == 0) {
        for (int s = 0; s < OZM_STAGES; ++s) {
            gpch::tc::mbar_init(&full[s], 1);
            gpch::tc::mbar_init(&empty[s], 1);
        }
        gpch::tc::mbar_init(tfull, 1);
        gpch::tc::mbar_init(tempty, 4);
        gpch::tc::fence_mbar_init();
    }
    if (warp == 1) gpch::tc::tmem_alloc<OZM_TMEM>(tmem_slot);
    gpch::tc::tc_fence_before();
    __syncthreads();
    gpch::tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int NK = np * OZM_SPP;
    double acc64[OZM_N];
#pragma unroll
    for (int j = 0; j < OZM_N; ++j) acc64[j] = 0.0;

    if (warp == 0) {
        if (lane == 0) {
            gpch::tc::prefetch_tmap(&tm_a);
            gpch::tc::prefetch_tmap(&tm_s);
            int issued = 0;
            for (int kc = 0; kc < NK; ++kc) {
                const int s = kc % OZM_STAGES;
                if (kc >= OZM_STAGES && !gpch::tc::mbar_wait(&empty[s], ((kc / OZM_STAGES) - 1) & 1, OZM_SPIN)) {
                    atomicExch(oz.err, 1);
                    break;
                }
                uint8_t *stg = smem + s * OZM_STAGE;
                gpch::tc::mbar_arrive_expect_tx(&full[s], OZM_STAGE);
                for (int b = 0; b < 4; ++b)
                    gpch::tc::tma_load_2d(stg + b * OZM_ABOX, &tm_a, &full[s], 0,
                                          (int32_t)((((int64_t)blockIdx.x * NK + kc) * 4 + b) * OZM_BM));
                gpch::tc::tma_load_2d(stg + 4 * OZM_ABOX, &tm_s, &full[s], 0, (int32_t)(kc * 8 * OZM_N));
                ++issued;
            }
            // every copy this thread started has landed before the CTA exits
            for (int s = 0; s < OZM_STAGES && s < issued; ++s) {
                const int uses = (issued - 1 - s) / OZM_STAGES + 1;
                if (!gpch::tc::mbar_wait(&full[s], (uses - 1) & 1, OZM_SPIN)) atomicExch(oz.err, 4);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            bool ok = true;
            int kc = 0;
            for (int t = 0; t < np && ok; ++t) {
                // the accumulators must have been read out for pass t - 1
                if (t >= 1 && !gpch::tc::mbar_wait(tempty, (t - 1) & 1, 4 * OZM_SPIN)) {
                    atomicExch(oz.err, 2);
                    break;
                }
                gpch::tc::tc_fence_after();
                for (int q = 0; q < OZM_SPP; ++q, ++kc) {
                    const int s = kc % OZM_STAGES;
                    if (!gpch::tc::mbar_wait(&full[s], (kc / OZM_STAGES) & 1, OZM_SPIN)) {
                        atomicExch(oz.err, 2);
                        ok = false;
                        break;
                    }
                    gpch::tc::tc_fence_after();
                    const uint32_t sa = gpch::tc::smem_u32(smem + s * OZM_STAGE);
                    const uint64_t b = gpch::tc::sdesc_sw64(sa + 4 * OZM_ABOX);
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
#pragma unroll
                        for (int p = 0; p < OZM_CLASSES; ++p) {
                            const uint64_t a = gpch::tc::sdesc_sw128(sa + (p / 2) * OZM_ABOX) + 4 * (p & 1);
                            const uint32_t idesc = gpch::tc::idesc_bf16_f32(OZM_BM, OZM_N * (7 - p));
                            // the pass's first K step overwrites the accumulators
                            gpch::tc::mma_bf16(tmem + (uint32_t)ozm_base(p), a + 2 * k, b + 2 * k, idesc,
                                               (q > 0 || k > 0) ? 1u : 0u);
                        }
                        if constexpr (FULL) {
                            // class 7: digit p of A against digit 7 - p of the
                            // vectors (their 16 rows start (7 - p) 1024 bytes
                            // into the stacked box: +64 in the descriptor)
                            const uint32_t idesc7 = gpch::tc::idesc_bf16_f32(OZM_BM, OZM_N);
#pragma unroll
                            for (int p = 0; p < 8; ++p) {
                                const uint64_t a = gpch::tc::sdesc_sw128(sa + (p / 2) * OZM_ABOX) + 4 * (p & 1);
                                gpch::tc::mma_bf16(tmem + OZM_C7, a + 2 * k, b + (uint64_t)(64 * (7 - p)) + 2 * k,
                                                   idesc7, (q > 0 || k > 0 || p > 0) ? 1u : 0u);
                            }
                        }
                    }
                    gpch::tc::mma_commit(&empty[s]);
                }
                if (ok) gpch::tc::mma_commit(tfull);
            }
        }
        __syncwarp();
    } else if (warp >= 4) {
        const int qw = warp & 3;
        const int64_t row = i0 + qw * 32 + lane;
        const bool row_ok = row < n;
        const uint32_t tl = tmem + ((uint32_t)(qw * 32) << 16);
        for (int t = 0; t < np; ++t) {
            bool ok = gpch::tc::mbar_wait(tfull, t & 1, 4 * OZM_SPIN);
            ok = __all_sync(0xffffffffu, ok);
            gpch::tc::tc_fence_after();
            if (!ok) {
                if (lane == 0) atomicExch(oz.err, 3);
                break;
            }
            // class sums S_D = sum_{p + d = D} S_pd (exact in FP32: at most
            // 7 integers of magnitude 2^21), four pair blocks per TMEM wait
            float cs[OZM_CLASSES][OZM_N];
#pragma unroll
            for (int D = 0; D < OZM_CLASSES; ++D)
#pragma unroll
                for (int j = 0; j < OZM_N; ++j) cs[D][j] = 0.0f;
#pragma unroll
            for (int g = 0; g < 28; g += 4) {
                uint32_t v[4][16];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    // pair number g + u in the order p = 0 (d = 0..6), p = 1 (d = 0..5), ...
                    int p = 0, d = g + u;
#pragma unroll
                    for (int pp = 0; pp < OZM_CLASSES; ++pp)
                        if (d >= 7 - p) {
                            d -= 7 - p;
                            ++p;
                        }
                    gpch::tc::tmem_ld16_nowait(tl + (uint32_t)(ozm_base(p) + d * OZM_N), v[u]);
                }
                gpch::tc::tmem_ld_wait();
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    int p = 0, d = g + u;
#pragma unroll
                    for (int pp = 0; pp < OZM_CLASSES; ++pp)
                        if (d >= 7 - p) {
                            d -= 7 - p;
                            ++p;
                        }
#pragma unroll
                    for (int j = 0; j < OZM_N; ++j) cs[p + d][j] += __uint_as_float(v[u][j]);
                }
            }
            float c7[OZM_N];
            if constexpr (FULL) {
                uint32_t v7[16];
                gpch::tc::tmem_ld16_nowait(tl + OZM_C7, v7);
                gpch::tc::tmem_ld_wait();
#pragma unroll
                for (int j = 0; j < OZM_N; ++j) c7[j] = __uint_as_float(v7[j]);
            }
            // the accumulators are read: the MMAs of pass t + 1 may start
            gpch::tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) gpch::tc::mbar_arrive(tempty);
            const int er = row_ok ? oz.EA[(int64_t)t * oz.npad + row] : 0;
#pragma unroll
            for (int j = 0; j < OZM_N; ++j) {
                // T = sum_D S_D 128^(6 - D) = H 2^28 + L exactly; the
                // product is 2^(e_r + f_j - 52) T
                long long H = 0, L = 0;
#pragma unroll
                for (int D = 0; D < 3; ++D) H = H * 128 + __float2int_rn(cs[D][j]);
#pragma unroll
                for (int D = 3; D < 7; ++D) L = L * 128 + __float2int_rn(cs[D][j]);
                int sc = er + __ldg(&oz.ES[t * OZM_N + j]) - 52;
                if constexpr (FULL) {
                    // one more place: T 128 + S_7 = (128 H) 2^28 + (128 L + S_7)
                    H *= 128;
                    L = L * 128 + __float2int_rn(c7[j]);
                    sc -= 7;
                }
                acc64[j] += gpch::oz_round_scaled(H, L, sc);
            }
        }
    }
    // the products are in; the stages' memory holds them for the reductions
    gpch::tc::tc_fence_before();
    __syncthreads();
    double *tcol = reinterpret_cast<double *>(smem);
    if (warp >= 4) {
        const int r = (warp & 3) * 32 + lane;
#pragma unroll
        for (int j = 0; j < OZM_N; ++j) tcol[r * OZM_N + j] = acc64[j];
    }
    const int64_t wrows = (n - i0 < OZM_BM) ? n - i0 : OZM_BM;
    mv_finish<OZM_BM, OZM_N>(i0, (int)wrows, nrhs, S, lds, T, ldt, st, mode, sr, tcol);
    __syncthreads();
    if (warp == 1) {
        gpch::tc::tc_fence_after();
        gpch::tc::tmem_dealloc<OZM_TMEM>(tmem);
    }
}

// SS[i * NR + r] = (head, tail) of inv[r] * V[i, r]: float(v) and
// float(v - float(v)) (conversions on the FP64 pipe, once per entry).
template <int NR>
__global__ void __launch_bounds__(THREADS) df_split_vec_kernel(int64_t n, int nrhs, const double *__restrict__ V,
                                                               int64_t ldv, float2 *__restrict__ SS,
                                                               const double *__restrict__ inv, const int *done)
{
    if (done && *done) return;
    const int64_t e = (int64_t)blockIdx.x * THREADS + threadIdx.x;
    if (e >= n * NR) return;
    const int64_t i = e / NR;
    const int r = (int)(e % NR);
    float2 o = make_float2(0.0f, 0.0f);
    if (r < nrhs) {
        const double v = V[i + r * ldv] * inv[r];
        o.x = __double2float_rn(v);
        o.y = __double2float_rn(v - (double)o.x);
    }
    SS[e] = o;
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

// Single-reduction step on the vectors of active columns:
// p = r + beta p; s = w + beta s; x += alpha p; r -= alpha s (not on a
// replacement iteration, whose r is recomputed from x).
__global__ void __launch_bounds__(THREADS) cgsr_vec_kernel(int64_t n, int nrhs, double *X, int64_t ldx, double *R,
                                                           const double *Wv, double *P, double *S, int64_t ldv,
                                                           CGState st, int replace)
{
    if (*st.done) return;
    const int64_t i = (int64_t)blockIdx.x * THREADS + threadIdx.x;
    if (i >= n) return;
    for (int r = 0; r < nrhs; ++r) {
        if (!st.active[r]) continue;
        const double a = st.alpha[r], b = st.beta[r];
        const double p = fma(b, P[i + r * ldv], R[i + r * ldv]);
        const double s = fma(b, S[i + r * ldv], Wv[i + r * ldv]);
        P[i + r * ldv] = p;
        S[i + r * ldv] = s;
        X[i + r * ldx] = fma(a, p, X[i + r * ldx]);
        if (!replace) R[i + r * ldv] = fma(-a, s, R[i + r * ldv]);
    }
}

// r = b - t on active columns (all columns with `all`).
__global__ void __launch_bounds__(THREADS) cg_resid_kernel(int64_t n, int nrhs, double *R, const double *T,
                                                           const double *B, int64_t ldb, int64_t ldv, CGState st,
                                                           int all)
{
    if (!all && *st.done) return;
    const int64_t i = (int64_t)blockIdx.x * THREADS + threadIdx.x;
    if (i >= n) return;
    for (int r = 0; r < nrhs; ++r)
        if (all || st.active[r]) R[i + r * ldv] = B[i + r * ldb] - T[i + r * ldv];
}

// Double-float set-up: ea from max_i A_ii (FP64 A; 0 for FP32 A), es_r from
// max_i |B_ir|; writes scale, inv and ebias.  dmax: [0] max diagonal,
// [1 + r] max |b_r| (bit patterns of non-negative doubles).
__global__ void df_scales_kernel(int nrhs, const double *dmax, int split_a, double *scale, double *inv, int *ebias)
{
    const int r = threadIdx.x;
    int ea = 0;
    if (split_a && dmax[0] > 0.0) ea = ilogb(dmax[0]);
    ea = ea < -800 ? -800 : (ea > 800 ? 800 : ea);
    if (r == 0) *ebias = 896 + ea;
    if (r < MAXRHS) {
        const double bm = r < nrhs ? dmax[1 + r] : 0.0;
        int es = bm > 0.0 ? ilogb(bm) : 0;
        es = es < -900 ? -900 : (es > 900 ? 900 : es);
        scale[r] = ldexp(1.0, ea + es);
        inv[r] = ldexp(1.0, -es);
    }
}

// Order-independent maxima of non-negative doubles through their bit
// patterns (which order like the values).
__device__ inline void atomic_max_nonneg(double *addr, double v)
{
    atomicMax(reinterpret_cast<unsigned long long *>(addr), (unsigned long long)__double_as_longlong(v));
}

// *out = max(0, max_i A_ii).
template <typename TA>
__global__ void __launch_bounds__(THREADS) diag_max_kernel(int64_t n, const TA *__restrict__ A, int64_t lda,
                                                           double *out)
{
    double m = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * THREADS)
        m = fmax(m, (double)A[i + i * lda]);
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

// Column width per CTA and right-hand-side bucket of a matvec launch.
// Narrow column blocks make many CTAs, so the last partial wave is a small
// share of the launch; the double-float path reads the split vector once
// per CTA, so it takes wider blocks.
inline int mv_nr(int nrhs) { return nrhs <= 1 ? 1 : nrhs <= 2 ? 2 : nrhs <= 4 ? 4 : nrhs <= 8 ? 8 : 16; }
inline int mv_width(int nrhs, int prod)
{
    if (prod == PROD_OZ) return OZM_BM;
    if (prod == PROD_DF) return nrhs <= 2 ? 8 : TW;
    return nrhs <= 1 ? 4 : nrhs <= 2 ? 8 : nrhs <= 4 ? 4 : 2;
}

template <typename TA, bool DF>
void launch_mv_kernel(int64_t n, int64_t ncols, int nrhs, const TA *A, int64_t lda, const double *S, int64_t lds,
                      double *T, int64_t ldt, const CGState &st, int mode, SRArgs sr, DFArgs df, int vec,
                      cudaStream_t s)
{
#define GPCH_MV(Wc, NRc)                                                                                        \
    cg_matvec_kernel<TA, Wc, NRc, DF><<<(unsigned)((ncols + Wc - 1) / Wc), THREADS, 0, s>>>(                  \
        n, ncols, nrhs, A, lda, S, lds, T, ldt, st, mode, sr, df, vec)
#define GPCH_MVT(NRc)                                                                                           \
    cg_matvec_df_tiled_kernel<TA, NRc><<<(unsigned)((ncols + TW - 1) / TW), THREADS, 0, s>>>(                 \
        n, ncols, nrhs, A, lda, S, lds, T, ldt, st, mode, sr, df, vec)
    if constexpr (DF) {
        if (nrhs <= 1) GPCH_MV(8, 1);
        else if (nrhs <= 2) GPCH_MV(8, 2);
        else if (nrhs <= 4) GPCH_MVT(4);
        else if (nrhs <= 8) GPCH_MVT(8);
        else GPCH_MVT(16);
    } else {
        if (nrhs <= 1) GPCH_MV(4, 1);
        else if (nrhs <= 2) GPCH_MV(8, 2);
        else if (nrhs <= 4) GPCH_MV(4, 4);
        else if (nrhs <= 8) GPCH_MV(2, 8);
        else GPCH_MV(2, 16);
    }
#undef GPCH_MV
#undef GPCH_MVT
}

// ------------------------------- symmetric matvec from the lower triangle
//
// T = A S for a symmetric A of which only the lower triangle (i >= j)
// affects the result, with double-float products as cg_matvec_kernel's DF
// path: every stored entry serves twice, A_ij s_i in t_j (down column j)
// and, for i > j, A_ij s_j in t_i, so the product reads about half of A's
// bytes.  The work is cut into units of one strip of SY_SW columns (J) by
// one chunk of SY_R rows (c), from the strip's diagonal block down: rows
// r0 = J SY_SW + c SY_R ..  In a unit, warp w takes the strip's columns
// 32 w .. 32 w + 31, SY_CG at a time, and walks the chunk in 64-row
// segments; each segment's SY_CG x 64 block is copied into the warp's
// shared memory by cp.async (lane l: rows 2l, 2l + 1 of each column, 16
// bytes), SY_ST segments in flight, so the loads of later segments overlap
// the arithmetic on the current one.  Lane l works on rows 2l, 2l + 1.  The
// column sums of a group stay in registers over the chunk and are reduced
// over the warp at its end; the row sums of a segment are added into the
// warp's slice of shared memory and summed over the warps in warp order
// once per unit.  The partials go out as double-float pairs of the scaled
// products to dotp (column j, chunk c: dotp[(c n + j) NR + r]) and axp (row
// i, strip J: axp[(J n + i) NR + r]); sym_mv_finish_kernel adds them in a
// fixed order and scales back.  Nothing in the loop is FP64 arithmetic:
// this part's FP64 pipe is slow enough that a few widenings per column
// group held the loop back.
//
// The source of the entries (SRC):
//   SY_FP64   A itself; each entry is cut into its float head and tail
//             (df_split_a, integer operations);
//   SY_WRITE  as SY_FP64, and the heads and tails are also stored in the
//             packed copy AP, so that later products with the same A
//             skip the cutting;
//   SY_PACKED the packed copy: strip J holds columns J SY_SW .. + SY_SW - 1,
//             rows J SY_SW .. n2 - 1 (n2 = n rounded up to even), column
//             major with ld n2 - J SY_SW, from float2 offset
//             sy_off(n, J); entries above the diagonal and rows at or past
//             n are zero.
// In the diagonal chunk the entries above the diagonal are replaced by
// zeros before they are used (from A they may be read, never used).
constexpr int SY_SW = THREADS;   // columns per strip: one finishing CTA per strip
constexpr int SY_R = 256;        // rows per chunk
constexpr int SY_CG = 8;         // columns a warp takes at a time
constexpr int SY_ST = 3;         // segments in flight per warp
enum SySrc : int { SY_FP64 = 0, SY_WRITE = 1, SY_PACKED = 2 };
template <bool B> struct SyTag { static constexpr bool value = B; };
static_assert(SY_R % 64 == 0 && SY_R >= SY_SW && SY_SW == (THREADS / 32) * 32, "unit shape");

inline int64_t sy_chunks(int64_t n) { return (n + SY_R - 1) / SY_R; }
inline int64_t sy_strips(int64_t n) { return (n + SY_SW - 1) / SY_SW; }
inline size_t sy_smem(int nr)
{
    return (size_t)(THREADS / 32) * (SY_ST * SY_CG * 64 * sizeof(double) + SY_R * nr * sizeof(float2));
}
// doubles (8-byte slots: double-float pairs) of the two partial arrays
inline size_t sy_part_doubles(int64_t n, int nr) { return (size_t)(sy_chunks(n) + sy_strips(n)) * n * nr; }
static_assert(SY_SW == gpch::SYM_STRIP, "the packed copy's strips are the units' strips");
using gpch::sy_off;

__device__ __forceinline__ void cp_async16_zfill(void *dst, const void *src, bool ok)
{
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(ok ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async8_zfill(void *dst, const void *src, bool ok)
{
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(ok ? 8 : 0) : "memory");
}

template <int NR, int SRC>
__global__ void __launch_bounds__(THREADS, 2) sym_mv_df_kernel(int64_t n, const double *__restrict__ A, int64_t lda,
                                                               float2 *AP, DFArgs df, float2 *__restrict__ dotp,
                                                               float2 *__restrict__ axp, const int *done, int vec)
{
    extern __shared__ __align__(16) double sy_smem_raw[];
    if (done && *done) return;
    const int64_t J = blockIdx.y, c = blockIdx.x;
    const int64_t cs = J * SY_SW;   // the strip's first column
    const int64_t r0 = cs + c * SY_R;
    if (r0 >= n) return;
    const int rows = (int)((n - r0 < SY_R) ? n - r0 : SY_R);
    const int nseg = (rows + 63) / 64;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool dg = c == 0;   // the chunk holds the strip's diagonal block
    const int64_t n2 = (n + 1) & ~int64_t(1), ldp = n2 - cs;   // the packed strip's column length
    float2 *APs = (SRC != SY_FP64) ? AP + sy_off(n, J) : nullptr;
    const unsigned ebias = (SRC != SY_PACKED) ? (unsigned)*df.ebias : 0u;
    // the warp's segment buffers [stage][column][64 rows] (16 bytes per
    // lane and column: two doubles, or two head-tail pairs), then every
    // warp's row sums
    double *buf = sy_smem_raw + (size_t)warp * SY_ST * SY_CG * 64;
    float2 *axs = reinterpret_cast<float2 *>(sy_smem_raw + (size_t)(THREADS / 32) * SY_ST * SY_CG * 64);
    float2 *ax = axs + (size_t)warp * SY_R * NR;
    for (int e = lane; e < SY_R * NR; e += 32) ax[e] = make_float2(0.0f, 0.0f);
    // Everything below indexes from the chunk's first row r0 with 32-bit
    // offsets: 64-bit integer arithmetic shares the FP64 pipe on this part.
    const int rows2 = (int)((n2 - r0 < SY_R) ? n2 - r0 : SY_R);   // rows of the packed strip in the chunk
    const float2 *SSr = df.SS + r0 * NR;
    for (int g = 0; g < 32 / SY_CG; ++g) {
        const int64_t j0 = cs + warp * 32 + g * SY_CG;   // the group's first column
        if (j0 >= n) break;
        const int ncg = (int)((n - j0 < SY_CG) ? n - j0 : SY_CG);   // columns of the group inside A
        const int dlt = (int)(r0 - j0);   // row r0 + rl lies (rl + dlt - q) below column j0 + q's diagonal
        float ch[SY_CG][NR], cl[SY_CG][NR], dh[SY_CG][NR], dl[SY_CG][NR];
#pragma unroll
        for (int q = 0; q < SY_CG; ++q)
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const float2 v = (q < ncg) ? df.SS[(j0 + q) * NR + r] : make_float2(0.0f, 0.0f);
                ch[q][r] = v.x;
                cl[q][r] = v.y;
                dh[q][r] = dl[q][r] = 0.0f;
            }
        // the group's columns from row r0: in A, or in the packed strip
        const double *acol[SY_CG];
        float2 *pcol[SY_CG];
#pragma unroll
        for (int q = 0; q < SY_CG; ++q) {
            const int64_t jq = (q < ncg) ? j0 + q : j0;
            acol[q] = A + jq * lda + r0;
            pcol[q] = (SRC != SY_FP64) ? APs + (jq - cs) * ldp + (r0 - cs) : nullptr;
        }
        // in the diagonal chunk, segments wholly above the group's first column are skipped
        const int s0 = dg ? (-dlt) / 64 : 0;
        // segment sg into stage sg % SY_ST: this lane's rows of the SY_CG columns
        auto stage = [&](int sg) {
            double *b = buf + (sg % SY_ST) * SY_CG * 64;
            const int rl = sg * 64 + 2 * lane;
#pragma unroll
            for (int q = 0; q < SY_CG; ++q) {
                const bool colok = q < ncg;
                if constexpr (SRC == SY_PACKED) {
                    const bool ok = rl < rows2 && colok;
                    cp_async16_zfill(b + q * 64 + 2 * lane, ok ? (const void *)(pcol[q] + rl) : A, ok);
                } else if (vec) {
                    cp_async16_zfill(b + q * 64 + 2 * lane, (rl + 1 < rows) ? acol[q] + rl : A, rl + 1 < rows);
                } else {
                    cp_async8_zfill(b + q * 64 + 2 * lane, (rl < rows) ? acol[q] + rl : A, rl < rows);
                    cp_async8_zfill(b + q * 64 + 2 * lane + 1, (rl + 1 < rows) ? acol[q] + rl + 1 : A, rl + 1 < rows);
                }
            }
        };
        __syncwarp();   // the previous group's reads of the stages are done
        for (int k = 0; k < SY_ST - 1; ++k) {
            if (s0 + k < nseg) stage(s0 + k);
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        for (int sg = s0; sg < nseg; ++sg) {
            if (sg + SY_ST - 1 < nseg) stage(sg + SY_ST - 1);
            asm volatile("cp.async.commit_group;" ::: "memory");
            asm volatile("cp.async.wait_group %0;" ::"n"(SY_ST - 1) : "memory");
            double *b = buf + (sg % SY_ST) * SY_CG * 64;
            const int rl = sg * 64 + 2 * lane;   // the lane's first row, chunk-local
            if (SRC != SY_PACKED && vec && rl + 1 == rows && r0 + rows == n) {
                // n odd: the last row alone (the 16-byte copy was skipped)
#pragma unroll
                for (int q = 0; q < SY_CG; ++q) b[q * 64 + 2 * lane] = acol[q][rl];
            }
            float rh[2][NR], rt[2][NR], uh[2][NR], ul[2][NR];
#pragma unroll
            for (int p = 0; p < 2; ++p)
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const float2 v = (rl + p < rows) ? SSr[(rl + p) * NR + r] : make_float2(0.0f, 0.0f);
                    rh[p][r] = v.x;
                    rt[p][r] = v.y;
                    uh[p][r] = ul[p][r] = 0.0f;
                }
            // masks only where the segment meets the diagonal or the edges
            auto products = [&](auto tag) {
                constexpr bool MASKED = decltype(tag)::value;
#pragma unroll
                for (int q = 0; q < SY_CG; ++q) {
                    float hv[2], tv[2];
                    if constexpr (SRC == SY_PACKED) {
                        const float4 v = *reinterpret_cast<const float4 *>(b + q * 64 + 2 * lane);
                        hv[0] = v.x;
                        tv[0] = v.y;
                        hv[1] = v.z;
                        tv[1] = v.w;
                    } else {
                        const double2 av = *reinterpret_cast<const double2 *>(b + q * 64 + 2 * lane);
                        df_split_a(av.x, ebias, hv[0], tv[0]);
                        df_split_a(av.y, ebias, hv[1], tv[1]);
                    }
                    float hd[2], td[2], hx[2], tx[2];
#pragma unroll
                    for (int p = 0; p < 2; ++p) {
                        hd[p] = hx[p] = hv[p];
                        td[p] = tx[p] = tv[p];
                        if constexpr (MASKED) {
                            // row - column = rl + p + dlt - q
                            const int below = rl + p + dlt - q;
                            const bool in = rl + p < rows && q < ncg;
                            const bool okd = in && (!dg || below >= 0), okx = in && (!dg || below > 0);
                            hx[p] = okx ? hv[p] : 0.0f;
                            tx[p] = okx ? tv[p] : 0.0f;
                            hd[p] = okd ? hv[p] : 0.0f;
                            td[p] = okd ? tv[p] : 0.0f;
                        }
                    }
                    if constexpr (SRC == SY_WRITE) {
                        // the masked heads and tails: zero above the diagonal and past n
                        if (rl < rows2 && q < ncg)
                            *reinterpret_cast<float4 *>(pcol[q] + rl) = make_float4(hd[0], td[0], hd[1], td[1]);
                    }
#pragma unroll
                    for (int p = 0; p < 2; ++p)
#pragma unroll
                        for (int r = 0; r < NR; ++r) {
                            // t_j += A_ij s_i
                            const float pd = hd[p] * rh[p][r];
                            float ed = fmaf(hd[p], rh[p][r], -pd);
                            ed = fmaf(hd[p], rt[p][r], ed);
                            ed = fmaf(td[p], rh[p][r], ed);
                            df_add(dh[q][r], dl[q][r], pd, ed);
                            // t_i += A_ij s_j
                            const float px = hx[p] * ch[q][r];
                            float ex = fmaf(hx[p], ch[q][r], -px);
                            ex = fmaf(hx[p], cl[q][r], ex);
                            ex = fmaf(tx[p], ch[q][r], ex);
                            df_add(uh[p][r], ul[p][r], px, ex);
                        }
                }
            };
            const bool clean = !(dg && sg * 64 + dlt < SY_CG) && sg * 64 + 64 <= rows && ncg == SY_CG;
            if (clean) products(SyTag<false>{});
            else products(SyTag<true>{});
#pragma unroll
            for (int p = 0; p < 2; ++p)
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    float2 v = ax[(rl + p) * NR + r];
                    df_add2(v.x, v.y, uh[p][r], ul[p][r]);
                    ax[(rl + p) * NR + r] = v;
                }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        // the group's column sums over the warp
#pragma unroll
        for (int q = 0; q < SY_CG; ++q)
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                float h = dh[q][r], l = dl[q][r];
#pragma unroll
                for (int off = 16; off > 0; off >>= 1)
                    df_add2(h, l, __shfl_xor_sync(0xffffffffu, h, off), __shfl_xor_sync(0xffffffffu, l, off));
                if (lane == 0 && q < ncg) dotp[(c * n + j0 + q) * NR + r] = make_float2(h, l);
            }
    }
    __syncthreads();
    // the row sums over the warps, in warp order
    for (int e = tid; e < rows * NR; e += THREADS) {
        float h = axs[e].x, l = axs[e].y;
        for (int w = 1; w < THREADS / 32; ++w)
            df_add2(h, l, axs[(size_t)w * SY_R * NR + e].x, axs[(size_t)w * SY_R * NR + e].y);
        axp[(J * n + r0) * NR + e] = make_float2(h, l);
    }
}

// t_i for the rows of strip blockIdx.x: the chunks' column sums of column
// i and the strips' row sums of row i, in four interleaved double-float
// sums (index mod 4) combined in a fixed order, widened and scaled once;
// then the mode's reductions as the other matvecs (mv_finish).
template <int NR>
__global__ void __launch_bounds__(THREADS) sym_mv_finish_kernel(int64_t n, int nrhs, const float2 *__restrict__ dotp,
                                                                const float2 *__restrict__ axp, const double *scale,
                                                                const double *__restrict__ S, int64_t lds, double *T,
                                                                int64_t ldt, CGState st, int mode, SRArgs sr)
{
    __shared__ double tcol[SY_SW * NR];
    if (*st.done) return;
    const int64_t J = blockIdx.x, i0 = J * SY_SW;
    const int wcols = (int)((n - i0 < SY_SW) ? n - i0 : SY_SW);
    const int tid = threadIdx.x;
    if (tid < wcols) {
        const int nch = (int)((n - i0 + SY_R - 1) / SY_R), nst = (int)J + 1;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const float2 *dp = dotp + (i0 + tid) * NR + r, *xp = axp + (i0 + tid) * NR + r;
            const int64_t step = n * NR;
            float h[4] = {0.0f, 0.0f, 0.0f, 0.0f}, l[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            int c = 0;
            for (; c + 4 <= nch; c += 4)
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float2 v = dp[(int64_t)(c + u) * step];
                    df_add2(h[u], l[u], v.x, v.y);
                }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (c + u < nch) {
                    const float2 v = dp[(int64_t)(c + u) * step];
                    df_add2(h[u], l[u], v.x, v.y);
                }
            int K = 0;
            for (; K + 4 <= nst; K += 4)
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float2 v = xp[(int64_t)(K + u) * step];
                    df_add2(h[u], l[u], v.x, v.y);
                }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (K + u < nst) {
                    const float2 v = xp[(int64_t)(K + u) * step];
                    df_add2(h[u], l[u], v.x, v.y);
                }
            df_add2(h[0], l[0], h[1], l[1]);
            df_add2(h[2], l[2], h[3], l[3]);
            df_add2(h[0], l[0], h[2], l[2]);
            tcol[tid * NR + r] = ((double)h[0] + (double)l[0]) * scale[r];
        }
    }
    mv_finish<SY_SW, NR>(i0, wcols, nrhs, S, lds, T, ldt, st, mode, sr, tcol);
}

// One matvec T = A S (plus the mode's reductions).  With PROD_DF the vector
// S is split into df.SS first (one small launch).
template <typename TA>
gpch_status launch_matvec(gpch_ctx *ctx, int64_t n, int nrhs, const TA *A, int64_t lda, const double *S,
                          int64_t lds, double *T, int64_t ldt, const CGState &st, int mode, cudaStream_t s,
                          int prod = PROD_FP64, DFArgs df = DFArgs{}, SRArgs sr = SRArgs{0.0, 0, 0},
                          int64_t ncols = -1)
{
    if (ncols < 0) ncols = n;
    const int vec = ((reinterpret_cast<uintptr_t>(A) & 15) == 0 && ((lda * (int64_t)sizeof(TA)) & 15) == 0) ? 1 : 0;
    if (prod == PROD_OZ || prod == PROD_OZ_FULL) {
        // the vectors' digits, then the tensor-core product (A's digits
        // were made once per solve by oz_prepare)
        const OzArgs &oz = df.oz;
        const int *done = (mode == MV_SR && sr.first) ? nullptr : st.done;
        oz_split_cols_kernel<double><<<(unsigned)((OZM_N * oz.np + 7) / 8), 256, 0, s>>>(
            n, oz.np, oz.kpt, S, lds, nrhs, OZM_N, oz.DS, oz.ES, done, 0);
        GPCH_LAUNCH_CHECK(ctx);
        CUtensorMap ma, ms;
        GPCH_CHECK(gpch::oz_map(ctx, &ma, oz.DA, oz.npad * (oz.kpt / OZM_KSTAGE) * 4, 64, OZM_BM));
        GPCH_CHECK(gpch::oz_map(ctx, &ms, oz.DS, (oz.kpt / OZM_KSTAGE) * 8 * OZM_N, 32, 8 * OZM_N, true));
        static gpch::DeviceOnce attr_once;
        GPCH_CHECK(gpch::once_per_device(ctx, attr_once, [&]() -> gpch_status {
            GPCH_CUDA(ctx, cudaFuncSetAttribute(oz_matvec_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)OZM_SMEM));
            GPCH_CUDA(ctx, cudaFuncSetAttribute(oz_matvec_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)OZM_SMEM));
            return GPCH_OK;
        }));
        gpch::PhaseScope ph(ctx, GPCH_PHASE_CG_MATVEC, s,
                            (double)n * oz.kpt * 16.0 + (double)(n + ncols) * nrhs * sizeof(double));
        const unsigned grid = (unsigned)((n + OZM_BM - 1) / OZM_BM);
        if (prod == PROD_OZ_FULL)
            oz_matvec_kernel<true><<<grid, THREADS, OZM_SMEM, s>>>(ma, ms, n, nrhs, S, lds, T, ldt, st, mode, sr, oz);
        else
            oz_matvec_kernel<false><<<grid, THREADS, OZM_SMEM, s>>>(ma, ms, n, nrhs, S, lds, T, ldt, st, mode, sr, oz);
        GPCH_LAUNCH_CHECK(ctx);
        return GPCH_OK;
    }
    if (prod == PROD_DF) {
        const int nr = mv_nr(nrhs);
        const unsigned blocks = (unsigned)((n * nr + THREADS - 1) / THREADS);
        // the set-up product of the single-reduction form runs before `done` is meaningful
        const int *done = (mode == MV_SR && sr.first) ? nullptr : st.done;
        switch (nr) {
        case 1: df_split_vec_kernel<1><<<blocks, THREADS, 0, s>>>(n, nrhs, S, lds, df.SS, df.inv, done); break;
        case 2: df_split_vec_kernel<2><<<blocks, THREADS, 0, s>>>(n, nrhs, S, lds, df.SS, df.inv, done); break;
        case 4: df_split_vec_kernel<4><<<blocks, THREADS, 0, s>>>(n, nrhs, S, lds, df.SS, df.inv, done); break;
        case 8: df_split_vec_kernel<8><<<blocks, THREADS, 0, s>>>(n, nrhs, S, lds, df.SS, df.inv, done); break;
        default: df_split_vec_kernel<16><<<blocks, THREADS, 0, s>>>(n, nrhs, S, lds, df.SS, df.inv, done); break;
        }
        GPCH_LAUNCH_CHECK(ctx);
    }
    gpch::PhaseScope ph(ctx, GPCH_PHASE_CG_MATVEC, s,
                        (double)n * ncols * sizeof(TA) + (double)(n + ncols) * nrhs * sizeof(double));
    if (prod == PROD_DF)
        launch_mv_kernel<TA, true>(n, ncols, nrhs, A, lda, S, lds, T, ldt, st, mode, sr, df, vec, s);
    else
        launch_mv_kernel<TA, false>(n, ncols, nrhs, A, lda, S, lds, T, ldt, st, mode, sr, df, vec, s);
    GPCH_LAUNCH_CHECK(ctx);
    return GPCH_OK;
}

// T = A S (nrhs <= 2) from A's lower triangle with double-float products
// (sym_mv_df_kernel), plus the mode's reductions; S is split into df.SS
// first.  src: SY_FP64 (AP unused), SY_WRITE (also fills the packed copy
// AP, sy_off(n, sy_strips(n)) float2) or SY_PACKED (reads AP, made by an
// SY_WRITE product of the same A with the same df scales).  part:
// sy_part_doubles(n, mv_nr(nrhs)) doubles of scratch.
gpch_status launch_symv_df(gpch_ctx *ctx, int64_t n, int nrhs, const double *A, int64_t lda, const double *S,
                           int64_t lds, double *T, int64_t ldt, const CGState &st, int mode, cudaStream_t s,
                           const DFArgs &df, double *part, float2 *AP = nullptr, int src = SY_FP64)
{
    if (nrhs < 1 || nrhs > 2) return gpch::fail(ctx, GPCH_INVALID_ARG, "symmetric matvec takes 1 or 2 columns");
    if (src != SY_FP64 && AP == nullptr) return gpch::fail(ctx, GPCH_INVALID_ARG, "packed copy missing");
    const int nr = mv_nr(nrhs);
    const unsigned blocks = (unsigned)((n * nr + THREADS - 1) / THREADS);
    if (nr == 1) df_split_vec_kernel<1><<<blocks, THREADS, 0, s>>>(n, nrhs, S, lds, df.SS, df.inv, st.done);
    else df_split_vec_kernel<2><<<blocks, THREADS, 0, s>>>(n, nrhs, S, lds, df.SS, df.inv, st.done);
    GPCH_LAUNCH_CHECK(ctx);
#define GPCH_SY_ATTR(NRc, SRCc)                                                                                 \
    GPCH_CUDA(ctx, cudaFuncSetAttribute(sym_mv_df_kernel<NRc, SRCc>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                        (int)sy_smem(NRc)))
    static gpch::DeviceOnce attr_once;
    GPCH_CHECK(gpch::once_per_device(ctx, attr_once, [&]() -> gpch_status {
        GPCH_SY_ATTR(1, SY_FP64);
        GPCH_SY_ATTR(1, SY_WRITE);
        GPCH_SY_ATTR(1, SY_PACKED);
        GPCH_SY_ATTR(2, SY_FP64);
        GPCH_SY_ATTR(2, SY_WRITE);
        GPCH_SY_ATTR(2, SY_PACKED);
        return GPCH_OK;
    }));
#undef GPCH_SY_ATTR
    const int vec = ((reinterpret_cast<uintptr_t>(A) & 15) == 0 && (lda & 1) == 0) ? 1 : 0;
    float2 *dotp = reinterpret_cast<float2 *>(part), *axp = dotp + (size_t)sy_chunks(n) * n * nr;
    const dim3 grid((unsigned)sy_chunks(n), (unsigned)sy_strips(n));
    const double abytes = (src == SY_WRITE ? 2.0 : 1.0) * (double)n * (double)(n + 1) / 2.0 * sizeof(double);
    gpch::PhaseScope ph(ctx, GPCH_PHASE_CG_MATVEC, s, abytes + 2.0 * n * nrhs * sizeof(double));
#define GPCH_SY(NRc, SRCc)                                                                                      \
    sym_mv_df_kernel<NRc, SRCc><<<grid, THREADS, sy_smem(NRc), s>>>(n, A, lda, AP, df, dotp, axp, st.done, vec)
    if (nr == 1) {
        if (src == SY_WRITE) GPCH_SY(1, SY_WRITE);
        else if (src == SY_PACKED) GPCH_SY(1, SY_PACKED);
        else GPCH_SY(1, SY_FP64);
        GPCH_LAUNCH_CHECK(ctx);
        sym_mv_finish_kernel<1><<<(unsigned)sy_strips(n), THREADS, 0, s>>>(n, nrhs, dotp, axp, df.scale, S, lds, T,
                                                                          ldt, st, mode, SRArgs{0.0, 0, 0});
    } else {
        if (src == SY_WRITE) GPCH_SY(2, SY_WRITE);
        else if (src == SY_PACKED) GPCH_SY(2, SY_PACKED);
        else GPCH_SY(2, SY_FP64);
        GPCH_LAUNCH_CHECK(ctx);
        sym_mv_finish_kernel<2><<<(unsigned)sy_strips(n), THREADS, 0, s>>>(n, nrhs, dotp, axp, df.scale, S, lds, T,
                                                                          ldt, st, mode, SRArgs{0.0, 0, 0});
    }
#undef GPCH_SY
    GPCH_LAUNCH_CHECK(ctx);
    return GPCH_OK;
}

// Loads every kernel cg_run may launch on the current device for the
// classic FP64-product solve.  Under lazy module loading a kernel's code is
// placed in device memory at its first launch; asking for its attributes
// loads it ahead of time.
template <typename TA>
cudaError_t cg_kernels_load()
{
    cudaFuncAttributes a;
    const void *fns[] = {(const void *)cg_matvec_kernel<TA, 4, 1, false>,
                         (const void *)cg_matvec_kernel<TA, 8, 2, false>,
                         (const void *)cg_matvec_kernel<TA, 4, 4, false>,
                         (const void *)cg_matvec_kernel<TA, 2, 8, false>,
                         (const void *)cg_matvec_kernel<TA, 2, 16, false>,
                         (const void *)cg_init_kernel,
                         (const void *)cg_update_kernel,
                         (const void *)cg_xupdate_kernel,
                         (const void *)cg_dir_kernel};
    for (const void *f : fns) {
        cudaError_t e = cudaFuncGetAttributes(&a, f);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Doubles of per-CTA partials: a matvec stores mv_nr (two sets in the
// single-reduction form) per CTA, the vector kernels (one CTA per THREADS
// rows) up to 3 * MAXRHS.
inline size_t part_doubles(int64_t n, int nrhs, int prod = PROD_FP64, int variant = VAR_CLASSIC)
{
    const int sets = variant == VAR_SINGLE_REDUCTION ? 2 : 1;
    const int nr = prod == PROD_OZ ? OZM_N : mv_nr(nrhs);
    const size_t mv = (size_t)((n + mv_width(nrhs, prod) - 1) / mv_width(nrhs, prod)) * nr * sets;
    const size_t vec = (size_t)((n + THREADS - 1) / THREADS) * 3 * MAXRHS;
    return mv > vec ? mv : vec;
}

struct CGBufs {
    double *R, *S, *T, *P, *Wv;   // P, Wv: single-reduction form only
    CGState st;
    double *sc;
    int *ic;
    DFArgs df;
    double *dmax;                 // [1 + MAXRHS]: max diagonal, max |b_r|
};

// Carves the scratch of one CG group; with a null base only sizes it.
inline size_t cg_carve(void *base, int64_t n, int nrhs, int prod, int variant, CGBufs *b)
{
    gpch::Carver cv(base);
    CGBufs t;
    t.R = cv.take<double>((size_t)n * nrhs);
    t.S = cv.take<double>((size_t)n * nrhs);
    t.T = cv.take<double>((size_t)n * nrhs);
    t.P = t.Wv = nullptr;
    if (variant == VAR_SINGLE_REDUCTION) {
        t.P = cv.take<double>((size_t)n * nrhs);
        t.Wv = cv.take<double>((size_t)n * nrhs);
    }
    t.sc = cv.take<double>(4 * MAXRHS);
    t.st.u = t.sc;
    t.st.u0 = t.sc + MAXRHS;
    t.st.alpha = t.sc + 2 * MAXRHS;
    t.st.beta = t.sc + 3 * MAXRHS;
    t.ic = cv.take<int>(2 * MAXRHS + 1);
    t.st.active = t.ic;
    t.st.iters = t.ic + MAXRHS;
    t.st.done = t.ic + 2 * MAXRHS;
    t.st.counter = cv.take<unsigned>(2);
    t.st.part = cv.take<double>(part_doubles(n, nrhs, prod, variant));
    t.df = DFArgs{nullptr, nullptr, nullptr, nullptr, OzArgs{nullptr, nullptr, nullptr, nullptr, nullptr, 0, 0, 0}};
    t.dmax = nullptr;
    if (prod == PROD_OZ) {
        OzArgs &oz = t.df.oz;
        oz.np = (int)((n + 511) / 512);
        oz.kpt = (int64_t)oz.np * 512;
        oz.npad = (n + OZM_BM - 1) / OZM_BM * OZM_BM;
        oz.err = cv.take<int>(1);
        oz.DA = cv.take<__nv_bfloat16>((size_t)4 * oz.npad * 2 * oz.kpt);
        oz.EA = cv.take<int>((size_t)oz.np * oz.npad);
        oz.DS = cv.take<__nv_bfloat16>((size_t)4 * OZM_N * 2 * oz.kpt);
        oz.ES = cv.take<int>((size_t)oz.np * OZM_N);
    }
    if (prod == PROD_DF) {
        t.df.SS = cv.take<float2>((size_t)n * mv_nr(nrhs));
        double *d = cv.take<double>(2 * MAXRHS);
        t.df.scale = d;
        t.df.inv = d + MAXRHS;
        t.df.ebias = cv.take<int>(1);
        t.dmax = cv.take<double>(1 + MAXRHS);
    }
    if (b) *b = t;
    return cv.off;
}

// Bytes of scratch one CG group of nrhs (<= 16) columns needs.
size_t cg_scratch_bytes(int64_t n, int nrhs, int prod = PROD_FP64, int variant = VAR_CLASSIC)
{
    return cg_carve(nullptr, n, nrhs, prod, variant, nullptr);
}

// Enqueues the double-float scales of one solve (ea from A's diagonal, es_r
// from B's columns).
template <typename TA>
gpch_status df_prepare(gpch_ctx *ctx, int64_t n, int nrhs, const TA *A, int64_t lda, const double *B, int64_t ldb,
                       const CGBufs &b, cudaStream_t s)
{
    GPCH_CUDA(ctx, cudaMemsetAsync(b.dmax, 0, (1 + MAXRHS) * sizeof(double), s));
    const unsigned vec_ctas = (unsigned)((n + THREADS - 1) / THREADS);
    if (sizeof(TA) == 8) {
        diag_max_kernel<TA><<<vec_ctas < 148 ? vec_ctas : 148, THREADS, 0, s>>>(n, A, lda, b.dmax);
        GPCH_LAUNCH_CHECK(ctx);
    }
    absmax_cols_kernel<<<vec_ctas, THREADS, 0, s>>>(n, nrhs, B, ldb, b.dmax + 1);
    GPCH_LAUNCH_CHECK(ctx);
    df_scales_kernel<<<1, 32, 0, s>>>(nrhs, b.dmax, sizeof(TA) == 8 ? 1 : 0, const_cast<double *>(b.df.scale),
                                      const_cast<double *>(b.df.inv), const_cast<int *>(b.df.ebias));
    GPCH_LAUNCH_CHECK(ctx);
    return GPCH_OK;
}

// Enqueues the digit copy of A^T for the tensor-core products of one solve
// (A symmetric: A^T's rows are A's columns, read contiguously).
template <typename TA>
gpch_status oz_prepare(gpch_ctx *ctx, int64_t n, const TA *A, int64_t lda, const CGBufs &b, cudaStream_t s)
{
    const OzArgs &oz = b.df.oz;
    GPCH_CUDA(ctx, cudaMemsetAsync(oz.err, 0, sizeof(int), s));
    oz_split_cols_kernel<TA><<<(unsigned)((oz.npad * oz.np + 7) / 8), 256, 0, s>>>(
        n, oz.np, oz.kpt, A, lda, n, oz.npad, oz.DA, oz.EA, nullptr, 1);
    GPCH_LAUNCH_CHECK(ctx);
    return GPCH_OK;
}

// One CG group on caller-provided scratch (cg_scratch_bytes(n, nrhs, prod,
// variant) bytes of device memory at `scratch`) and a host staging block
// `hbuf` of at least 64 + 4*16*8 + 34*4 bytes (pinned or pageable).
template <typename TA>
gpch_status cg_run(gpch_ctx *ctx, int64_t n, const TA *A, int64_t lda, const double *B, int64_t ldb, double *X,
                   int64_t ldx, int nrhs, double rtol, int maxit, int R, cudaStream_t s, void *scratch, void *hbuf,
                   int *h_iters, double *h_relres, int prod = PROD_FP64, int variant = VAR_CLASSIC)
{
    const int64_t ldv = n;
    const unsigned vec_ctas = (unsigned)((n + THREADS - 1) / THREADS);
    CGBufs b;
    cg_carve(scratch, n, nrhs, prod, variant, &b);
    CGState &st = b.st;
    GPCH_CUDA(ctx, cudaMemsetAsync(st.counter, 0, 2 * sizeof(unsigned), s));
    GPCH_CUDA(ctx, cudaMemsetAsync(b.ic, 0, (2 * MAXRHS + 1) * sizeof(int), s));
    if (prod == PROD_DF) GPCH_CHECK(df_prepare<TA>(ctx, n, nrhs, A, lda, B, ldb, b, s));
    if (prod == PROD_OZ) GPCH_CHECK(oz_prepare<TA>(ctx, n, A, lda, b, s));
    const double rtol2 = rtol * rtol;
    // the true residuals b - A x: FP64 products, or with the tensor-core
    // products their form that keeps weight class 7 too (FP64-level)
    const int tprod = prod == PROD_OZ ? PROD_OZ_FULL : PROD_FP64;

    if (variant == VAR_CLASSIC) {
        // line 1: s = r = b - A x
        GPCH_CHECK(launch_matvec<TA>(ctx, n, nrhs, A, lda, X, ldx, b.T, ldv, st, MV_PLAIN, s, tprod, b.df));
        cg_init_kernel<<<vec_ctas, THREADS, 0, s>>>(n, nrhs, b.R, b.S, b.T, B, ldb, ldv, st);
        GPCH_LAUNCH_CHECK(ctx);
    } else {
        // r = b - A x; w = A r with gamma_0, delta_0, alpha_0; p = s = 0
        GPCH_CHECK(launch_matvec<TA>(ctx, n, nrhs, A, lda, X, ldx, b.T, ldv, st, MV_PLAIN, s, tprod, b.df));
        cg_resid_kernel<<<vec_ctas, THREADS, 0, s>>>(n, nrhs, b.R, b.T, B, ldb, ldv, st, 1);
        GPCH_LAUNCH_CHECK(ctx);
        GPCH_CUDA(ctx, cudaMemsetAsync(b.P, 0, (size_t)n * nrhs * sizeof(double), s));
        GPCH_CUDA(ctx, cudaMemsetAsync(b.S, 0, (size_t)n * nrhs * sizeof(double), s));
        GPCH_CHECK(launch_matvec<TA>(ctx, n, nrhs, A, lda, b.R, ldv, b.Wv, ldv, st, MV_SR, s, prod, b.df,
                                     SRArgs{rtol2, maxit, 1}));
    }

    int *h_done = static_cast<int *>(hbuf);
    const int chunk = 16;
    int it = 0;
    while (it < maxit) {
        const int k = (maxit - it < chunk) ? maxit - it : chunk;
        for (int q = 0; q < k; ++q) {
            const int iter = it + q + 1;   // 1-based number of the iteration being run
            const bool replace = R > 0 && iter % R == 0;
            if (variant == VAR_CLASSIC) {
                GPCH_CHECK(launch_matvec<TA>(ctx, n, nrhs, A, lda, b.S, ldv, b.T, ldv, st, MV_ALPHA, s, prod, b.df));
                gpch::PhaseScope phv(ctx, GPCH_PHASE_CG_VECTOR, s, 9.0 * (double)n * nrhs * sizeof(double));
                if (replace) {
                    cg_xupdate_kernel<<<vec_ctas, THREADS, 0, s>>>(n, nrhs, X, ldx, b.S, ldv, st);
                    GPCH_LAUNCH_CHECK(ctx);
                    GPCH_CHECK(launch_matvec<TA>(ctx, n, nrhs, A, lda, X, ldx, b.T, ldv, st, MV_PLAIN, s, tprod,
                                                 b.df));
                    cg_update_kernel<<<vec_ctas, THREADS, 0, s>>>(n, nrhs, X, ldx, b.R, b.S, b.T, B, ldb, ldv, st,
                                                                  rtol2, maxit, 1);
                } else {
                    cg_update_kernel<<<vec_ctas, THREADS, 0, s>>>(n, nrhs, X, ldx, b.R, b.S, b.T, B, ldb, ldv, st,
                                                                  rtol2, maxit, 0);
                }
                GPCH_LAUNCH_CHECK(ctx);
                cg_dir_kernel<<<vec_ctas, THREADS, 0, s>>>(n, nrhs, b.R, b.S, ldv, st);
                GPCH_LAUNCH_CHECK(ctx);
            } else {
                {
                    gpch::PhaseScope phv(ctx, GPCH_PHASE_CG_VECTOR, s, 11.0 * (double)n * nrhs * sizeof(double));
                    cgsr_vec_kernel<<<vec_ctas, THREADS, 0, s>>>(n, nrhs, X, ldx, b.R, b.Wv, b.P, b.S, ldv, st,
                                                                 replace ? 1 : 0);
                    GPCH_LAUNCH_CHECK(ctx);
                }
                if (replace) {
                    GPCH_CHECK(launch_matvec<TA>(ctx, n, nrhs, A, lda, X, ldx, b.T, ldv, st, MV_PLAIN, s, tprod,
                                                 b.df));
                    cg_resid_kernel<<<vec_ctas, THREADS, 0, s>>>(n, nrhs, b.R, b.T, B, ldb, ldv, st, 0);
                    GPCH_LAUNCH_CHECK(ctx);
                    GPCH_CHECK(launch_matvec<TA>(ctx, n, nrhs, A, lda, b.P, ldv, b.S, ldv, st, MV_PLAIN, s, prod,
                                                 b.df));
                }
                GPCH_CHECK(launch_matvec<TA>(ctx, n, nrhs, A, lda, b.R, ldv, b.Wv, ldv, st, MV_SR, s, prod, b.df,
                                             SRArgs{rtol2, maxit, 0}));
            }
        }
        it += k;
        GPCH_CUDA(ctx, cudaMemcpyAsync(h_done, st.done, sizeof(int), cudaMemcpyDeviceToHost, s));
        GPCH_CUDA(ctx, cudaStreamSynchronize(s));
        if (*h_done) break;
    }
    // statistics
    double *h_sc = reinterpret_cast<double *>(static_cast<char *>(hbuf) + 64);
    int *h_ic = reinterpret_cast<int *>(static_cast<char *>(hbuf) + 64 + 4 * MAXRHS * sizeof(double));
    GPCH_CUDA(ctx, cudaMemcpyAsync(h_sc, b.sc, 4 * MAXRHS * sizeof(double), cudaMemcpyDeviceToHost, s));
    GPCH_CUDA(ctx, cudaMemcpyAsync(h_ic, b.ic, (2 * MAXRHS + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
    int *h_ozerr = h_ic + 2 * MAXRHS + 1;
    if (prod == PROD_OZ) GPCH_CUDA(ctx, cudaMemcpyAsync(h_ozerr, b.df.oz.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    GPCH_CUDA(ctx, cudaStreamSynchronize(s));
    if (prod == PROD_OZ && *h_ozerr != 0)
        return gpch::fail(ctx, GPCH_TIMEOUT, "tensor-core product wait gave up (%d)", *h_ozerr);
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
                     int *h_iters, double *h_relres, int prod = PROD_FP64, int variant = VAR_CLASSIC)
{
    GPCH_CHECK(gpch::ws_reserve(ctx, cg_scratch_bytes(n, nrhs, prod, variant)));
    return cg_run<TA>(ctx, n, A, lda, B, ldb, X, ldx, nrhs, rtol, maxit, R, s, ctx->ws, ctx->pinned, h_iters,
                      h_relres, prod, variant);
}

// ------------------------------------------------------------ PCG (A9)
//
// Refined solve: preconditioned CG with M = Lt Lt^T, Lt the low-precision
// factor (FP32 storage), applied by the forward/back substitution of
// solve.cu.  A, x, r, dot products and recurrences stay in FP64; the
// iteration's products t = A s and the true residuals b - A x take
// double-float products (relative error below about 2^-44 per product,
// summed without further loss), so each entry of the measured residual is
// within about 2^-44 sum_j |A_ij| |x_j| of the exact one: at most 2^-44 of
// the backward error's denominator ||A||_inf ||x||_inf.  The host
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

struct RefineResult {
    int iterations = 0;
    double bwd[MAXRHS] = {0};
};

// PCG on one group of <= 16 right-hand sides.  L: FP32 factor (ldl);
// anorm_dev: ||A||_inf on the device (from mixed_init_enqueue).
gpch_status pcg_group(gpch_ctx *ctx, int64_t n, const double *A, int64_t lda, const float *L, int64_t ldl,
                      const double *B, int64_t ldb, double *X, int64_t ldx, int nrhs, double bwd_tol, int maxit,
                      int R, char *wsbase, cudaStream_t s, RefineResult &res, const double *anorm_dev,
                      float2 *packed_pre = nullptr)
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
    st.part = cv.take<double>(part_doubles(n, nrhs, PROD_DF));
    // double-float products for t = A s and the true residuals; with one
    // or two right-hand sides they read A's lower triangle only
    // (launch_symv_df; the first of them also stores the heads and tails of
    // A's lower triangle in a packed copy that the later ones read instead
    // of A), else all of A
    const bool sym = nrhs <= 2;
    double *sym_part = sym ? cv.take<double>(sy_part_doubles(n, mv_nr(nrhs))) : nullptr;
    // (a copy the input pass already wrote serves every product)
    float2 *sym_ap = !sym ? nullptr : packed_pre ? packed_pre : cv.take<float2>((size_t)sy_off(n, sy_strips(n)));
    bool sym_packed = packed_pre != nullptr;   // the packed copy is made
    CGBufs dfb{};
    dfb.df.SS = cv.take<float2>((size_t)n * mv_nr(nrhs));
    {
        double *d = cv.take<double>(2 * MAXRHS);
        dfb.df.scale = d;
        dfb.df.inv = d + MAXRHS;
        dfb.df.ebias = cv.take<int>(1);
        dfb.dmax = cv.take<double>(1 + MAXRHS);
    }
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
    GPCH_CHECK(df_prepare<double>(ctx, n, nrhs, A, lda, B, ldb, dfb, s));
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
        if (sym) {
            GPCH_CHECK(launch_symv_df(ctx, n, nrhs, A, lda, Sv, ldv, Tv, ldv, st, MV_ALPHA, s, dfb.df, sym_part, sym_ap,
                                      sym_packed ? SY_PACKED : SY_WRITE));
            sym_packed = true;
        } else {
            GPCH_CHECK(launch_matvec<double>(ctx, n, nrhs, A, lda, Sv, ldv, Tv, ldv, st, MV_ALPHA, s, PROD_DF, dfb.df));
        }
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
            if (sym)
                GPCH_CHECK(launch_symv_df(ctx, n, nrhs, A, lda, X, ldx, Tv, ldv, st, MV_PLAIN, s, dfb.df, sym_part,
                                          sym_ap, SY_PACKED));
            else
                GPCH_CHECK(launch_matvec<double>(ctx, n, nrhs, A, lda, X, ldx, Tv, ldv, st, MV_PLAIN, s, PROD_DF,
                                                 dfb.df));
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

size_t pcg_ws_bytes(int64_t n, int nrhs, bool own_packed = true)
{
    gpch::Carver dry(nullptr);
    for (int i = 0; i < 4; ++i) dry.take<double>((size_t)n * nrhs);
    dry.take<char>(gpch::solve_ws_bytes(n, nrhs));
    dry.take<double>(4 * MAXRHS);
    dry.take<int>(2 * MAXRHS + 1);
    dry.take<unsigned>(2);
    dry.take<double>(part_doubles(n, nrhs, PROD_DF));
    if (nrhs <= 2) {
        dry.take<double>(sy_part_doubles(n, mv_nr(nrhs)));
        if (own_packed) dry.take<float2>((size_t)sy_off(n, sy_strips(n)));
    }
    dry.take<float2>((size_t)n * mv_nr(nrhs));
    dry.take<double>(2 * MAXRHS);
    dry.take<int>(1);
    dry.take<double>(1 + MAXRHS);
    dry.take<double>(6 * MAXRHS + 2);
    return dry.off;
}

// max_i A_ii (for the shift schedule), synchronously.
gpch_status diag_max(gpch_ctx *ctx, int64_t n, const double *A, int64_t lda, double *dev2, cudaStream_t s,
                     double *out)
{
    GPCH_CUDA(ctx, cudaMemsetAsync(dev2, 0, 2 * sizeof(double), s));
    diag_max_kernel<double><<<(unsigned)((n + THREADS - 1) / THREADS < 148 ? (n + THREADS - 1) / THREADS : 148), THREADS, 0,
                      s>>>(n, A, lda, dev2 + 1);
    GPCH_LAUNCH_CHECK(ctx);
    double *h = static_cast<double *>(ctx->pinned);
    GPCH_CUDA(ctx, cudaMemcpyAsync(h, dev2, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    GPCH_CUDA(ctx, cudaStreamSynchronize(s));
    *out = h[1];
    return GPCH_OK;
}

}  // namespace

extern "C" gpch_status gpch_cg_solve_ex(gpch_ctx *ctx, int64_t n, const void *A, gpch_dtype dtype, int64_t lda,
                                        const double *B, int64_t ldb, double *X, int64_t ldx, int nrhs, double rtol,
                                        int maxit, int replace_every, const gpch_cg_opts *opts, void *stream,
                                        gpch_cg_stats *stats)
{
    GPCH_ARG(ctx, ctx != nullptr, "null context");
    if (stats) *stats = gpch_cg_stats{0, 0, 0.0};
    const int variant = opts ? opts->variant : GPCH_CG_CLASSIC;
    const int prod = opts ? opts->products : GPCH_CG_PRODUCTS_FP64;
    GPCH_ARG(ctx, variant == GPCH_CG_CLASSIC || variant == GPCH_CG_SINGLE_REDUCTION, "bad CG variant");
    GPCH_ARG(ctx,
             prod == GPCH_CG_PRODUCTS_FP64 || prod == GPCH_CG_PRODUCTS_DOUBLE_FLOAT || prod == GPCH_CG_PRODUCTS_TENSOR,
             "bad CG products");
    GPCH_ARG(ctx, n >= 0 && nrhs >= 0, "n < 0 or nrhs < 0");
    GPCH_ARG(ctx, prod != GPCH_CG_PRODUCTS_TENSOR || (n + 127) / 128 * 128 * ((n + 511) / 512 * 16) * 4 < (int64_t)0x7fffffff,
             "n too large for the tensor-core path");
    GPCH_ARG(ctx, lda >= (n > 0 ? n : 1) && ldb >= (n > 0 ? n : 1) && ldx >= (n > 0 ? n : 1), "ld < n");
    GPCH_ARG(ctx, dtype == GPCH_F64 || dtype == GPCH_F32, "bad dtype");
    GPCH_ARG(ctx, maxit > 0 && replace_every >= 0 && rtol >= 0.0, "bad maxit / replace_every / rtol");
    if (n == 0 || nrhs == 0) return GPCH_OK;
    GPCH_ARG(ctx, A && B && X, "null pointer");
    GPCH_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    const int pv = prod == GPCH_CG_PRODUCTS_DOUBLE_FLOAT ? PROD_DF : prod == GPCH_CG_PRODUCTS_TENSOR ? PROD_OZ : PROD_FP64;
    const int vv = variant == GPCH_CG_SINGLE_REDUCTION ? VAR_SINGLE_REDUCTION : VAR_CLASSIC;
    int max_it = 0, conv = 0;
    double rel_max = 0.0;
    for (int r0 = 0; r0 < nrhs; r0 += MAXRHS) {
        const int g = (nrhs - r0 < MAXRHS) ? nrhs - r0 : MAXRHS;
        int iters[MAXRHS];
        double rel[MAXRHS];
        gpch_status st;
        if (dtype == GPCH_F64)
            st = cg_group<double>(ctx, n, static_cast<const double *>(A), lda, B + r0 * ldb, ldb, X + r0 * ldx,
                                  ldx, g, rtol, maxit, replace_every, s, iters, rel, pv, vv);
        else
            st = cg_group<float>(ctx, n, static_cast<const float *>(A), lda, B + r0 * ldb, ldb, X + r0 * ldx,
                                 ldx, g, rtol, maxit, replace_every, s, iters, rel, pv, vv);
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

extern "C" gpch_status gpch_cg_solve(gpch_ctx *ctx, int64_t n, const void *A, gpch_dtype dtype, int64_t lda,
                                     const double *B, int64_t ldb, double *X, int64_t ldx, int nrhs, double rtol,
                                     int maxit, int replace_every, void *stream, gpch_cg_stats *stats)
{
    return gpch_cg_solve_ex(ctx, n, A, dtype, lda, B, ldb, X, ldx, nrhs, rtol, maxit, replace_every, nullptr, stream,
                            stats);
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
    GPCH_ARG(ctx, tile == 0 || (tile >= 64 && tile <= 1024 && tile % 64 == 0),
             "tile must be 0 (tuned) or a multiple of 64 in [64, 1024]");
    GPCH_ARG(ctx, bwd_tol > 0.0 && maxit > 0, "bad bwd_tol / maxit");
    if (tile == 0) tile = gpch::tune_table(ctx->device).refined_tile[gpch::tune_bucket(n)];
    GPCH_ARG(ctx, n < (int64_t)1 << 31, "n too large");
    if (n == 0 || nrhs == 0) return GPCH_OK;
    GPCH_ARG(ctx, A && B && X, "null pointer");
    GPCH_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t ldw = (n + 31) / 32 * 32;
    const int g = nrhs < MAXRHS ? nrhs : MAXRHS;
    // with one or two right-hand sides the input pass also writes the
    // products' packed copy of A's lower triangle (next to W, outside the
    // factor's workspace, which the products' partials reuse)
    const bool pre_packed = nrhs <= 2;
    const size_t packed_n = pre_packed ? (size_t)sy_off(n, sy_strips(n)) : 0;
    gpch::Carver dry(nullptr);
    dry.take<float>((size_t)ldw * n);
    dry.take<double>(3);
    dry.take<float>(gpch::anorm_ws_floats(n));
    if (pre_packed) dry.take<float2>(packed_n);
    const size_t fixed = dry.off;
    const size_t mix = gpch::mixed_ws_bytes(n, tile);
    size_t pcg = pcg_ws_bytes(n, g, !pre_packed);
    if (nrhs > MAXRHS && nrhs % MAXRHS != 0) {
        // the last group is smaller and may take the lower-triangle product's partials
        const size_t last = pcg_ws_bytes(n, nrhs % MAXRHS);
        if (last > pcg) pcg = last;
    }
    GPCH_CHECK(gpch::ws_reserve(ctx, fixed + 256 + (mix > pcg ? mix : pcg)));
    gpch::Carver cv(ctx->ws);
    float *W = cv.take<float>((size_t)ldw * n);
    double *dev2 = cv.take<double>(3);   // [0, 2): diag_max, [2]: ||A||_inf
    float *norm_ws = cv.take<float>(gpch::anorm_ws_floats(n));
    float2 *packed = pre_packed ? cv.take<float2>(packed_n) : nullptr;
    char *rest = static_cast<char *>(ctx->ws) + ((cv.off + 255) & ~size_t(255));

    double dmax = 0.0;
    GPCH_CHECK(diag_max(ctx, n, A, lda, dev2, s, &dmax));
    // unit roundoff of the step-3 operands: bf16 8 bits, split bf16 ~16 bits,
    // scaled split binary16 ~22 bits
    const double ulow = (prec == GPCH_PREC_BF16) ? 1.0 / 256.0
                        : (prec == GPCH_PREC_SPLIT_BF16) ? 1.0 / 65536.0
                                                         : 1.0 / 4194304.0;
    double shift = (prec == GPCH_PREC_BF16) ? 2.0 * ulow * dmax : 0.0;
    // the packed copy's exponent offset, as df_scales_kernel derives it
    // from the same largest diagonal entry
    int pack_ea = dmax > 0.0 ? std::ilogb(dmax) : 0;
    pack_ea = pack_ea < -800 ? -800 : (pack_ea > 800 ? 800 : pack_ea);
    const unsigned pack_ebias = (unsigned)(896 + pack_ea);
    int attempts = 0;
    int64_t info = 1;
    for (; attempts < 9; ++attempts) {
        // W = A + shift I and ||A||_inf, run by the factor block column by
        // block column ahead of its use
        const gpch::MixedInit mi{A, lda, shift, dev2 + 2, norm_ws, packed, pack_ebias};
        int64_t *d_info;
        int *d_err;
        GPCH_CHECK(gpch::mixed_factor_enqueue(ctx, n, tile, W, ldw, (int)prec, rest, &d_info, &d_err, s, &mi));
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
                             rest, s, rr, dev2 + 2, packed));
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

// Y = A X from A's lower triangle with double-float products, the product
// of the refined solve's iteration (sym_mv_df_kernel), columns in pairs.
extern "C" gpch_status gpch_symv_lower(gpch_ctx *ctx, int64_t n, const double *A, int64_t lda, const double *X,
                                       int64_t ldx, double *Y, int64_t ldy, int nrhs, void *stream)
{
    GPCH_ARG(ctx, ctx != nullptr, "null context");
    GPCH_ARG(ctx, n >= 0 && nrhs >= 0, "n < 0 or nrhs < 0");
    GPCH_ARG(ctx, lda >= (n > 0 ? n : 1) && ldx >= (n > 0 ? n : 1) && ldy >= (n > 0 ? n : 1), "ld < n");
    GPCH_ARG(ctx, n < (int64_t)1 << 24, "n too large");
    if (n == 0 || nrhs == 0) return GPCH_OK;
    GPCH_ARG(ctx, A && X && Y, "null pointer");
    GPCH_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    const int nr = nrhs >= 2 ? 2 : 1;
    auto carve = [&](gpch::Carver &cv, CGBufs &b, double *&part) {
        b.df.SS = cv.take<float2>((size_t)n * nr);
        double *d = cv.take<double>(2 * MAXRHS);
        b.df.scale = d;
        b.df.inv = d + MAXRHS;
        b.df.ebias = cv.take<int>(1);
        b.dmax = cv.take<double>(1 + MAXRHS);
        b.st.done = cv.take<int>(1);
        b.st.counter = cv.take<unsigned>(2);
        part = cv.take<double>(sy_part_doubles(n, nr));
    };
    CGBufs b{};
    double *part = nullptr;
    {
        gpch::Carver dry(nullptr);
        carve(dry, b, part);
        GPCH_CHECK(gpch::ws_reserve(ctx, dry.off));
    }
    gpch::Carver cv(ctx->ws);
    carve(cv, b, part);
    GPCH_CUDA(ctx, cudaMemsetAsync(b.st.done, 0, sizeof(int), s));
    for (int r0 = 0; r0 < nrhs; r0 += 2) {
        const int g = (nrhs - r0 < 2) ? nrhs - r0 : 2;
        GPCH_CHECK(df_prepare<double>(ctx, n, g, A, lda, X + (int64_t)r0 * ldx, ldx, b, s));
        GPCH_CHECK(launch_symv_df(ctx, n, g, A, lda, X + (int64_t)r0 * ldx, ldx, Y + (int64_t)r0 * ldy, ldy, b.st,
                                  MV_PLAIN, s, b.df, part));
    }
    return GPCH_OK;
}

// ---------------------------------------- row-split CG building blocks (f4)
//
// One rank of a CG solve whose rows are split over ranks (the paper's
// horizontal split of Sec. 3.1, carried from CPU/GPU to GPU/GPU): a rank
// owns rows r0 .. r0+m-1 of A, stored by symmetry as the n x m column block
// A[:, r0 : r0+m], and the matching m rows of every vector.  The caller
// moves data between ranks (an allgather of the vector fed to the product,
// an allreduce of two sums per right-hand side); these calls do every
// arithmetic step of the single-reduction iteration on the rank's rows.

namespace {

// per-CTA partial sums of r^T r and w^T r over the rank's rows; the last
// CTA adds them in a fixed order into sums[0, nrhs) and sums[nrhs, 2 nrhs).
__global__ void __launch_bounds__(THREADS) cgsr_partials_kernel(int64_t m, int nrhs, const double *R, int64_t ldr,
                                                                const double *Wv, int64_t ldw, double *part,
                                                                unsigned *counter, double *sums)
{
    __shared__ double red[THREADS / 32][2 * MAXRHS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t i = (int64_t)blockIdx.x * THREADS + tid;
    for (int r = 0; r < nrhs; ++r) {
        double g = 0.0, d = 0.0;
        if (i < m) {
            const double ri = R[i + r * ldr];
            g = ri * ri;
            d = Wv[i + r * ldw] * ri;
        }
        g = warp_sum(g);
        d = warp_sum(d);
        if (lane == 0) {
            red[warp][r] = g;
            red[warp][MAXRHS + r] = d;
        }
    }
    __syncthreads();
    if (tid < 2 * nrhs) {
        const int q = tid < nrhs ? tid : MAXRHS + tid - nrhs;
        double v = 0.0;
        for (int w = 0; w < THREADS / 32; ++w) v += red[w][q];
        part[(size_t)blockIdx.x * 2 * MAXRHS + q] = v;
    }
    if (last_cta(counter)) {
        if (tid < 2 * nrhs) {
            const int q = tid < nrhs ? tid : MAXRHS + tid - nrhs;
            double v = 0.0;
            for (unsigned b = 0; b < gridDim.x; ++b) v += __ldcg(&part[(size_t)b * 2 * MAXRHS + q]);
            sums[tid] = v;
        }
        if (tid == 0) *counter = 0;
    }
}

// The scalar step of the single-reduction form from the ranks' reduced sums
// (gamma' = sums[r], delta = sums[nrhs + r]); one thread per column.
__global__ void cgsr_scalars_kernel(int nrhs, const double *sums, gpch_cgsr_state *st, int first, double rtol2,
                                    int maxit)
{
    __shared__ int any_active;
    const int r = threadIdx.x;
    if (r == 0) any_active = 0;
    __syncthreads();
    if (r < nrhs) {
        const double g = sums[r], d = sums[nrhs + r];
        if (first) {
            st->gamma0[r] = g;
            st->gamma[r] = g;
            st->iters[r] = 0;
            st->beta[r] = 0.0;
            st->alpha[r] = g > 0.0 ? g / d : 0.0;
            st->active[r] = g > 0.0 ? 1 : 0;
        } else if (st->active[r]) {
            const int it = st->iters[r] + 1;
            st->iters[r] = it;
            const double b = g / st->gamma[r];
            st->alpha[r] = g / (d - b * g / st->alpha[r]);
            st->beta[r] = b;
            st->gamma[r] = g;
            if (g <= rtol2 * st->gamma0[r] || it >= maxit) st->active[r] = 0;
        }
        if (st->active[r]) atomicOr(&any_active, 1);
    }
    __syncthreads();
    if (r == 0) st->done = any_active ? 0 : 1;
}

inline CGState state_view(gpch_cgsr_state *st)
{
    CGState v;
    v.u = st->gamma;
    v.u0 = st->gamma0;
    v.alpha = st->alpha;
    v.beta = st->beta;
    v.active = st->active;
    v.iters = st->iters;
    v.done = &st->done;
    v.counter = nullptr;
    v.part = nullptr;
    return v;
}

template <typename TA>
gpch_status block_matvec(gpch_ctx *ctx, int64_t n, int64_t m, int64_t r0, const TA *A, int64_t lda, const double *V,
                         int64_t ldv, double *T, int64_t ldt, int nrhs, int prod, cudaStream_t s)
{
    // scratch: a zero `done` word, and for double-float products the split
    // vector and its scales
    gpch::Carver dry(nullptr);
    dry.take<int>(1);
    if (prod == PROD_DF) {
        dry.take<float2>((size_t)n * mv_nr(nrhs));
        dry.take<double>(2 * MAXRHS);
        dry.take<int>(1);
        dry.take<double>(1 + MAXRHS);
    }
    GPCH_CHECK(gpch::ws_reserve(ctx, dry.off));
    gpch::Carver cv(ctx->ws);
    CGState st{};
    st.done = cv.take<int>(1);
    GPCH_CUDA(ctx, cudaMemsetAsync(st.done, 0, sizeof(int), s));
    DFArgs df{nullptr, nullptr, nullptr, nullptr};
    if (prod == PROD_DF) {
        df.SS = cv.take<float2>((size_t)n * mv_nr(nrhs));
        double *d = cv.take<double>(2 * MAXRHS);
        df.scale = d;
        df.inv = d + MAXRHS;
        df.ebias = cv.take<int>(1);
        double *dmax = cv.take<double>(1 + MAXRHS);
        GPCH_CUDA(ctx, cudaMemsetAsync(dmax, 0, (1 + MAXRHS) * sizeof(double), s));
        const unsigned mc = (unsigned)((m + THREADS - 1) / THREADS), nc = (unsigned)((n + THREADS - 1) / THREADS);
        if (sizeof(TA) == 8) {
            // the block's diagonal entries A[r0 + j, j]
            diag_max_kernel<TA><<<mc < 148 ? mc : 148, THREADS, 0, s>>>(m, A + r0, lda, dmax);
            GPCH_LAUNCH_CHECK(ctx);
        }
        absmax_cols_kernel<<<nc, THREADS, 0, s>>>(n, nrhs, V, ldv, dmax + 1);
        GPCH_LAUNCH_CHECK(ctx);
        df_scales_kernel<<<1, 32, 0, s>>>(nrhs, dmax, sizeof(TA) == 8 ? 1 : 0, d, d + MAXRHS,
                                          const_cast<int *>(df.ebias));
        GPCH_LAUNCH_CHECK(ctx);
    }
    return launch_matvec<TA>(ctx, n, nrhs, A, lda, V, ldv, T, ldt, st, MV_PLAIN, s, prod, df, SRArgs{0.0, 0, 0}, m);
}

}  // namespace

extern "C" gpch_status gpch_block_matvec(gpch_ctx *ctx, int64_t n, int64_t m, int64_t r0, const void *Ablk,
                                         gpch_dtype dtype, int64_t lda, const double *V, int64_t ldv, double *T,
                                         int64_t ldt, int nrhs, int32_t products, void *stream)
{
    GPCH_ARG(ctx, ctx != nullptr, "null context");
    GPCH_ARG(ctx, n >= 0 && m >= 0 && r0 >= 0 && r0 + m <= n, "need 0 <= r0 <= r0 + m <= n");
    GPCH_ARG(ctx, nrhs >= 0 && nrhs <= MAXRHS, "need 0 <= nrhs <= 16");
    GPCH_ARG(ctx, lda >= (n > 0 ? n : 1) && ldv >= (n > 0 ? n : 1) && ldt >= (m > 0 ? m : 1), "ld too small");
    GPCH_ARG(ctx, dtype == GPCH_F64 || dtype == GPCH_F32, "bad dtype");
    GPCH_ARG(ctx, products == GPCH_CG_PRODUCTS_FP64 || products == GPCH_CG_PRODUCTS_DOUBLE_FLOAT, "bad products");
    if (n == 0 || m == 0 || nrhs == 0) return GPCH_OK;
    GPCH_ARG(ctx, Ablk && V && T, "null pointer");
    GPCH_CUDA(ctx, cudaSetDevice(ctx->device));
    const int prod = products == GPCH_CG_PRODUCTS_DOUBLE_FLOAT ? PROD_DF : PROD_FP64;
    if (dtype == GPCH_F64)
        return block_matvec<double>(ctx, n, m, r0, static_cast<const double *>(Ablk), lda, V, ldv, T, ldt, nrhs, prod,
                                    (cudaStream_t)stream);
    return block_matvec<float>(ctx, n, m, r0, static_cast<const float *>(Ablk), lda, V, ldv, T, ldt, nrhs, prod,
                               (cudaStream_t)stream);
}

extern "C" gpch_status gpch_cgsr_partials(gpch_ctx *ctx, int64_t m, int nrhs, const double *R, int64_t ldr,
                                          const double *W, int64_t ldw, double *sums, void *stream)
{
    GPCH_ARG(ctx, ctx != nullptr, "null context");
    GPCH_ARG(ctx, m >= 0 && nrhs >= 0 && nrhs <= MAXRHS, "need m >= 0 and 0 <= nrhs <= 16");
    GPCH_ARG(ctx, ldr >= (m > 0 ? m : 1) && ldw >= (m > 0 ? m : 1), "ld < m");
    if (nrhs == 0) return GPCH_OK;
    GPCH_ARG(ctx, sums != nullptr && (m == 0 || (R && W)), "null pointer");
    GPCH_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    if (m == 0) {
        GPCH_CUDA(ctx, cudaMemsetAsync(sums, 0, 2 * nrhs * sizeof(double), s));
        return GPCH_OK;
    }
    const unsigned ctas = (unsigned)((m + THREADS - 1) / THREADS);
    gpch::Carver dry(nullptr);
    dry.take<unsigned>(1);
    dry.take<double>((size_t)ctas * 2 * MAXRHS);
    GPCH_CHECK(gpch::ws_reserve(ctx, dry.off));
    gpch::Carver cv(ctx->ws);
    unsigned *counter = cv.take<unsigned>(1);
    double *part = cv.take<double>((size_t)ctas * 2 * MAXRHS);
    GPCH_CUDA(ctx, cudaMemsetAsync(counter, 0, sizeof(unsigned), s));
    cgsr_partials_kernel<<<ctas, THREADS, 0, s>>>(m, nrhs, R, ldr, W, ldw, part, counter, sums);
    GPCH_LAUNCH_CHECK(ctx);
    return GPCH_OK;
}

extern "C" gpch_status gpch_cgsr_scalars(gpch_ctx *ctx, int nrhs, const double *sums, gpch_cgsr_state *state,
                                         int first, double rtol, int maxit, void *stream)
{
    GPCH_ARG(ctx, ctx != nullptr, "null context");
    GPCH_ARG(ctx, nrhs >= 0 && nrhs <= MAXRHS, "need 0 <= nrhs <= 16");
    GPCH_ARG(ctx, rtol >= 0.0 && maxit > 0, "bad rtol / maxit");
    GPCH_ARG(ctx, sums && state, "null pointer");
    GPCH_CUDA(ctx, cudaSetDevice(ctx->device));
    cgsr_scalars_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(nrhs, sums, state, first, rtol * rtol, maxit);
    GPCH_LAUNCH_CHECK(ctx);
    return GPCH_OK;
}

extern "C" gpch_status gpch_cgsr_vectors(gpch_ctx *ctx, int64_t m, int nrhs, gpch_cgsr_state *state, double *X,
                                         int64_t ldx, double *R, const double *W, double *P, double *S, int64_t ld,
                                         int replace, void *stream)
{
    GPCH_ARG(ctx, ctx != nullptr, "null context");
    GPCH_ARG(ctx, m >= 0 && nrhs >= 0 && nrhs <= MAXRHS, "need m >= 0 and 0 <= nrhs <= 16");
    GPCH_ARG(ctx, ldx >= (m > 0 ? m : 1) && ld >= (m > 0 ? m : 1), "ld < m");
    if (m == 0 || nrhs == 0) return GPCH_OK;
    GPCH_ARG(ctx, state && X && R && W && P && S, "null pointer");
    GPCH_CUDA(ctx, cudaSetDevice(ctx->device));
    cgsr_vec_kernel<<<(unsigned)((m + THREADS - 1) / THREADS), THREADS, 0, (cudaStream_t)stream>>>(
        m, nrhs, X, ldx, R, W, P, S, ld, state_view(state), replace ? 1 : 0);
    GPCH_LAUNCH_CHECK(ctx);
    return GPCH_OK;
}

extern "C" gpch_status gpch_cgsr_residual(gpch_ctx *ctx, int64_t m, int nrhs, gpch_cgsr_state *state,
                                          const double *B, int64_t ldb, const double *T, double *R, int64_t ld,
                                          int all, void *stream)
{
    GPCH_ARG(ctx, ctx != nullptr, "null context");
    GPCH_ARG(ctx, m >= 0 && nrhs >= 0 && nrhs <= MAXRHS, "need m >= 0 and 0 <= nrhs <= 16");
    GPCH_ARG(ctx, ldb >= (m > 0 ? m : 1) && ld >= (m > 0 ? m : 1), "ld < m");
    if (m == 0 || nrhs == 0) return GPCH_OK;
    GPCH_ARG(ctx, state && B && T && R, "null pointer");
    GPCH_CUDA(ctx, cudaSetDevice(ctx->device));
    cg_resid_kernel<<<(unsigned)((m + THREADS - 1) / THREADS), THREADS, 0, (cudaStream_t)stream>>>(
        m, nrhs, R, T, B, ldb, ld, state_view(state), all ? 1 : 0);
    GPCH_LAUNCH_CHECK(ctx);
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
