// solve.cu -- A5: forward and back substitution with the Cholesky factor,
// L Y = B then L^T X = Y (Sec. 2.2), blocked by 64 rows.
//
// The 64 x 64 diagonal blocks of L are inverted once (one launch).  Each
// sweep is then ONE cooperative launch of one CTA per SM.  Block row I is
// owned by CTA I mod P, which keeps its partial sums in shared memory.
// Walking the blocks in sweep order, every CTA waits for the solved block J
// (a flag word per block, bounded wait), adds L_IJ y_J (forward) or
// L_JI^T x_J (back) to each block I it owns further down the sweep, and the
// owner of the next block does that block first, solves it with its
// inverted diagonal block and publishes it before touching its other
// blocks, so the serial chain is one 64 x 64 update and one 64 x 64 solve
// per block.  L is read once per sweep.  With an FP64 factor all products
// are FP64; with the FP32 (preconditioner) factor each 64 x 64 block
// product runs in FP32 and is added to FP64 partial sums, and the diagonal
// block solves stay FP64.
//
// The preconditioner's sweeps (FP32 factor, one or two right-hand sides)
// use 128-row blocks and the coupling blocks of couple_kernel, which leave
// one 128 x 128 block product per block on the serial chain
// (trsv_sweep128_kernel).
#include <mutex>
#include <type_traits>

#include "dense_fp64.cuh"
#include "tc_ptx.cuh"

namespace {

using gpch::LEAF;

constexpr int SW_THREADS = 256;
constexpr int SW_MAXRHS = 16;
constexpr uint32_t FLAG_SPIN_LIMIT = 1u << 22;

// Arithmetic type of the sweep: FP32 products for an FP32 factor, FP64
// for an FP64 factor.
template <typename TL>
using sweep_math_t = typename std::conditional<sizeof(TL) == 4, float, double>::type;

// Inverts the 64 x 64 diagonal blocks of L in FP64 and stores them in the
// sweep's arithmetic type.
template <typename TL>
__global__ void __launch_bounds__(256) inv_diag_blocks_kernel(int64_t n, const TL *__restrict__ L,
                                                              int64_t ldl, sweep_math_t<TL> *Linv)
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
    sweep_math_t<TL> *dst = Linv + J * LEAF * LEAF;
    for (int e = threadIdx.x; e < LEAF * LEAF; e += blockDim.x) {
        int r = e % LEAF, c = e / LEAF;
        dst[r + c * LEAF] = (sweep_math_t<TL>)Vi[r][c];
    }
}

// 128 x 128 inverses of the diagonal blocks of an FP32 factor, from the
// 64 x 64 ones: inv([L11 0; L21 L22]) = [inv11 0; -inv22 L21 inv11 inv22],
// the off-diagonal block in FP32 arithmetic (the sweeps that use these
// blocks compute in FP32).  One CTA per 128-block; padding past n is the
// identity.  Out: column-major, ld 128.
__global__ void __launch_bounds__(256) inv128_kernel(int64_t n, const float *__restrict__ L, int64_t ldl,
                                                     const float *__restrict__ Linv64, float *Linv128)
{
    __shared__ float A[64][65], Bm[64][65];
    const int tid = threadIdx.x;
    const int64_t B = blockIdx.x, o = B * 128;
    const int64_t N64 = (n + LEAF - 1) / LEAF;
    const bool has2 = 2 * B + 1 < N64;
    const float *inv11 = Linv64 + (2 * B) * LEAF * LEAF;
    const float *inv22 = Linv64 + (2 * B + 1) * LEAF * LEAF;
    float *dst = Linv128 + B * 128 * 128;
    // T = L21 inv11: A = L21, Bm = inv11
    for (int e = tid; e < LEAF * LEAF; e += 256) {
        const int r = e % LEAF, c = e / LEAF;
        const int64_t row = o + LEAF + r;
        A[r][c] = (has2 && row < n) ? L[row + (o + c) * ldl] : 0.0f;
        Bm[r][c] = inv11[e];
    }
    __syncthreads();
    const int tr = tid % 16, tc = tid / 16;   // 4 x 4 outputs: rows tr + 16i, columns tc + 16j
    float t[4][4] = {};
    for (int k = 0; k < LEAF; ++k)
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) t[i][j] = fmaf(A[tr + 16 * i][k], Bm[k][tc + 16 * j], t[i][j]);
    __syncthreads();
    // X = -inv22 T: A = inv22, Bm = T
    for (int e = tid; e < LEAF * LEAF; e += 256) {
        const int r = e % LEAF, c = e / LEAF;
        A[r][c] = has2 ? inv22[e] : (r == c ? 1.0f : 0.0f);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) Bm[tr + 16 * i][tc + 16 * j] = t[i][j];
    __syncthreads();
    float x[4][4] = {};
    for (int k = 0; k < LEAF; ++k)
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) x[i][j] = fmaf(A[tr + 16 * i][k], Bm[k][tc + 16 * j], x[i][j]);
    for (int e = tid; e < 128 * 128; e += 256) {
        const int r = e % 128, c = e / 128;
        float v = 0.0f;
        if (r < LEAF && c < LEAF) v = inv11[r + c * LEAF];
        else if (r >= LEAF && c >= LEAF) v = has2 ? inv22[(r - LEAF) + (c - LEAF) * LEAF] : (r == c ? 1.0f : 0.0f);
        dst[e] = v;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) dst[(LEAF + tr + 16 * i) + (tc + 16 * j) * 128] = -x[i][j];
}

// Coupling blocks of the FP32 sweeps with 128-row blocks (once per factor),
// from the 128 x 128 diagonal-block inverses Linv128 (column-major, ld 128):
//   F_I = inv(L_II) L_{I,I-1}     (1 <= I < N), the forward coupling, and
//   G_I = L_{I+1,I} inv(L_II)     (0 <= I < N-1), the back coupling,
// so that the forward sweep's block I is inv(L_II)(b_I - sum_{K<I-1} L_IK y_K)
// - F_I y_{I-1} and the back sweep's block I is inv(L_II)^T(y_I -
// sum_{K>I+1} L_KI^T x_K) - G_I^T x_{I+1}.  Both are stored in (N 128) x 128
// column-major matrices of leading dimension N 128 with block I in rows
// 128 I .. 128 I + 127: F_I(t, k) at row 128 I + t, column k; G_I(k, t) at
// row 128 I + k, column t (the orientation of L_{I+1,I}).  Rows of L past n
// count as zero.  Grid (N, 2): y = 0 makes F_I, y = 1 makes G_I; 256
// threads, 8 x 8 outputs each, K in chunks of 32 through shared memory.
__global__ void __launch_bounds__(256) couple_kernel(int64_t n, const float *__restrict__ L, int64_t ldl,
                                                     const float *__restrict__ Linv128, float *F, float *G)
{
    __shared__ float As[32][132], Bs[32][132];   // As[u][i] = A(i, u), Bs[u][j] = B(u, j)
    const int64_t N = (n + 127) / 128, I = blockIdx.x, ld = N * 128;
    const bool fwd = blockIdx.y == 0;
    float *out = fwd ? F : G;
    if ((fwd && I == 0) || (!fwd && I == N - 1)) {
        // no coupling: zero block
        for (int e = threadIdx.x; e < 128 * 128; e += 256) out[(I * 128 + e % 128) + (int64_t)(e / 128) * ld] = 0.0f;
        return;
    }
    const float *inv = Linv128 + I * 128 * 128;
    const int tid = threadIdx.x, ti = tid % 16, tj = tid / 16;   // outputs rows ti + 16a, columns tj + 16b
    float acc[8][8] = {};
    for (int u0 = 0; u0 < 128; u0 += 32) {
        // every global read walks down a column (coalesced)
        for (int e = tid; e < 32 * 128; e += 256) {
            const int i = e % 128, u = u0 + e / 128;
            if (fwd) {
                As[u - u0][i] = inv[i + u * 128];   // A = inv(L_II): row i, column u
            } else {
                const int64_t row = (I + 1) * 128 + i;   // A = L_{I+1,I}: row i, column u
                As[u - u0][i] = row < n ? L[row + (I * 128 + u) * ldl] : 0.0f;
            }
        }
        for (int e = tid; e < 32 * 128; e += 256) {
            const int u = u0 + e % 32, j = e / 32;
            if (fwd) {
                const int64_t row = I * 128 + u;         // B = L_{I,I-1}: row u, column j
                Bs[u - u0][j] = row < n ? L[row + ((I - 1) * 128 + j) * ldl] : 0.0f;
            } else {
                Bs[u - u0][j] = inv[u + j * 128];        // B = inv(L_II): row u, column j
            }
        }
        __syncthreads();
#pragma unroll 4
        for (int u = 0; u < 32; ++u) {
            float av[8], bv[8];
#pragma unroll
            for (int x = 0; x < 8; ++x) {
                av[x] = As[u][ti + 16 * x];
                bv[x] = Bs[u][tj + 16 * x];
            }
#pragma unroll
            for (int x = 0; x < 8; ++x)
#pragma unroll
                for (int y = 0; y < 8; ++y) acc[x][y] = fmaf(av[x], bv[y], acc[x][y]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int x = 0; x < 8; ++x)
#pragma unroll
        for (int y = 0; y < 8; ++y) out[(I * 128 + ti + 16 * x) + (int64_t)(tj + 16 * y) * ld] = acc[x][y];
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void cp_async_elem(void *dst, const void *src, int bytes)
{
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    if (bytes == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Blocks of L staged per step: 4 (FP32 factor) or 2 (FP64 factor).
template <typename TL, int BS>
constexpr int sweep_slots()
{
    return sizeof(TL) == 4 ? 4 : 2;
}
// Staged block of L: entry (t, k) at k * (BS + 1) + (k / (BS / 4)) * PADQ + t.
// The four lanes that share an item t read k-ranges BS/4 apart; the extra
// PADQ per range puts them in different banks (FP32: 8 words, FP64: 4).
template <typename TL>
constexpr int padq()
{
    return sizeof(TL) == 4 ? 8 : 4;
}
template <int BS>
constexpr int lstride()
{
    return BS * (BS + 1) + 32;
}
// Solved block: rhs c, row r at c * YSTRIDE + (r / (BS/4)) * (BS/4 + 1) + r % (BS/4).
template <int BS>
constexpr int ystride()
{
    return 4 * (BS / 4 + 1);
}
// Inverse block, column stride: r + 4p (FP64, half-warp) or r + 8p (FP32,
// warp) then fall in distinct banks.
template <typename TL, int BS>
constexpr int istride()
{
    return sizeof(TL) == 4 ? BS + 8 : BS + 4;
}

// Dynamic shared memory of one sweep CTA owning `nown` blocks.
template <typename TL, int BS>
size_t sweep_smem_bytes(int nown, int nrhs, int maxrhs)
{
    using TM = sweep_math_t<TL>;
    return (size_t)maxrhs * BS * sizeof(double) + (size_t)maxrhs * (ystride<BS>() + BS) * sizeof(TM) +
           (size_t)BS * istride<TL, BS>() * sizeof(TM) + (size_t)sweep_slots<TL, BS>() * lstride<BS>() * sizeof(TL) +
           (size_t)nown * BS * nrhs * sizeof(double);
}

// One sweep.  FWD: Y = L^-1 B.  BWD: Y = L^-T B.  Y (n x nrhs, ldy) gets
// the solved blocks.  nrhs <= 16.
//
// CTA `me` owns blocks me, me + P, ... and keeps their partial sums in
// shared memory.  Per step J every CTA first starts copying into shared
// memory the blocks of L it will need (staged so that entry k * 65 + t
// multiplies y_J[k] for item t of the owned block: row t of L_IJ forward,
// column t of L_JI back), plus, for the owner of the next block, that
// block's inverse and right-hand side; then it waits for block J.  Each
// (item, rhs) sum of 64 terms is split over four adjacent lanes and joined
// by two shuffles, so updates need no barrier of their own.  The owner of
// the next block updates, solves and publishes it before its other updates,
// so the serial chain per block is: y_J seen -> one 64 x 64 block product
// -> one 64 x 64 inverse-block product -> publish.
//
// Publishing.  FP32 factor: each solved value goes out as one 64-bit word,
// its FP32 value in the low half and the sweep's tag in the high half, so
// a reader polls the words themselves and needs no flag, fence or second
// read (the products use the FP32 value; Y gets the FP64 one).  FP64
// factor: Y is written, then flags[J] = tag with release semantics; readers
// acquire the flag and read Y.
template <typename TL, bool FWD, int BS>
__global__ void __launch_bounds__(SW_THREADS) trsv_sweep_kernel(int64_t n, int nrhs, const TL *__restrict__ L,
                                                                int64_t ldl, const sweep_math_t<TL> *__restrict__ Linv,
                                                                const double *B, int64_t ldb, double *Y, int64_t ldy,
                                                                unsigned *flags, unsigned long long *tagw,
                                                                unsigned tag, int *err, int maxrhs)
{
    using TM = sweep_math_t<TL>;
    constexpr bool TAGGED = sizeof(TL) == 4;
    constexpr int SLOTS = sweep_slots<TL, BS>();
    constexpr int PQ = padq<TL>();
    constexpr int IS = istride<TL, BS>();
    constexpr int LSTRIDE = lstride<BS>();   // one staged block
    constexpr int YSTRIDE = ystride<BS>();
    constexpr int QK = BS / 4;   // k-range of one of the four lanes of an item
    extern __shared__ __align__(16) double sw_smem[];
    double *bst = sw_smem;                                            // staged B rows of the next block
    TM *yv = reinterpret_cast<TM *>(bst + BS * maxrhs);               // solved block being applied
    TM *vv = yv + YSTRIDE * maxrhs;                                   // right-hand side of the block being solved
    TM *Li = vv + BS * maxrhs;                                        // inverse of the next block, (r, k) at r + k * IS
    TL *Ls = reinterpret_cast<TL *>(Li + BS * IS);                    // [SLOTS][LSTRIDE]
    double *acc = reinterpret_cast<double *>(Ls + SLOTS * LSTRIDE);   // [owned][BS * nrhs]
    __shared__ int abort_flag;
    const int tid = threadIdx.x;
    const int64_t N = (n + BS - 1) / BS;
    const int64_t P = gridDim.x, me = blockIdx.x;
    const int nown = (int)((N - me + P - 1) / P);
    if (tid == 0) abort_flag = 0;

    auto rows_of = [&](int64_t J) { return (int)((n - J * BS < BS) ? n - J * BS : BS); };
    auto own_index = [&](int64_t I) { return (int)((I - me) / P); };

    auto stage = [&](int slot, int64_t I, int64_t J) {
        const int nI = rows_of(I), nJ = rows_of(J);
        TL *dst = Ls + slot * LSTRIDE;
        for (int e = tid; e < BS * BS; e += SW_THREADS) {
            // walk the global block down its columns (coalesced)
            const int a = e % BS, b = e / BS;
            const int t = FWD ? a : b, k = FWD ? b : a;
            TL *d = dst + k * (BS + 1) + (k / QK) * PQ + t;
            const TL *src = FWD ? L + (I * BS + t) + (J * BS + k) * ldl : L + (J * BS + k) + (I * BS + t) * ldl;
            if (t < nI && k < nJ) cp_async_elem(d, src, (int)sizeof(TL));
            else *d = TL(0);
        }
    };
    // Both sweeps read the inverse block as Li[r + k * IS], the weight of
    // v[k] in item r: forward that is (L_JJ^-1)(r, k), back (L_JJ^-1)(k, r).
    auto stage_solve = [&](int64_t J) {
        const TM *src = Linv + J * BS * BS;
        for (int e = tid; e < BS * BS; e += SW_THREADS) {
            const int a = e % BS, b = e / BS;
            cp_async_elem(Li + (FWD ? a + b * IS : b + a * IS), src + e, (int)sizeof(TM));
        }
        const int nb = rows_of(J);
        for (int e = tid; e < BS * nrhs; e += SW_THREADS) {
            const int r = e % BS, c = e / BS;
            if (r < nb) cp_async_elem(bst + e, B + J * BS + r + c * ldb, 8);
            else bst[e] = 0.0;
        }
    };

    for (int e = tid; e < nown * BS * nrhs; e += SW_THREADS) acc[e] = 0.0;

    // Solve block J from vv (= B_J - partial sums); write and publish.
    auto finalize = [&](int64_t J) {
        const int nb = rows_of(J);
        const int p = tid & 3;
        for (int item = tid >> 2; item < BS * nrhs; item += SW_THREADS / 4) {
            const int r = item % BS, c = item / BS;
            TM s = 0;
            if (FWD) {
                for (int k = p; k <= r; k += 4) s = fma(Li[r + k * IS], vv[k + c * BS], s);
            } else {
                for (int k = r + ((p - r) & 3); k < BS; k += 4) s = fma(Li[r + k * IS], vv[k + c * BS], s);
            }
            s += __shfl_xor_sync(0xffffffffu, s, 1);
            s += __shfl_xor_sync(0xffffffffu, s, 2);
            if (p == 0) {
                if (r < nb) Y[J * BS + r + c * ldy] = (double)s;
                if constexpr (TAGGED)
                    st_relaxed_u64(tagw + J * BS * nrhs + item,
                                   ((unsigned long long)tag << 32) | __float_as_uint(r < nb ? (float)s : 0.0f));
            }
        }
        if constexpr (!TAGGED) {
            __threadfence();
            __syncthreads();
            if (tid == 0) st_release(&flags[J], tag);
        }
    };

    // Contribution of the solved block (in yv) to owned block I from the
    // staged block in `slot`.  critical: vv = B_I - (partial sums + it);
    // otherwise it is added to the partial sums.
    auto contribution = [&](int slot, int64_t I, bool critical) {
        const TL *Lb = Ls + slot * LSTRIDE;
        double *a = acc + (size_t)own_index(I) * BS * nrhs;
        const int nI = rows_of(I);
        const int q = tid & 3;
        for (int item = tid >> 2; item < BS * nrhs; item += SW_THREADS / 4) {
            const int t = item % BS, c = item / BS;
            TM s0 = 0, s1 = 0;
            const TM *y = yv + c * YSTRIDE + q * (QK + 1);
            const TL *l = Lb + (q * QK) * (BS + 1) + q * PQ + t;
#pragma unroll
            for (int k = 0; k < QK; k += 2) {
                s0 = fma((TM)l[k * (BS + 1)], y[k], s0);
                s1 = fma((TM)l[(k + 1) * (BS + 1)], y[k + 1], s1);
            }
            TM s = s0 + s1;
            s += __shfl_xor_sync(0xffffffffu, s, 1);
            s += __shfl_xor_sync(0xffffffffu, s, 2);
            if (q == 0) {
                if (critical) vv[item] = (t < nI) ? (TM)(bst[item] - (a[item] + (double)s)) : TM(0);
                else a[item] += (double)s;
            }
        }
    };

    // Wait for block J and load it into yv.  False: a wait gave up.
    auto receive = [&](int64_t J) {
        bool ok = true;
        if constexpr (TAGGED) {
            for (int e = tid; e < BS * nrhs && ok; e += SW_THREADS) {
                const unsigned long long *w = tagw + J * BS * nrhs + e;
                unsigned long long v = ld_relaxed_u64(w);
                for (uint32_t it = 0; (unsigned)(v >> 32) != tag; ++it) {
                    if (it >= FLAG_SPIN_LIMIT) {
                        ok = false;
                        break;
                    }
                    if (it > 4096) __nanosleep(64);
                    v = ld_relaxed_u64(w);
                }
                const int r = e % BS, c = e / BS;
                yv[c * YSTRIDE + (r / QK) * (QK + 1) + r % QK] = __uint_as_float((unsigned)v);
            }
            if (!ok) {
                abort_flag = 1;
                atomicExch(err, 1);
            }
            return ok;
        } else {
            if (J % P != me && tid == 0) {
                ok = false;
                for (uint32_t it = 0; it < FLAG_SPIN_LIMIT; ++it) {
                    if (ld_acquire(&flags[J]) == tag) {
                        ok = true;
                        break;
                    }
                    if (it > 4096) __nanosleep(64);
                }
                if (!ok) {
                    abort_flag = 1;
                    atomicExch(err, 1);
                }
            }
            __syncthreads();
            if (abort_flag) return false;
            for (int e = tid; e < BS * nrhs; e += SW_THREADS) {
                const int r = e % BS, c = e / BS;
                yv[c * YSTRIDE + (r / QK) * (QK + 1) + r % QK] =
                    (r < rows_of(J)) ? __ldcg(&Y[J * BS + r + c * ldy]) : 0.0;
            }
            return true;
        }
    };

    __syncthreads();
    const int64_t first = FWD ? 0 : N - 1;
    if (first % P == me) {
        stage_solve(first);
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();
        if (abort_flag) return;
        for (int e = tid; e < BS * nrhs; e += SW_THREADS) vv[e] = (TM)bst[e];
        __syncthreads();
        finalize(first);
        __syncthreads();
    }
    for (int64_t s = 0; s < N; ++s) {
        const int64_t J = FWD ? s : N - 1 - s;
        const int64_t next = FWD ? J + 1 : J - 1;
        const bool own_next = next >= 0 && next < N && next % P == me;
        int64_t cur = next;
        if (!own_next) {
            if (FWD) {
                cur = me;
                if (cur <= J) cur += ((J - cur) / P + 1) * P;
            } else {
                cur = me + ((N - 1 - me) / P) * P;
                while (cur >= J && cur >= 0) cur -= P;
            }
        }
        auto in_range = [&](int64_t I) { return FWD ? (I > J && I < N) : (I < J && I >= 0); };
        int staged = 0;
        int64_t chunk[SLOTS];
        while (staged < SLOTS && in_range(cur)) {
            chunk[staged] = cur;
            stage(staged, cur, J);
            ++staged;
            cur = FWD ? cur + P : cur - P;
        }
        if (own_next) stage_solve(next);
        cp_async_commit();
        receive(J);
        cp_async_wait_all();
        __syncthreads();
        if (abort_flag) return;
        for (int q = 0; q < staged; ++q) {
            const bool crit = (q == 0 && own_next);
            contribution(q, chunk[q], crit);
            if (crit) {
                __syncthreads();
                finalize(next);
            }
        }
        // owned blocks beyond the first chunk
        while (in_range(cur)) {
            __syncthreads();
            int cnt = 0;
            while (cnt < SLOTS && in_range(cur)) {
                chunk[cnt] = cur;
                stage(cnt, cur, J);
                ++cnt;
                cur = FWD ? cur + P : cur - P;
            }
            cp_async_commit();
            cp_async_wait_all();
            __syncthreads();
            if (abort_flag) return;
            for (int q = 0; q < cnt; ++q) contribution(q, chunk[q], false);
        }
        __syncthreads();
    }
}

// The preconditioner's sweeps: FP32 factor, 128-row blocks, one or two
// right-hand sides.  FWD: Y = L^-1 B.  BWD: Y = L^-T B.  One cooperative
// launch of one CTA per SM; CTA `me` owns blocks me, me + P, ... and keeps
// their partial sums (FP64) in shared memory.  With the coupling blocks of
// couple_kernel the forward recurrence is
//   y_{I} = c_I - F_I y_{I-1},  c_I = inv(L_II) (B_I - sum_{K < I-1} L_IK y_K),
// and the back one x_I = c_I - G_I^T x_{I+1} with c_I = inv(L_II)^T (Y_I -
// sum_{K > I+1} L_KI^T x_K).  The owner of block I computes c_I as soon as
// the contribution of block I -2 (I + 2 back) is in its partial sums, one
// step before block I-1 (I + 1) arrives, so the serial chain per block is:
// block seen -> one 128 x 128 block product -> publish.
//
// Per step J every CTA with owned blocks past J copies the blocks of L it
// needs by TMA (the owner of the next block copies F_next or G_next
// instead of its block of L; the owner of the block after that also its
// inverse block and right-hand side), waits for block J, and adds L_IJ y_J
// (L_JI^T x_J) to its partial sums.  Each (item, rhs) sum of 128 terms is
// split over four adjacent lanes (k = q, q + 4, ...) and joined by two
// shuffles.  Solved values are published as 64-bit words, the FP32 value
// in the low half and the sweep's tag in the high half, which readers poll
// (bounded) directly; Y gets the FP64 value.  Tiles are padded to 136
// (forward) or 132 (back) rows in shared memory so that the four lanes of
// an item and the eight items of a warp fall in different banks.
constexpr int S128_THREADS = 512;
constexpr int S128_BS = 128;
template <bool FWD>
constexpr int s128_pad()
{
    return FWD ? 136 : 132;
}
template <bool FWD>
size_t s128_smem_bytes(int nown, int nrhs)
{
    const size_t tile = (size_t)s128_pad<FWD>() * S128_BS * sizeof(float);
    return 128 + 3 * tile + 2 * S128_BS * sizeof(double) + (2 * 2 * 4 * 36 + 2 * S128_BS) * sizeof(float) +
           (size_t)nown * S128_BS * nrhs * sizeof(double);
}

template <bool FWD>
__global__ void __launch_bounds__(S128_THREADS, 1) trsv_sweep128_kernel(
    int64_t n, int nrhs, const double *B, int64_t ldb, double *Y, int64_t ldy, unsigned long long *tagw,
    unsigned tag, int *err, const __grid_constant__ CUtensorMap tmL, const __grid_constant__ CUtensorMap tmI,
    const __grid_constant__ CUtensorMap tmC)
{
    constexpr int BS = S128_BS, TP = s128_pad<FWD>(), TILE = TP * BS, SLOTS = 2, NT = S128_THREADS;
    constexpr int VS = 4 * 36;   // per-rhs stride of a permuted vector
    constexpr uint32_t TILE_BYTES = TILE * sizeof(float);
    extern __shared__ __align__(16) double s128_raw[];
    float *Ls = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(s128_raw) + 127) & ~uintptr_t(127));
    float *Li = Ls + SLOTS * TILE;                        // inverse block: (r, k) of the forward map at r + k TP
    double *bst = reinterpret_cast<double *>(Li + TILE);  // staged right-hand side [2][BS]
    // vectors multiplied by a tile are stored permuted: row r of rhs c at
    // c VS + (r % 4) 36 + r / 4, so that the lane taking k = q, q + 4, ...
    // reads its 32 values as eight 16-byte words, the four lanes of an
    // item in different banks
    float *yv = reinterpret_cast<float *>(bst + 2 * BS);  // received block (permuted)
    float *vv = yv + 2 * VS;                              // c of the block this CTA solves next [rhs][BS]
    float *wv = vv + 2 * BS;                              // B - partial sums, while c is computed (permuted)
    double *acc = reinterpret_cast<double *>(wv + 2 * VS);
    __shared__ int abort_flag;
    __shared__ __align__(8) uint64_t tbar, cbar;   // copies of a step; the coupling block in Li
    uint32_t tphase = 0, cphase = 0;
    const int tid = threadIdx.x, q = tid & 3;
    const int64_t N = (n + BS - 1) / BS, P = gridDim.x, me = blockIdx.x;
    const int nown = (int)((N - me + P - 1) / P);
    const int nit = BS * nrhs;
    if (tid == 0) {
        abort_flag = 0;
        gpch::tc::mbar_init(&tbar, 1);
        gpch::tc::mbar_init(&cbar, 1);
        gpch::tc::fence_mbar_init();
    }
    for (int e = tid; e < nown * nit; e += NT) acc[e] = 0.0;

    auto rows_of = [&](int64_t J) { return (int)((n - J * BS < BS) ? n - J * BS : BS); };
    auto own_index = [&](int64_t I) { return (int)((I - me) / P); };
    auto valid = [&](int64_t I) { return I >= 0 && I < N; };
    auto stepI = [&](int64_t I) { return FWD ? I + P : I - P; };
    // this CTA's first block past J in sweep order (possibly invalid)
    auto first_after = [&](int64_t J64) {
        // 32-bit arithmetic: N < 2^24
        const int J = (int)J64, p = (int)P, m = (int)me, nb = (int)N;
        int I;
        if (FWD) {
            I = m;
            if (I <= J) I += ((J - I) / p + 1) * p;
        } else {
            I = m + ((nb - 1 - m) / p) * p;
            while (I >= J && I >= 0) I -= p;
        }
        return (int64_t)I;
    };
    // TMA copies (thread 0): block (I, J) of L forward, (J, I) back; the
    // coupling block of I; the inverse block of I
    auto load_tile = [&](int slot, int64_t I, int64_t J) {
        gpch::tc::tma_load_2d(Ls + slot * TILE, &tmL, &tbar, (int32_t)((FWD ? I : J) * BS),
                              (int32_t)((FWD ? J : I) * BS));
    };
    auto abort_now = [&]() {
        abort_flag = 1;
        atomicExch(err, 1);
    };
    auto wait_batch = [&]() {
        const bool ok = gpch::tc::mbar_wait(&tbar, tphase, FLAG_SPIN_LIMIT);
        tphase ^= 1u;
        if (!ok) abort_now();
    };
    // after c_I is in vv (and a barrier): block I's coupling block into Li
    auto load_coupling = [&](int64_t I) {
        if (tid == 32) {
            gpch::tc::mbar_arrive_expect_tx(&cbar, TILE_BYTES);
            gpch::tc::tma_load_2d(Li, &tmC, &cbar, (int32_t)(I * BS), 0);
        }
    };
    auto perm = [](int r) { return (r & 3) * 36 + (r >> 2); };
    auto stage_rhs = [&](int64_t I) {
        const int nb = rows_of(I);
        for (int e = tid; e < nit; e += NT) {
            const int r = e % BS, c = e / BS;
            if (r < nb) cp_async_elem(bst + e, B + I * BS + r + c * ldb, 8);
            else bst[e] = 0.0;
        }
        cp_async_commit();
    };
    auto publish = [&](int64_t J, int item, float s) {
        const int r = item % BS, c = item / BS;
        const bool in = r < rows_of(J);
        st_relaxed_u64(tagw + J * BS * nrhs + item,
                       ((unsigned long long)tag << 32) | __float_as_uint(in ? s : 0.0f));
        if (in) Y[J * BS + r + c * ldy] = (double)s;
    };
    // sum over k of M(t, k) v[k] for one item, this lane's k = q + 4j:
    // forward M(t, k) at t + k TP, back M(k, t) at k + t TP
    auto dot = [&](const float *M, int t, const float *v) {
        const float *m = FWD ? M + t + q * TP : M + t * TP + q;
        constexpr int KS = FWD ? 4 * TP : 4;
        const float4 *x = reinterpret_cast<const float4 *>(v + q * 36);   // v[q + 4j] at x[j / 4]
        float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
#pragma unroll
        for (int j = 0; j < BS / 4; j += 4) {
            const float4 xv = x[j / 4];
            s0 = fmaf(m[j * KS], xv.x, s0);
            s1 = fmaf(m[(j + 1) * KS], xv.y, s1);
            s2 = fmaf(m[(j + 2) * KS], xv.z, s2);
            s3 = fmaf(m[(j + 3) * KS], xv.w, s3);
        }
        float s = (s0 + s1) + (s2 + s3);
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        return s;
    };
    // c_I = inv(L_II) (B_I - partial sums) into vv (or, pub, publish it as
    // block I's solution); Li and bst hold block I's inverse and B rows
    auto prep_c = [&](int64_t I, bool pub) {
        const double *a = acc + (size_t)own_index(I) * nit;
        const int nb = rows_of(I);
        for (int e = tid; e < nit; e += NT)
            wv[(e / BS) * VS + perm(e % BS)] = (e % BS < nb) ? (float)(bst[e] - a[e]) : 0.0f;
        __syncthreads();
        for (int item = tid >> 2; item < nit; item += NT / 4) {
            const int r = item % BS, c = item / BS;
            // the inverse is triangular with zeros staged above (below) the
            // diagonal, so the full sum is the triangular one; the forward
            // sweep reads (r, k) at r + k TP, the back one (k, r) at k + r TP
            const float s = dot(Li, r, wv + c * VS);
            if (q == 0) {
                if (pub) publish(I, item, s);
                else vv[item] = s;
            }
        }
    };
    // block J's contribution to owned block I from the tile in `slot`
    auto contribution = [&](int slot, int64_t I, bool) {
        const float *M = Ls + slot * TILE;
        double *a = acc + (size_t)own_index(I) * nit;
        for (int item = tid >> 2; item < nit; item += NT / 4) {
            const int t = item % BS, c = item / BS;
            const float s = dot(M, t, yv + c * VS);
            if (q == 0) a[item] += (double)s;
        }
    };
    // Wait for block J (bounded) and load it into yv.  Warp 0 alone polls,
    // every lane keeping all of its words' loads in flight at once.  A CTA
    // that is not about to solve a block (urgent false) first has one lane
    // watch the block's last word with sleeps in between, so that the
    // lines the two urgent CTAs poll are not crowded by every other CTA.
    auto receive = [&](int64_t J, bool urgent) {
        if (tid >= 32) return;
        constexpr int MAXW = 2 * BS / 32;   // words per lane, two right-hand sides
        const int nw = nit / 32;
        const unsigned long long *w = tagw + J * BS * nrhs + tid;
        unsigned pending = (1u << nw) - 1u;
        bool ok = true;
        if (!urgent) {
            // one lane watches the block's last word first
            if (tid == 0) {
                const unsigned long long *last = tagw + J * BS * nrhs + (nit - 1);
                for (uint32_t it = 0; (unsigned)(ld_relaxed_u64(last) >> 32) != tag; ++it) {
                    if (it >= FLAG_SPIN_LIMIT) {
                        ok = false;
                        break;
                    }
                    __nanosleep(256);
                }
            }
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok) pending = 0;
        }
        for (uint32_t it = 0; pending != 0; ++it) {
            if (it >= FLAG_SPIN_LIMIT) {
                ok = false;
                break;
            }
            if (it > 4096) __nanosleep(64);
            unsigned long long v[MAXW];
#pragma unroll
            for (int k = 0; k < MAXW; ++k)
                if (pending & (1u << k)) v[k] = ld_relaxed_u64(w + 32 * k);
#pragma unroll
            for (int k = 0; k < MAXW; ++k) {
                if ((pending & (1u << k)) && (unsigned)(v[k] >> 32) == tag) {
                    const int e = tid + 32 * k;
                    yv[(e / BS) * VS + perm(e % BS)] = __uint_as_float((unsigned)v[k]);
                    pending &= ~(1u << k);
                }
            }
        }
        if (!ok) abort_now();
    };

    __syncthreads();
    // the first block, and c of the second (with its coupling block)
    const int64_t first = FWD ? 0 : N - 1, second = FWD ? 1 : N - 2;
    for (int pass = 0; pass < 2; ++pass) {
        const int64_t I = pass == 0 ? first : second;
        if (!valid(I) || I % P != me) continue;
        stage_rhs(I);
        if (tid == 32) {
            gpch::tc::mbar_arrive_expect_tx(&tbar, TILE_BYTES);
            gpch::tc::tma_load_2d(Li, &tmI, &tbar, 0, (int32_t)(I * BS));
        }
        cp_async_wait_all();
        wait_batch();
        __syncthreads();
        if (abort_flag) return;
        prep_c(I, pass == 0);
        __syncthreads();
        if (pass == 1) load_coupling(I);
    }
    for (int64_t s = 0; s < N; ++s) {
        const int64_t J = FWD ? s : N - 1 - s;
        const int64_t next = FWD ? J + 1 : J - 1, nn = FWD ? J + 2 : J - 2, n3 = FWD ? J + 3 : J - 3;
        const bool own_next = valid(next) && (int)next % (int)P == (int)me;
        const bool own_nn = valid(nn) && (int)nn % (int)P == (int)me;
        int64_t cur = first_after(J);
        if (!valid(cur)) continue;   // nothing of this CTA's depends on block J any more
        // the next block (when owned) is solved from its coupling block,
        // already in Li; the other owned blocks take tiles of L
        if (own_next) cur = stepI(cur);
        int staged = 0;
        int64_t chunk[SLOTS];
        while (staged < SLOTS && valid(cur)) {
            chunk[staged++] = cur;
            cur = stepI(cur);
        }
        if (own_nn) stage_rhs(nn);
        const bool batch = staged > 0 || own_nn;
        // the copies of a step (the critical CTA's only after it has
        // published: they would delay its polls)
        auto issue = [&]() {
            if (tid != 32) return;
            if (batch) {
                gpch::tc::mbar_arrive_expect_tx(&tbar, (uint32_t)(staged + (own_nn ? 1 : 0)) * TILE_BYTES);
                for (int i = 0; i < staged; ++i) load_tile(i, chunk[i], J);
                if (own_nn) gpch::tc::tma_load_2d(Li, &tmI, &tbar, 0, (int32_t)(nn * BS));
            }
            // into L2 now, what this CTA copies at the next step
            if (valid(next)) {
                int64_t I = first_after(next);
                for (int i = 0; i < SLOTS && valid(I); ++i, I = stepI(I)) {
                    if (I == nn) gpch::tc::tma_prefetch_2d(&tmC, (int32_t)(nn * BS), 0);
                    else gpch::tc::tma_prefetch_2d(&tmL, (int32_t)((FWD ? I : next) * BS),
                                                   (int32_t)((FWD ? next : I) * BS));
                }
                if (valid(n3) && (int)n3 % (int)P == (int)me) gpch::tc::tma_prefetch_2d(&tmI, 0, (int32_t)(n3 * BS));
            }
        };
        if (!own_next) issue();   // warp 0 polls meanwhile
        // the critical step: block next = c - (coupling block) block J, the
        // coupling block taken into registers (this thread's 32 entries of
        // row t = (tid / 4) % 128, k = q + 4j) before block J arrives
        float mreg[BS / 4];
        if (own_next) {
            const bool ok = gpch::tc::mbar_wait(&cbar, cphase, FLAG_SPIN_LIMIT);
            cphase ^= 1u;
            if (!ok) abort_now();
            const int t = (tid >> 2) % BS;
            const float *m = FWD ? Li + t + q * TP : Li + t * TP + q;
#pragma unroll
            for (int j = 0; j < BS / 4; ++j) mreg[j] = m[j * (FWD ? 4 * TP : 4)];
        }
        receive(J, own_next || own_nn);
        if (own_next) {
            __syncthreads();
            if (abort_flag) return;
            const int nI = rows_of(next);
            for (int item = tid >> 2; item < nit; item += NT / 4) {
                const int t = item % BS, c = item / BS;
                const float4 *x = reinterpret_cast<const float4 *>(yv + c * VS + q * 36);
                float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
#pragma unroll
                for (int j = 0; j < BS / 4; j += 4) {
                    const float4 xv = x[j / 4];
                    s0 = fmaf(mreg[j], xv.x, s0);
                    s1 = fmaf(mreg[j + 1], xv.y, s1);
                    s2 = fmaf(mreg[j + 2], xv.z, s2);
                    s3 = fmaf(mreg[j + 3], xv.w, s3);
                }
                float v = (s0 + s1) + (s2 + s3);
                v += __shfl_xor_sync(0xffffffffu, v, 1);
                v += __shfl_xor_sync(0xffffffffu, v, 2);
                if (q == 0) publish(next, item, (t < nI) ? vv[item] - v : 0.0f);
            }
            issue();
        }
        if (own_nn) cp_async_wait_all();
        if (batch) wait_batch();
        __syncthreads();
        if (abort_flag) return;
        for (int i = 0; i < staged; ++i) {
            contribution(i, chunk[i], false);
            if (own_nn && chunk[i] == nn) {
                __syncthreads();
                prep_c(nn, false);
                __syncthreads();
                load_coupling(nn);
            }
        }
        // owned blocks beyond the first batch
        while (valid(cur)) {
            __syncthreads();
            int cnt = 0;
            while (cnt < SLOTS && valid(cur)) {
                chunk[cnt++] = cur;
                cur = stepI(cur);
            }
            if (tid == 32) {
                gpch::tc::mbar_arrive_expect_tx(&tbar, (uint32_t)cnt * TILE_BYTES);
                for (int i = 0; i < cnt; ++i) load_tile(i, chunk[i], J);
            }
            wait_batch();
            __syncthreads();
            if (abort_flag) return;
            for (int i = 0; i < cnt; ++i) contribution(i, chunk[i], false);
        }
        __syncthreads();
    }
}

// SM count of the context's device: it sizes the cooperative sweeps' grids,
// which must fit on the device they run on.  Asked for on every launch
// (a cheap attribute query), so devices of different sizes and contexts on
// several host threads each get their own value.
int sm_count(gpch_ctx *ctx)
{
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess || v <= 0) {
        cudaGetLastError();
        v = 1;
    }
    return v;
}

template <typename TL, bool FWD, int BS>
gpch_status launch_sweep(gpch_ctx *ctx, int64_t n, int nrhs, const TL *L, int64_t ldl, const double *Linv_ws,
                         const double *B, int64_t ldb, double *Y, int64_t ldy, unsigned *flags,
                         unsigned long long *tagw, unsigned tag, int *err, cudaStream_t st)
{
    const sweep_math_t<TL> *Linv = reinterpret_cast<const sweep_math_t<TL> *>(Linv_ws);
    const int64_t N = (n + BS - 1) / BS;
    const int P = (int)(N < sm_count(ctx) ? N : sm_count(ctx));
    const int nown = (int)((N + P - 1) / P);
    const int maxrhs = SW_MAXRHS;
    const size_t smem = sweep_smem_bytes<TL, BS>(nown, nrhs, maxrhs);
    int maxsmem = 0;
    GPCH_CUDA(ctx, cudaDeviceGetAttribute(&maxsmem, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
    if (smem + 1024 > (size_t)maxsmem)
        return gpch::fail(ctx, GPCH_INVALID_ARG, "substitution sweep: n * nrhs too large for shared memory");
    {
        // Raised once per device to the largest size any launch may ask for:
        // the needed size varies with n and nrhs, and contexts on other host
        // threads launch this kernel concurrently.
        static std::mutex mu;
        static bool done[64] = {};
        std::lock_guard<std::mutex> lock(mu);
        if (ctx->device >= 64 || !done[ctx->device]) {
            GPCH_CUDA(ctx, cudaFuncSetAttribute(trsv_sweep_kernel<TL, FWD, BS>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, maxsmem - 1024));
            if (ctx->device < 64) done[ctx->device] = true;
        }
    }
    int maxrhs_arg = maxrhs;
    void *args[] = {&n, &nrhs, &L, &ldl, &Linv, &B, &ldb, &Y, &ldy, &flags, &tagw, &tag, &err, &maxrhs_arg};
    GPCH_CUDA(ctx, cudaLaunchCooperativeKernel((const void *)trsv_sweep_kernel<TL, FWD, BS>, dim3(P), dim3(SW_THREADS),
                                               args, smem, st));
    GPCH_LAUNCH_CHECK(ctx);
    return GPCH_OK;
}


// One sweep of trsv_sweep128_kernel: L (FP32, n x n, ld ldl, 16-byte
// aligned), the 128 x 128 inverse blocks Linv128 and the coupling blocks
// Cpl (F128 forward, G128 back).
template <bool FWD>
gpch_status launch_sweep128(gpch_ctx *ctx, int64_t n, int nrhs, const float *L, int64_t ldl, const float *Linv128,
                            const float *Cpl, const double *B, int64_t ldb, double *Y, int64_t ldy,
                            unsigned long long *tagw, unsigned tag, int *err, cudaStream_t st)
{
    constexpr int BS = S128_BS;
    const int64_t N = (n + BS - 1) / BS;
    const int P = (int)(N < sm_count(ctx) ? N : sm_count(ctx));
    const int nown = (int)((N + P - 1) / P);
    const size_t smem = s128_smem_bytes<FWD>(nown, nrhs);
    auto enc = gpch::tc::tmap_encoder();
    if (!enc) return gpch::fail(ctx, GPCH_CUDA_ERROR, "cuTensorMapEncodeTiled not available");
    CUtensorMap tmL, tmI, tmC;
    // boxes of TP rows x BS columns; rows past a map's end read as zeros
    const cuuint32_t box[2] = {(cuuint32_t)s128_pad<FWD>(), (cuuint32_t)BS};
    const cuuint32_t estr[2] = {1, 1};
    auto encode = [&](CUtensorMap *m, const float *base, cuuint64_t rows, cuuint64_t cols, cuuint64_t ld) {
        const cuuint64_t dims[2] = {rows, cols};
        const cuuint64_t strides[1] = {ld * sizeof(float)};
        return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    };
    if (encode(&tmL, L, (cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)ldl) != CUDA_SUCCESS ||
        encode(&tmI, Linv128, BS, (cuuint64_t)(N * BS), BS) != CUDA_SUCCESS ||
        encode(&tmC, Cpl, (cuuint64_t)(N * BS), BS, (cuuint64_t)(N * BS)) != CUDA_SUCCESS)
        return gpch::fail(ctx, GPCH_CUDA_ERROR, "tensor maps of the substitution sweep failed");
    int maxsmem = 0;
    GPCH_CUDA(ctx, cudaDeviceGetAttribute(&maxsmem, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
    if (smem + 1024 > (size_t)maxsmem)
        return gpch::fail(ctx, GPCH_INVALID_ARG, "substitution sweep: n * nrhs too large for shared memory");
    static gpch::DeviceOnce attr_once;
    GPCH_CHECK(gpch::once_per_device(ctx, attr_once, [&]() -> gpch_status {
        GPCH_CUDA(ctx, cudaFuncSetAttribute(trsv_sweep128_kernel<FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            maxsmem - 1024));
        return GPCH_OK;
    }));
    void *args[] = {&n, &nrhs, &B, &ldb, &Y, &ldy, &tagw, &tag, &err, &tmL, &tmI, &tmC};
    GPCH_CUDA(ctx, cudaLaunchCooperativeKernel((const void *)trsv_sweep128_kernel<FWD>, dim3(P), dim3(S128_THREADS),
                                               args, smem, st));
    GPCH_LAUNCH_CHECK(ctx);
    return GPCH_OK;
}
}  // namespace

namespace gpch {

size_t solve_ws_bytes(int64_t n, int nrhs)
{
    Carver dry(nullptr);
    const int64_t N = (n + LEAF - 1) / LEAF;
    dry.take<double>((size_t)N * LEAF * LEAF);
    dry.take<double>((size_t)n * (nrhs < SW_MAXRHS ? nrhs : SW_MAXRHS));
    dry.take<unsigned>((size_t)2 * N);
    dry.take<unsigned long long>((size_t)(N + 1) * LEAF * (nrhs < SW_MAXRHS ? nrhs : SW_MAXRHS));
    dry.take<float>((size_t)((n + 127) / 128) * 128 * 128);
    dry.take<float>((size_t)((n + 127) / 128) * 128 * 128);
    dry.take<float>((size_t)((n + 127) / 128) * 128 * 128);
    dry.take<int>(4);
    return dry.off;
}

SolveWs carve_solve(void *base, int64_t n, int nrhs)
{
    Carver cv(base);
    const int64_t N = (n + LEAF - 1) / LEAF;
    SolveWs w;
    w.Linv = cv.take<double>((size_t)N * LEAF * LEAF);
    w.Y = cv.take<double>((size_t)n * (nrhs < SW_MAXRHS ? nrhs : SW_MAXRHS));
    w.flags = cv.take<unsigned>((size_t)2 * N);
    w.tagw_words = (size_t)(N + 1) * LEAF * (nrhs < SW_MAXRHS ? nrhs : SW_MAXRHS);
    w.tagw = cv.take<unsigned long long>(w.tagw_words);
    w.Linv128 = cv.take<float>((size_t)((n + 127) / 128) * 128 * 128);
    w.F128 = cv.take<float>((size_t)((n + 127) / 128) * 128 * 128);
    w.G128 = cv.take<float>((size_t)((n + 127) / 128) * 128 * 128);
    w.err = cv.take<int>(4);
    w.epoch = 0;
    return w;
}

// Invert the diagonal blocks of L and clear the flags (once per factor).
template <typename TL>
gpch_status solve_prepare_t(gpch_ctx *ctx, int64_t n, const TL *L, int64_t ldl, SolveWs &w, cudaStream_t st)
{
    const int64_t N = (n + LEAF - 1) / LEAF;
    constexpr size_t INV_SMEM = 2 * LEAF * (LEAF + 1) * sizeof(double);
    static gpch::DeviceOnce attr_once;
    GPCH_CHECK(gpch::once_per_device(ctx, attr_once, [&]() -> gpch_status {
        GPCH_CUDA(ctx, cudaFuncSetAttribute(inv_diag_blocks_kernel<TL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)INV_SMEM));
        return GPCH_OK;
    }));
    inv_diag_blocks_kernel<TL>
        <<<(unsigned)N, 256, INV_SMEM, st>>>(n, L, ldl, reinterpret_cast<sweep_math_t<TL> *>(w.Linv));
    GPCH_LAUNCH_CHECK(ctx);
    if (sizeof(TL) == 4) {
        inv128_kernel<<<(unsigned)((n + 127) / 128), 256, 0, st>>>(
            n, reinterpret_cast<const float *>(L), ldl, reinterpret_cast<const float *>(w.Linv), w.Linv128);
        GPCH_LAUNCH_CHECK(ctx);
        couple_kernel<<<dim3((unsigned)((n + 127) / 128), 2), 256, 0, st>>>(n, reinterpret_cast<const float *>(L),
                                                                           ldl, w.Linv128, w.F128, w.G128);
        GPCH_LAUNCH_CHECK(ctx);
    }
    GPCH_CUDA(ctx, cudaMemsetAsync(w.flags, 0, 2 * N * sizeof(unsigned), st));
    GPCH_CUDA(ctx, cudaMemsetAsync(w.tagw, 0, w.tagw_words * sizeof(unsigned long long), st));
    GPCH_CUDA(ctx, cudaMemsetAsync(w.err, 0, 4 * sizeof(int), st));
    w.epoch = 0;
    return GPCH_OK;
}

// B <- (L L^T)^-1 B, in place, after solve_prepare.
template <typename TL>
gpch_status solve_apply_t(gpch_ctx *ctx, int64_t n, const TL *L, int64_t ldl, double *B, int64_t ldb, int nrhs,
                          SolveWs &w, cudaStream_t st)
{
    const int64_t N = (n + LEAF - 1) / LEAF;
    PhaseScope ph(ctx, GPCH_PHASE_SOLVE, st, 2.0 * (double)n * n * nrhs);
    // FP32 factor, one or two right-hand sides: 128-row blocks when their
    // shared memory fits
    // (the TMA copies of that variant need a 16-byte aligned L and ldl)
    if constexpr (sizeof(TL) == 4) {
        if (nrhs <= 2 && (uintptr_t)L % 16 == 0 && (ldl * sizeof(TL)) % 16 == 0) {
            const int64_t N2 = (n + 127) / 128;
            const int P2 = (int)(N2 < sm_count(ctx) ? N2 : sm_count(ctx));
            const int nown2 = (int)((N2 + P2 - 1) / P2);
            int maxsmem = 0;
            GPCH_CUDA(ctx, cudaDeviceGetAttribute(&maxsmem, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
            if (s128_smem_bytes<true>(nown2, nrhs) + 1024 <= (size_t)maxsmem) {
                ++w.epoch;
                GPCH_CHECK(launch_sweep128<true>(ctx, n, nrhs, L, ldl, w.Linv128, w.F128, B, ldb, w.Y, n, w.tagw,
                                                 2 * w.epoch, w.err, st));
                GPCH_CHECK(launch_sweep128<false>(ctx, n, nrhs, L, ldl, w.Linv128, w.G128, w.Y, n, B, ldb, w.tagw,
                                                  2 * w.epoch + 1, w.err, st));
                return GPCH_OK;
            }
        }
    }
    // right-hand sides per sweep: at most 16, fewer if the owned blocks'
    // partial sums would not fit in shared memory
    const int P = (int)(N < sm_count(ctx) ? N : sm_count(ctx));
    const int nown = (int)((N + P - 1) / P);
    int gmax = SW_MAXRHS;
    while (gmax > 1 && sweep_smem_bytes<TL, 64>(nown, gmax, SW_MAXRHS) > 200 * 1024) gmax /= 2;
    for (int c0 = 0; c0 < nrhs; c0 += gmax) {
        const int g = (nrhs - c0 < gmax) ? nrhs - c0 : gmax;
        double *Bc = B + (int64_t)c0 * ldb;
        // tags 2e (forward) and 2e + 1 (back) of epoch e >= 1 never match
        // the cleared words or an earlier sweep's
        ++w.epoch;
        GPCH_CHECK((launch_sweep<TL, true, 64>(ctx, n, g, L, ldl, w.Linv, Bc, ldb, w.Y, n, w.flags, w.tagw,
                                               2 * w.epoch, w.err, st)));
        GPCH_CHECK((launch_sweep<TL, false, 64>(ctx, n, g, L, ldl, w.Linv, w.Y, n, Bc, ldb, w.flags + N, w.tagw,
                                                2 * w.epoch + 1, w.err, st)));
    }
    return GPCH_OK;
}

gpch_status solve_prepare(gpch_ctx *ctx, int64_t n, const double *L, int64_t ldl, SolveWs &w, cudaStream_t st)
{
    return solve_prepare_t<double>(ctx, n, L, ldl, w, st);
}
gpch_status solve_prepare_f32(gpch_ctx *ctx, int64_t n, const float *L, int64_t ldl, SolveWs &w, cudaStream_t st)
{
    return solve_prepare_t<float>(ctx, n, L, ldl, w, st);
}
gpch_status solve_apply(gpch_ctx *ctx, int64_t n, const double *L, int64_t ldl, double *B, int64_t ldb, int nrhs,
                        SolveWs &w, cudaStream_t st)
{
    return solve_apply_t<double>(ctx, n, L, ldl, B, ldb, nrhs, w, st);
}
gpch_status solve_apply_f32(gpch_ctx *ctx, int64_t n, const float *L, int64_t ldl, double *B, int64_t ldb, int nrhs,
                            SolveWs &w, cudaStream_t st)
{
    return solve_apply_t<float>(ctx, n, L, ldl, B, ldb, nrhs, w, st);
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
    cudaStream_t st = (cudaStream_t)stream;
    GPCH_CHECK(gpch::ws_reserve(ctx, gpch::solve_ws_bytes(n, nrhs)));
    gpch::SolveWs w = gpch::carve_solve(ctx->ws, n, nrhs);
    GPCH_CHECK(gpch::solve_prepare(ctx, n, L, ldl, w, st));
    GPCH_CHECK(gpch::solve_apply(ctx, n, L, ldl, B, ldb, nrhs, w, st));
    int *h = static_cast<int *>(ctx->pinned);
    GPCH_CUDA(ctx, cudaMemcpyAsync(h, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    GPCH_CUDA(ctx, cudaStreamSynchronize(st));
    if (*h != 0) return gpch::fail(ctx, GPCH_TIMEOUT, "substitution sweep wait gave up");
    return GPCH_OK;
}

extern "C" gpch_status gpch_chol_solve_f32(gpch_ctx *ctx, int64_t n, const float *L, int64_t ldl, double *B,
                                           int64_t ldb, int nrhs, void *stream)
{
    GPCH_ARG(ctx, ctx != nullptr, "null context");
    GPCH_ARG(ctx, n >= 0 && nrhs >= 0, "n < 0 or nrhs < 0");
    GPCH_ARG(ctx, ldl >= (n > 0 ? n : 1) && ldb >= (n > 0 ? n : 1), "ldl or ldb < n");
    if (n == 0 || nrhs == 0) return GPCH_OK;
    GPCH_ARG(ctx, L != nullptr && B != nullptr, "null pointer");
    GPCH_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    GPCH_CHECK(gpch::ws_reserve(ctx, gpch::solve_ws_bytes(n, nrhs)));
    gpch::SolveWs w = gpch::carve_solve(ctx->ws, n, nrhs);
    GPCH_CHECK(gpch::solve_prepare_f32(ctx, n, L, ldl, w, st));
    GPCH_CHECK(gpch::solve_apply_f32(ctx, n, L, ldl, B, ldb, nrhs, w, st));
    int *h = static_cast<int *>(ctx->pinned);
    GPCH_CUDA(ctx, cudaMemcpyAsync(h, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    GPCH_CUDA(ctx, cudaStreamSynchronize(st));
    if (*h != 0) return gpch::fail(ctx, GPCH_TIMEOUT, "substitution sweep wait gave up");
    return GPCH_OK;
}
