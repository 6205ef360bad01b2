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
#include <cstring>
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

// Sweep block size BS: 64 for every factor; 128 for an FP32 factor with at
// most two right-hand sides, which halves the serial steps of a sweep.
// Blocks of L staged per step: BS = 64: 4 (FP32) or 2 (FP64); BS = 128: 2.
template <typename TL, int BS>
constexpr int sweep_slots()
{
    return BS == 128 ? 2 : (sizeof(TL) == 4 ? 4 : 2);
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

// FP32 factor, 128-row blocks: the blocks of L and the inverse blocks are
// copied in by TMA as 2-D tiles whose inner (contiguous) extent is padded
// to 136 (forward) or 132 (back) rows, which spreads the four lanes that
// share an item over all banks.  Other variants stage element by element.
template <typename TL, int BS>
constexpr bool sweep_tma()
{
    return sizeof(TL) == 4 && BS == 128;
}
template <bool FWD>
constexpr int tma_pad()
{
    return FWD ? 136 : 132;
}

// Dynamic shared memory of one sweep CTA owning `nown` blocks.
template <typename TL, int BS, bool FWD = true>
size_t sweep_smem_bytes(int nown, int nrhs, int maxrhs)
{
    using TM = sweep_math_t<TL>;
    if (sweep_tma<TL, BS>()) {
        const int P = tma_pad<FWD>();
        return 128 + (size_t)sweep_slots<TL, BS>() * P * BS * sizeof(TL) + (size_t)P * BS * sizeof(TM) +
               (size_t)maxrhs * BS * sizeof(double) + (size_t)maxrhs * 2 * BS * sizeof(TM) +
               (size_t)nown * BS * nrhs * sizeof(double);
    }
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
                                                                unsigned tag, int *err, int maxrhs,
                                                                const __grid_constant__ CUtensorMap tmL,
                                                                const __grid_constant__ CUtensorMap tmI)
{
    using TM = sweep_math_t<TL>;
    constexpr bool TAGGED = sizeof(TL) == 4;
    constexpr bool TMAV = sweep_tma<TL, BS>();
    constexpr int SLOTS = sweep_slots<TL, BS>();
    constexpr int PQ = padq<TL>();
    constexpr int TP = tma_pad<FWD>();                       // TMA variant: padded inner extent
    constexpr int IS = TMAV ? TP : istride<TL, BS>();
    constexpr int LSTRIDE = TMAV ? TP * BS : lstride<BS>();   // one staged block
    constexpr int YSTRIDE = TMAV ? BS : ystride<BS>();
    constexpr int QK = BS / 4;   // k-range of one of the four lanes of an item (element-staged variants)
    extern __shared__ __align__(16) double sw_smem[];
    double *bst;   // staged B rows of the next block
    TM *yv, *vv, *Li;
    TL *Ls;
    double *acc;
    if constexpr (TMAV) {
        // the TMA destinations first, 128-byte aligned
        uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(sw_smem) + 127) & ~uintptr_t(127));
        Ls = reinterpret_cast<TL *>(base);                     // [SLOTS][TP * BS]: block (t, k) at
        Li = reinterpret_cast<TM *>(Ls + SLOTS * LSTRIDE);     //   t + k * TP (fwd) or k + t * TP (back)
        bst = reinterpret_cast<double *>(Li + TP * BS);        // inverse (r', k') at r' + k' * TP
        yv = reinterpret_cast<TM *>(bst + BS * maxrhs);
        vv = yv + BS * maxrhs;
        acc = reinterpret_cast<double *>(vv + BS * maxrhs);
    } else {
        bst = sw_smem;
        yv = reinterpret_cast<TM *>(bst + BS * maxrhs);            // solved block being applied
        vv = yv + YSTRIDE * maxrhs;                                // right-hand side of the block being solved
        Li = vv + BS * maxrhs;                                     // inverse of the next block, (r, k) at r + k * IS
        Ls = reinterpret_cast<TL *>(Li + BS * IS);                 // [SLOTS][LSTRIDE]
        acc = reinterpret_cast<double *>(Ls + SLOTS * LSTRIDE);    // [owned][64 * nrhs]
    }
    __shared__ int abort_flag;
    __shared__ __align__(8) uint64_t tbar;   // TMA variant: completion of a staging batch
    uint32_t tphase = 0;
    const int tid = threadIdx.x;
    const int64_t N = (n + BS - 1) / BS;
    const int64_t P = gridDim.x, me = blockIdx.x;
    const int nown = (int)((N - me + P - 1) / P);
    if (tid == 0) {
        abort_flag = 0;
        if constexpr (TMAV) {
            gpch::tc::mbar_init(&tbar, 1);
            gpch::tc::fence_mbar_init();
        }
    }

    auto rows_of = [&](int64_t J) { return (int)((n - J * BS < BS) ? n - J * BS : BS); };
    auto own_index = [&](int64_t I) { return (int)((I - me) / P); };

    // TMA variant: thread 0 issues the tile copies of a batch after
    // announcing its byte count; batch_wait() waits for all of them.
    auto tma_block = [&](int slot, int64_t I, int64_t J) {
        // forward: block (I, J) of L, x = rows of I; back: block (J, I), x = rows of J
        gpch::tc::tma_load_2d(Ls + slot * LSTRIDE, &tmL, &tbar, (int32_t)((FWD ? I : J) * BS),
                              (int32_t)((FWD ? J : I) * BS));
    };
    auto batch_wait = [&]() -> bool {
        const bool ok = gpch::tc::mbar_wait(&tbar, tphase, FLAG_SPIN_LIMIT);
        tphase ^= 1u;
        return ok;
    };
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
        if constexpr (!TMAV) {
            for (int e = tid; e < BS * BS; e += SW_THREADS) {
                const int a = e % BS, b = e / BS;
                cp_async_elem(Li + (FWD ? a + b * IS : b + a * IS), src + e, (int)sizeof(TM));
            }
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
            } else if constexpr (TMAV) {
                // the inverse block is staged untransposed: (L^-1)(k, r) at k + r * IS
                for (int k = r + ((p - r) & 3); k < BS; k += 4) s = fma(Li[k + r * IS], vv[k + c * BS], s);
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
            if constexpr (TMAV) {
                // lane q takes k = q, q + 4, ... (conflict-free with the padded tiles)
                const TM *y = yv + c * BS + q;
                const TL *l = FWD ? Lb + t + q * TP : Lb + t * TP + q;
                constexpr int KS = FWD ? 4 * TP : 4;   // step of k by 4
#pragma unroll 8
                for (int j = 0; j < BS / 4; j += 2) {
                    s0 = fma((TM)l[j * KS], y[4 * j], s0);
                    s1 = fma((TM)l[(j + 1) * KS], y[4 * j + 4], s1);
                }
            } else {
                const TM *y = yv + c * YSTRIDE + q * (QK + 1);
                const TL *l = Lb + (q * QK) * (BS + 1) + q * PQ + t;
#pragma unroll
                for (int k = 0; k < QK; k += 2) {
                    s0 = fma((TM)l[k * (BS + 1)], y[k], s0);
                    s1 = fma((TM)l[(k + 1) * (BS + 1)], y[k + 1], s1);
                }
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
                if constexpr (TMAV) yv[c * BS + r] = __uint_as_float((unsigned)v);
                else yv[c * YSTRIDE + (r / QK) * (QK + 1) + r % QK] = __uint_as_float((unsigned)v);
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

    // TMA variant: thread 0 announces the bytes of a batch of tile copies
    // (cnt blocks of L for step J, plus the inverse of block Jinv) and
    // issues them; every thread then waits with batch_wait().
    auto issue_batch = [&](int cnt, const int64_t *ch, int64_t J, bool with_inv, int64_t Jinv) {
        if constexpr (TMAV) {
            if (tid == 0) {
                const uint32_t bytes = (uint32_t)(cnt + (with_inv ? 1 : 0)) * (uint32_t)(TP * BS * sizeof(TL));
                gpch::tc::mbar_arrive_expect_tx(&tbar, bytes);
                for (int i = 0; i < cnt; ++i) tma_block(i, ch[i], J);
                if (with_inv) gpch::tc::tma_load_2d(Li, &tmI, &tbar, 0, (int32_t)(Jinv * BS));
            }
        }
    };
    __syncthreads();
    const int64_t first = FWD ? 0 : N - 1;
    if (first % P == me) {
        stage_solve(first);
        cp_async_commit();
        issue_batch(0, nullptr, 0, true, first);
        cp_async_wait_all();
        if constexpr (TMAV) {
            if (!batch_wait()) {
                abort_flag = 1;
                atomicExch(err, 1);
            }
        }
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
            if constexpr (!TMAV) stage(staged, cur, J);
            ++staged;
            cur = FWD ? cur + P : cur - P;
        }
        if (own_next) stage_solve(next);
        cp_async_commit();
        const bool batch = staged > 0 || own_next;
        if (batch) issue_batch(staged, chunk, J, own_next, next);
        if constexpr (TMAV) {
            // the tiles this CTA copies at the next step, into L2 now: its
            // blocks of step J' = next, and the inverse it solves with then
            const int64_t Jn = next, Jnn = FWD ? J + 2 : J - 2;
            if (tid == 0 && Jn >= 0 && Jn < N) {
                int64_t I = me;
                if (FWD) {
                    if (I <= Jn) I += ((Jn - I) / P + 1) * P;
                } else {
                    I = me + ((N - 1 - me) / P) * P;
                    while (I >= Jn && I >= 0) I -= P;
                }
                for (int q = 0; q < SLOTS && (FWD ? I < N : I >= 0); ++q, I = FWD ? I + P : I - P)
                    gpch::tc::tma_prefetch_2d(&tmL, (int32_t)((FWD ? I : Jn) * BS), (int32_t)((FWD ? Jn : I) * BS));
                if (Jnn >= 0 && Jnn < N && Jnn % P == me) gpch::tc::tma_prefetch_2d(&tmI, 0, (int32_t)(Jnn * BS));
            }
        }
        receive(J);
        cp_async_wait_all();
        if constexpr (TMAV) {
            if (batch && !batch_wait()) {
                abort_flag = 1;
                atomicExch(err, 1);
            }
        }
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
                if constexpr (!TMAV) stage(cnt, cur, J);
                ++cnt;
                cur = FWD ? cur + P : cur - P;
            }
            cp_async_commit();
            issue_batch(cnt, chunk, J, false, 0);
            cp_async_wait_all();
            if constexpr (TMAV) {
                if (!batch_wait()) {
                    abort_flag = 1;
                    atomicExch(err, 1);
                }
            }
            __syncthreads();
            if (abort_flag) return;
            for (int q = 0; q < cnt; ++q) contribution(q, chunk[q], false);
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
    const int maxrhs = BS == 128 ? 2 : SW_MAXRHS;
    const size_t smem = sweep_smem_bytes<TL, BS, FWD>(nown, nrhs, maxrhs);
    CUtensorMap tmL, tmI;
    memset(&tmL, 0, sizeof tmL);
    memset(&tmI, 0, sizeof tmI);
    if (sweep_tma<TL, BS>()) {
        // L as an n x n FP32 matrix (box: TP rows x BS columns), and the
        // inverse blocks as a BS x (N BS) matrix (box: TP x BS); rows past
        // the ends read as zeros
        auto enc = gpch::tc::tmap_encoder();
        if (!enc) return gpch::fail(ctx, GPCH_CUDA_ERROR, "cuTensorMapEncodeTiled not available");
        const cuuint32_t box[2] = {(cuuint32_t)tma_pad<FWD>(), (cuuint32_t)BS};
        const cuuint32_t estr[2] = {1, 1};
        const cuuint64_t dl[2] = {(cuuint64_t)n, (cuuint64_t)n};
        const cuuint64_t sl[1] = {(cuuint64_t)ldl * sizeof(TL)};
        CUresult r = enc(&tmL, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<TL *>(L), dl, sl, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return gpch::fail(ctx, GPCH_CUDA_ERROR, "tensor map of L failed (%d)", (int)r);
        const cuuint64_t di[2] = {(cuuint64_t)BS, (cuuint64_t)(N * BS)};
        const cuuint64_t si[1] = {(cuuint64_t)BS * sizeof(sweep_math_t<TL>)};
        r = enc(&tmI, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<sweep_math_t<TL> *>(Linv), di, si, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
            return gpch::fail(ctx, GPCH_CUDA_ERROR, "tensor map of the inverse blocks failed (%d)", (int)r);
    }
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
    void *args[] = {&n, &nrhs, &L, &ldl, &Linv, &B, &ldb, &Y, &ldy, &flags, &tagw, &tag, &err, &maxrhs_arg, &tmL, &tmI};
    GPCH_CUDA(ctx, cudaLaunchCooperativeKernel((const void *)trsv_sweep_kernel<TL, FWD, BS>, dim3(P), dim3(SW_THREADS),
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
    if (sizeof(TL) == 4 && nrhs <= 2 && (uintptr_t)L % 16 == 0 && (ldl * sizeof(TL)) % 16 == 0) {
        const int64_t N2 = (n + 127) / 128;
        const int P2 = (int)(N2 < sm_count(ctx) ? N2 : sm_count(ctx));
        const int nown2 = (int)((N2 + P2 - 1) / P2);
        int maxsmem = 0;
        GPCH_CUDA(ctx, cudaDeviceGetAttribute(&maxsmem, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
        if (sweep_smem_bytes<TL, 128>(nown2, nrhs, 2) + 1024 <= (size_t)maxsmem) {
            ++w.epoch;
            const double *Li = reinterpret_cast<const double *>(w.Linv128);
            GPCH_CHECK((launch_sweep<TL, true, 128>(ctx, n, nrhs, L, ldl, Li, B, ldb, w.Y, n, w.flags, w.tagw,
                                                    2 * w.epoch, w.err, st)));
            GPCH_CHECK((launch_sweep<TL, false, 128>(ctx, n, nrhs, L, ldl, Li, w.Y, n, B, ldb, w.flags + N, w.tagw,
                                                     2 * w.epoch + 1, w.err, st)));
            return GPCH_OK;
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
