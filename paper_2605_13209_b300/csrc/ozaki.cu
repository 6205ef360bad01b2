// ozaki.cu -- FP64-accurate products on the bf16 tensor cores (an
// error-free splitting in the manner of the Ozaki scheme): C -= A B^T for
// FP64 A (m x k) and B (n x k), the operation of Algorithm 1 step 3 and of
// any FP64 GEMM, at a rate set by the tensor cores instead of this part's
// FP64 pipe (2 FMAs per clock per SM).
//
// Splitting.  Row r of A is scaled by 2^(54 - e_r), e_r the smallest
// integer with |A_rc| < 2^e_r for the whole row, and rounded to the integer
// N_rc (|N_rc| <= 2^54); N_rc is written as 8 balanced base-128 digits,
// N = sum_p d_p 128^(7-p) with d_p in [-64, 63] (the top digit within
// [-33, 33]).  Every digit is exact in bf16.  B's rows likewise with f_j.
// Then A_rc B_jc ~= 2^(e_r + f_j - 108) sum_{p,q} d_p d'_q 128^(14-p-q).
//
// Products.  The digit pairs with p + q = D <= 7 (36 of 64) are kept; the
// dropped ones weigh at most about 2^-49 of the row scales' product per
// term.  Each digit product is at most 2^12 in magnitude and a weight class
// D holds at most 8 pairs, so over k <= 512 every class sum S_D is an
// integer of magnitude at most 2^24: the FP32 tensor-core accumulation of
// bf16 products is exact.  The 8 class sums live in 8 TMEM accumulators
// (all 512 columns of an SM's TMEM for a 128 x 64 tile).
//
// Combination.  T = sum_D S_D 2^(7(7-D)) is formed exactly as
// H 2^28 + L with H = sum_{D<4} S_D 2^(7(3-D)) and L = sum_{D>=4} S_D
// 2^(7(7-D)) (each below 2^47) in 128-bit integer arithmetic, rounded once
// to the FP64 value of 2^(e_r + f_j - 59) T with integer operations, and
// subtracted from C in FP64 (one FP64 operation per entry: this part's FP64
// pipe is slow).
// Longer k is done in passes of at most 512 columns, each rounded once.
//
// Accuracy.  Per entry the error is at most about
// k 2^-48 2^(e_r + f_j) (splitting and dropped pairs) plus one FP64
// rounding per pass: the size of FP64 GEMM's own worst-case bound
// (k u |A||B|) when the row's largest entries set its scale.
#include <cuda_bf16.h>

#include "internal.cuh"
#include "ozaki.cuh"
#include "tc_ptx.cuh"

namespace {

using gpch::oz_map;
using gpch::oz_pos;
using gpch::oz_round_scaled;

constexpr int OZ_DIGITS = 8;          // base-128 digits per entry
constexpr int OZ_CLASSES = 8;         // weight classes D = p + q kept (0..7)
constexpr int OZ_KMAX = 512;          // k per exact pass
constexpr int OZ_BM = 128, OZ_BN = 64;
constexpr int OZ_KSTAGE = 32;         // K columns per pipeline stage
constexpr int OZ_BOXES = OZ_DIGITS / 2;                 // two digits per 128-byte box row
constexpr uint32_t OZ_ABOX = OZ_BM * 128;               // bytes of one A box (128 rows x 128 B)
constexpr uint32_t OZ_BBOX = OZ_BN * 128;               // bytes of one B box
constexpr uint32_t OZ_STAGE = OZ_BOXES * (OZ_ABOX + OZ_BBOX);   // 96 KB
constexpr int OZ_STAGES = 2;
constexpr int OZ_THREADS = 192;       // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
constexpr uint32_t OZ_TMEM_COLS = OZ_CLASSES * OZ_BN;   // 512
constexpr uint32_t OZ_SPIN = 1u << 26;
constexpr size_t OZ_SMEM = OZ_STAGES * OZ_STAGE + 1024 + 256;

// Digits of the rows of X (rows x k, ld ldx) into D: row r's digits of box b
// at row b * rows + r of a (4 rows) x (2 kp) bf16 array (kp = k rounded up
// to 32; columns past k are zero), and the row exponent e_r into E.  One
// warp per row.
__global__ void __launch_bounds__(256) oz_split_kernel(int64_t rows, int k, int kp, const double *__restrict__ X,
                                                       int64_t ldx, __nv_bfloat16 *__restrict__ D,
                                                       int *__restrict__ E)
{
    const int lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (r >= rows) return;
    const double *x = X + r;
    double mx = 0.0;
    for (int c = lane; c < k; c += 32) mx = fmax(mx, fabs(x[(int64_t)c * ldx]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    // e: smallest integer with every |x| < 2^e (a zero row gets e = 0)
    int e = 0;
    if (mx > 0.0) {
        int ex;
        frexp(mx, &ex);   // mx = f 2^ex, f in [0.5, 1): mx < 2^ex
        e = ex;
    }
    if (lane == 0) E[r] = e;
    const int64_t ld = 2 * (int64_t)kp;
    for (int c = lane; c < kp; c += 32) {
        // N = round(x 2^(54 - e)) from the bit pattern (integer operations)
        long long N = 0;
        if (c < k) {
            const unsigned long long bits = (unsigned long long)__double_as_longlong(x[(int64_t)c * ldx]);
            const int E11 = (int)((bits >> 52) & 0x7ff);
            unsigned long long mant = bits & 0xfffffffffffffull;
            int ebits = E11;
            if (E11 == 0) ebits = 1;
            else mant |= 1ull << 52;
            // x = mant 2^(ebits - 1075); shift to 2^(54 - e) units
            const int s = ebits - 1075 + 54 - e;
            unsigned long long a;
            if (s >= 0) a = mant << s;                     // s <= 1: |x| < 2^e
            else if (s > -64) a = (mant + (1ull << (-s - 1))) >> (-s);
            else a = 0;
            N = (bits >> 63) ? -(long long)a : (long long)a;
        }
        // balanced base-128 digits, least significant first
#pragma unroll
        for (int p = OZ_DIGITS - 1; p >= 0; --p) {
            long long d;
            if (p > 0) {
                d = ((N + 64) & 127) - 64;
                N = (N - d) >> 7;
            } else {
                d = N;   // |N| <= 2^54 / 128^7 + 1 = 33
            }
            D[(int64_t)(p / 2) * rows * ld + r * ld + oz_pos(p, c)] = __float2bfloat16_rn((float)d);
        }
    }
}

}  // namespace

namespace {

// C[m x n] -= A B^T for one 128 x 64 output tile per CTA, from the digit
// copies of A (tensor map tm_a over a (4 m) x (2 kp) bf16 array) and of B
// (tm_b, (4 n) x (2 kp)) and the row exponents ea, eb; kp <= 512, a
// multiple of 32.  lower: only entries with row >= column are written
// (C square); the grid then lists only tiles that hold such entries.
// Roles: warp 0 lane 0 issues the TMA loads (2 stages of 4 + 4 boxes), warp
// 1 owns the TMEM (all 512 columns: 8 class accumulators of 64 columns) and
// its lane 0 issues the MMAs, warps 2-5 combine the class sums (warp w:
// tile rows 32 (w % 4) .. +31, its TMEM lanes).  err: device status word,
// nonzero if a bounded wait gave up.
__global__ void __launch_bounds__(OZ_THREADS, 1)
    oz_gemm_kernel(const __grid_constant__ CUtensorMap tm_a, const __grid_constant__ CUtensorMap tm_b, int64_t m,
                   int64_t n, int kp, const int *__restrict__ ea, const int *__restrict__ eb, double *C, int64_t ldc,
                   int lower, int64_t tiles_n, int *err)
{
    extern __shared__ __align__(1024) uint8_t oz_smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(oz_smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + OZ_STAGES * OZ_STAGE);
    uint64_t *empty = full + OZ_STAGES;
    uint64_t *tfull = empty + OZ_STAGES;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tfull + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // tile (ti, tj): a rectangle lists row tiles x column tiles; the lower
    // case lists, row tile by row tile, the column tiles 0 .. (2 ti + 1)
    // that touch the triangle (a 128-row tile spans two 64-column tiles)
    int64_t ti, tj;
    const int64_t t = blockIdx.x;
    if (!lower) {
        ti = t / tiles_n;
        tj = t % tiles_n;
    } else {
        // row tile ti holds min(2 ti + 2, tiles_n) tiles; find ti by search
        int64_t lo = 0, hi = (m + OZ_BM - 1) / OZ_BM - 1;
        auto before = [&](int64_t r) {   // tiles in row tiles 0 .. r-1
            const int64_t full_rows = (tiles_n / 2 < r) ? tiles_n / 2 : r;   // rows with 2r+2 <= tiles_n
            return full_rows * (full_rows + 1) + (r - full_rows) * tiles_n;
        };
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) / 2;
            if (before(mid) <= t) lo = mid;
            else hi = mid - 1;
        }
        ti = lo;
        tj = t - before(ti);
    }
    const int64_t i0 = ti * OZ_BM, j0 = tj * OZ_BN;

    if (threadIdx.x == 0) {
        for (int s = 0; s < OZ_STAGES; ++s) {
            gpch::tc::mbar_init(&full[s], 1);
            gpch::tc::mbar_init(&empty[s], 1);
        }
        gpch::tc::mbar_init(tfull, 1);
        gpch::tc::fence_mbar_init();
    }
    if (warp == 1) gpch::tc::tmem_alloc<OZ_TMEM_COLS>(tmem_slot);
    gpch::tc::tc_fence_before();
    __syncthreads();
    gpch::tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int NK = kp / OZ_KSTAGE;

    if (warp == 0) {
        if (lane == 0) {
            gpch::tc::prefetch_tmap(&tm_a);
            gpch::tc::prefetch_tmap(&tm_b);
            int issued = 0;
            for (int kc = 0; kc < NK; ++kc) {
                const int s = kc % OZ_STAGES;
                if (kc >= OZ_STAGES && !gpch::tc::mbar_wait(&empty[s], ((kc / OZ_STAGES) - 1) & 1, OZ_SPIN)) {
                    atomicExch(err, 1);
                    break;
                }
                uint8_t *st = smem + s * OZ_STAGE;
                gpch::tc::mbar_arrive_expect_tx(&full[s], OZ_STAGE);
                const int32_t x = (int32_t)(kc * 2 * OZ_KSTAGE);
                for (int b = 0; b < OZ_BOXES; ++b) {
                    gpch::tc::tma_load_2d(st + b * OZ_ABOX, &tm_a, &full[s], x, (int32_t)(b * m + i0));
                    gpch::tc::tma_load_2d(st + OZ_BOXES * OZ_ABOX + b * OZ_BBOX, &tm_b, &full[s], x,
                                          (int32_t)(b * n + j0));
                }
                ++issued;
            }
            for (int s = 0; s < OZ_STAGES && s < issued; ++s) {
                const int uses = (issued - 1 - s) / OZ_STAGES + 1;
                if (!gpch::tc::mbar_wait(&full[s], (uses - 1) & 1, OZ_SPIN)) atomicExch(err, 4);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = gpch::tc::idesc_bf16_f32(OZ_BM, OZ_BN);
            bool ok = true;
            for (int kc = 0; kc < NK && ok; ++kc) {
                const int s = kc % OZ_STAGES;
                if (!gpch::tc::mbar_wait(&full[s], (kc / OZ_STAGES) & 1, OZ_SPIN)) {
                    atomicExch(err, 2);
                    ok = false;
                    break;
                }
                gpch::tc::tc_fence_after();
                const uint32_t sa = gpch::tc::smem_u32(smem + s * OZ_STAGE);
                const uint32_t sb = sa + OZ_BOXES * OZ_ABOX;
#pragma unroll
                for (int p = 0; p < OZ_DIGITS; ++p) {
                    const uint64_t a = gpch::tc::sdesc_sw128(sa + (p / 2) * OZ_ABOX) + 4 * (p & 1);
#pragma unroll
                    for (int q = 0; q + p < OZ_CLASSES; ++q) {
                        const uint64_t b = gpch::tc::sdesc_sw128(sb + (q / 2) * OZ_BBOX) + 4 * (q & 1);
                        const uint32_t acc = tmem + (uint32_t)((p + q) * OZ_BN);
                        // the first product into a class accumulator (p = 0
                        // starts every class) overwrites it
#pragma unroll
                        for (int k = 0; k < 2; ++k)
                            gpch::tc::mma_bf16(acc, a + 2 * k, b + 2 * k, idesc,
                                               (kc > 0 || k > 0 || p > 0) ? 1u : 0u);
                    }
                }
                gpch::tc::mma_commit(&empty[s]);
            }
            if (ok) gpch::tc::mma_commit(tfull);
        }
        __syncwarp();
    } else {
        // Epilogue: lane l of warp w holds tile row 32 (w % 4) + l.
        const int qw = warp & 3;
        const int64_t row = i0 + qw * 32 + lane;
        const bool row_ok = row < m;
        // while the MMAs run: the tile's column exponents into shared
        // memory, and its C lines (a warp's 32 rows of a column are one
        // 256-byte piece) into L2
        __shared__ int s_eb[OZ_BN];
        if (warp == 2)
            for (int j = lane; j < OZ_BN; j += 32) s_eb[j] = (j0 + j < n) ? eb[j0 + j] : 0;
        if (row_ok)
            for (int j = 0; j < OZ_BN; ++j)
                if (j0 + j < n && !(lower && j0 + j > row))
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(C + row + (j0 + j) * ldc));
        asm volatile("bar.sync 1, 128;" ::: "memory");   // the four epilogue warps
        bool ok = gpch::tc::mbar_wait(tfull, 0, 4 * OZ_SPIN);
        ok = __all_sync(0xffffffffu, ok);
        gpch::tc::tc_fence_after();
        if (!ok) {
            if (lane == 0) atomicExch(err, 3);
        } else {
            const int er = row_ok ? ea[row] : 0;
            const uint32_t tl = tmem + ((uint32_t)(qw * 32) << 16);
#pragma unroll 1
            for (int cc = 0; cc < OZ_BN / 16; ++cc) {
                uint32_t vr[OZ_CLASSES][16];
#pragma unroll
                for (int D = 0; D < OZ_CLASSES; ++D) gpch::tc::tmem_ld16_nowait(tl + D * OZ_BN + cc * 16, vr[D]);
                gpch::tc::tmem_ld_wait();
                // the chunk's C entries, all loads in flight together
                double cval[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int64_t col = j0 + cc * 16 + j;
                    const bool want = row_ok && col < n && !(lower && col > row);
                    cval[j] = want ? C[row + col * ldc] : 0.0;
                }
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int64_t col = j0 + cc * 16 + j;
                    if (!row_ok || col >= n || (lower && col > row)) continue;
                    // exact class sums (integers of magnitude <= 2^24)
                    long long H = 0, L = 0;
#pragma unroll
                    for (int D = 0; D < 4; ++D) H = H * 128 + __float2int_rn(__uint_as_float(vr[D][j]));
#pragma unroll
                    for (int D = 4; D < 8; ++D) L = L * 128 + __float2int_rn(__uint_as_float(vr[D][j]));
                    // one rounding of the product, then C's
                    C[row + col * ldc] = cval[j] - oz_round_scaled(H, L, er + s_eb[cc * 16 + j] - 59);
                }
            }
        }
    }
    gpch::tc::tc_fence_before();
    __syncthreads();
    if (warp == 1) gpch::tc::tmem_dealloc<OZ_TMEM_COLS>(tmem);
}

}  // namespace

namespace {

// Tiles of the lower case: row tile r holds min(2 r + 2, tiles_n) column tiles.
int64_t oz_lower_tiles(int64_t row_tiles, int64_t tiles_n)
{
    const int64_t F = (tiles_n / 2 < row_tiles) ? tiles_n / 2 : row_tiles;
    return F * (F + 1) + (row_tiles - F) * tiles_n;
}

}  // namespace

namespace gpch {

// Workspace bytes of oz_gemm_enqueue for m x k and n x k operands (k per
// pass <= 512): digit copies of A (and B unless it is A), exponents, the
// status word.
size_t oz_ws_bytes(int64_t m, int64_t n, bool same)
{
    gpch::Carver dry(nullptr);
    dry.take<int>(1);
    dry.take<__nv_bfloat16>((size_t)4 * m * 2 * OZ_KMAX);
    if (!same) dry.take<__nv_bfloat16>((size_t)4 * n * 2 * OZ_KMAX);
    dry.take<int>((size_t)m);
    if (!same) dry.take<int>((size_t)n);
    return dry.off;
}

// C[m x n] -= A B^T (lower: the lower triangle of the square C only) with
// FP64-accurate products on the tensor cores, in passes of at most 512
// K columns, on `ws` (oz_ws_bytes(m, n, B == A) bytes, 256-byte aligned).
// err_out: the device status word (nonzero after a bounded wait gave up),
// cleared here when *err_out is nullptr on entry.
gpch_status oz_gemm_enqueue(gpch_ctx *ctx, int64_t m, int64_t n, int64_t k, const double *A, int64_t lda,
                            const double *B, int64_t ldb, double *C, int64_t ldc, bool lower, void *ws,
                            cudaStream_t st, int **err_out)
{
    const bool same = (A == B && lda == ldb && m == n);
    gpch::Carver cv(ws);
    // the status word first: at the same place for every call on this
    // workspace, whatever the sizes (a caller's later calls keep it)
    int *err = cv.take<int>(1);
    __nv_bfloat16 *dA = cv.take<__nv_bfloat16>((size_t)4 * m * 2 * OZ_KMAX);
    __nv_bfloat16 *dB = same ? dA : cv.take<__nv_bfloat16>((size_t)4 * n * 2 * OZ_KMAX);
    int *ea = cv.take<int>((size_t)m);
    int *eb = same ? ea : cv.take<int>((size_t)n);
    if (*err_out == nullptr) GPCH_CUDA(ctx, cudaMemsetAsync(err, 0, sizeof(int), st));
    *err_out = err;
    if (m == 0 || n == 0 || k == 0) return GPCH_OK;
    static gpch::DeviceOnce attr_once;
    GPCH_CHECK(gpch::once_per_device(ctx, attr_once, [&]() -> gpch_status {
        GPCH_CUDA(ctx, cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OZ_SMEM));
        return GPCH_OK;
    }));
    const int64_t row_tiles = (m + OZ_BM - 1) / OZ_BM, tiles_n = (n + OZ_BN - 1) / OZ_BN;
    const int64_t tiles = lower ? oz_lower_tiles(row_tiles, tiles_n) : row_tiles * tiles_n;
    GPCH_ARG(ctx, tiles < (int64_t)0x7fffffff && 4 * (m > n ? m : n) < (int64_t)0x7fffffff, "matrix too large");
    for (int64_t k0 = 0; k0 < k; k0 += OZ_KMAX) {
        const int kk = (int)((k - k0 < OZ_KMAX) ? k - k0 : OZ_KMAX);
        const int kp = (kk + OZ_KSTAGE - 1) / OZ_KSTAGE * OZ_KSTAGE;
        oz_split_kernel<<<(unsigned)((m + 7) / 8), 256, 0, st>>>(m, kk, kp, A + k0 * lda, lda, dA, ea);
        GPCH_LAUNCH_CHECK(ctx);
        if (!same) {
            oz_split_kernel<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(n, kk, kp, B + k0 * ldb, ldb, dB, eb);
            GPCH_LAUNCH_CHECK(ctx);
        }
        CUtensorMap ma, mb;
        GPCH_CHECK(oz_map(ctx, &ma, dA, 4 * m, 2 * (int64_t)kp, OZ_BM));
        GPCH_CHECK(oz_map(ctx, &mb, dB, 4 * n, 2 * (int64_t)kp, OZ_BN));
        oz_gemm_kernel<<<(unsigned)tiles, OZ_THREADS, OZ_SMEM, st>>>(ma, mb, m, n, kp, ea, eb, C, ldc, lower ? 1 : 0,
                                                                     tiles_n, err);
        GPCH_LAUNCH_CHECK(ctx);
    }
    return GPCH_OK;
}

}  // namespace gpch

extern "C" gpch_status gpch_gemm_fp64_emulated(gpch_ctx *ctx, int64_t m, int64_t n, int64_t k, const double *A,
                                               int64_t lda, const double *B, int64_t ldb, double *C, int64_t ldc,
                                               int lower, void *stream)
{
    GPCH_ARG(ctx, ctx != nullptr, "null context");
    GPCH_ARG(ctx, m >= 0 && n >= 0 && k >= 0, "negative size");
    GPCH_ARG(ctx, !lower || m == n, "lower needs a square C");
    GPCH_ARG(ctx, lda >= (m > 0 ? m : 1) && ldb >= (n > 0 ? n : 1) && ldc >= (m > 0 ? m : 1), "ld too small");
    if (m == 0 || n == 0 || k == 0) return GPCH_OK;
    GPCH_ARG(ctx, A && B && C, "null pointer");
    GPCH_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    GPCH_CHECK(gpch::ws_reserve(ctx, gpch::oz_ws_bytes(m, n, A == B && lda == ldb && m == n)));
    int *err = nullptr;
    GPCH_CHECK(gpch::oz_gemm_enqueue(ctx, m, n, k, A, lda, B, ldb, C, ldc, lower != 0, ctx->ws, st, &err));
    int *h = static_cast<int *>(ctx->pinned);
    GPCH_CUDA(ctx, cudaMemcpyAsync(h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    GPCH_CUDA(ctx, cudaStreamSynchronize(st));
    if (*h != 0) return gpch::fail(ctx, GPCH_TIMEOUT, "tensor-core pipeline wait gave up (%d)", *h);
    return GPCH_OK;
}
