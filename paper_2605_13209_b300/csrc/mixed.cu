// mixed.cu -- A8: the low-precision factor used as the preconditioner of the
// refined solve.  Algorithm 1 (right) runs on an FP32 copy of the lower
// triangle of A (+ shift * I):
//   step 1  the diagonal tile is factored in FP32, left-looking, one
//           launch per 32-column block (diag_step_kernel);
//   step 2  SPLIT_F16: the panel is the tensor-core product A_ij L_jj^-T,
//           with L_jj^-1 from an FP32 forward substitution; the bf16 modes
//           solve it in FP32, 64 columns at a time, against FP32 inverses
//           of the diagonal tile's 64 x 64 blocks;
//   step 3  the trailing update A_ik -= A_ij A_kj^T runs on the tensor cores:
//           the panel is rounded to 16 bits (or split into a head and a
//           tail) in a K-major copy, TMA streams 128 x 64 boxes of it into
//           shared memory, tcgen05.mma accumulates 128 x 128 FP32 tiles in
//           TMEM, and the epilogue subtracts them from the FP32 matrix.
// Mixed precision is the paper's stated future work (Sec. 5); the factor's
// accuracy is recovered by the FP64 refinement in cg.cu.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "dense_fp64.cuh"
#include "tc_ptx.cuh"

namespace {

using gpch::LEAF;

constexpr int BM = 128;            // rows of an output tile (TMEM lanes)
constexpr int BN = 128;            // columns of an output tile (TMEM columns)
constexpr int BK = 64;             // K granularity of the 16-bit panel copies (zero-padded to it)
constexpr int BOX_K = 64;          // 16-bit values per box row: one 128-byte swizzle row
constexpr int STAGES = 3;
constexpr int TC_THREADS = 192;   // warp 0: TMA, warp 1: MMA, warps 2-5: epilogue
constexpr uint32_t BOX_BYTES = BM * BOX_K * 2;   // one 128-row box (BM == BN)
constexpr uint32_t STAGE_BYTES = 2 * BOX_BYTES;  // row tile and column tile
constexpr size_t TC_SMEM = 1024 + STAGES * STAGE_BYTES + 256;
constexpr uint32_t SPIN_LIMIT = 1u << 22;
constexpr uint32_t TMEM_COLS = 2 * BN;   // accumulator + running sum (two CTAs fill an SM's TMEM)

// Layout of the 16-bit panel copies.  A copy is K-major: row r holds the
// K columns of panel row r.  With one product (BF16) K column c sits at
// position c of the row.  Split copies interleave head and tail in chunks
// of 32 columns: the head of column c at (c / 32) * 64 + c % 32 and its tail
// 32 positions later, so that one 128-byte box row carries the head and the
// tail of 32 columns and a single TMA box feeds all three products.  Row
// strides are multiples of 64 positions; column offsets used are multiples
// of 32 (their position is 2c).
__host__ __device__ constexpr int64_t kpos(bool split, int64_t c) { return split ? 2 * c : c; }

// Trailing update C_lower -= P P^T on tensor cores.  P is the m x kp panel,
// a 16-bit copy described by tm_a (rows of the copy; K positions from
// kpos(k_off), k_off a multiple of 64).  split = 0: one product
// head*head^T; split = 1: head*head^T + head*tail^T + tail*head^T.  Only
// columns below ncol are written.
//
// The K range is a sequence of panels of panel_k columns (panel_k divides
// kp).  Each panel's product is summed on its own in the TMEM accumulator
// (the tensor-core sums stay one panel long), and the epilogue adds it in
// FP32, rounding to nearest, into a running sum kept in a second TMEM
// region; the last panel's sum is subtracted from C.  The result is that
// of subtracting the panels one by one (up to the order of the FP32
// additions) while C is read and written once per launch instead of once
// per panel.  The accumulator is released as soon as the epilogue has read
// it, so the next panel's MMAs wait only for that read.  Roles: warp 0
// lane 0 issues the TMA loads, warp 1 lane 0 the MMAs (warp 1 owns the
// TMEM allocation), warps 2-5 run the epilogue (warp w: tile rows
// 32 (w % 4) .. +31, its TMEM lanes).  One CTA per lower 128 x 128 tile of
// C.  A pipeline stage holds one 128 x 64 box of the row tile's copy and
// one of the column tile's (a diagonal tile loads its rows once): 32 K
// columns (head and tail) when split, 64 otherwise.  err: device status
// word, nonzero if a bounded wait gave up.
//
// MODE 0 is the update above.  MODE 1 is the product C = P Q^T
// (overwrite), MODE 2 the update C -= P Q^T, both over a rectangle of
// split-f16 operands: P (rows of tm_a) is m x kp, Q (rows of tm_b) is
// ncol x kp, every tile of the m x ncol rectangle (tile columns tk0 .. tk1-1)
// is computed, and the operands carry the scales 2^scale[1] (P) and
// 2^scale_b[1] (Q).  MODE 0 reads both operands through tm_a (tm_b is not
// used).  With ohi != nullptr (MODE 1 only) the result is also written as
// a split-f16 copy scaled by 2^oscale[1]: row r, column c at position
// kpos(true, c) of ohi + r * ldo (the copy the later updates read; ohi and
// ldo must make every row 16-byte aligned).
// A second MODE 0 update in the same launch (first_tiles > 0): CTAs from
// first_tiles on take the lower trapezoid of another block column, with its
// own C, m, ncol, K range (kp positions from k_off) and operand copy (tm_b,
// which MODE 0 does not otherwise read), so that a short pass and a long
// pass share one grid.
struct SyrkSecond {
    float *C;
    int64_t m, ncol;
    int64_t first_tiles;
    int kp, k_off;
};

template <int MODE>
__global__ void __maxnreg__(112)
    syrk_tc_kernel(const __grid_constant__ CUtensorMap tm_a, const __grid_constant__ CUtensorMap tm_b, int64_t m,
                   int kp, int split, float *__restrict__ C, int64_t ldc, int64_t tk0, int64_t tk1, int *err,
                   int prefetch_c, int f16, const int *scale, int k_off, int64_t ncol, int panel_k,
                   const int *scale_b, __half *ohi, int64_t ldo, const int *oscale, SyrkSecond sp)
{
    constexpr bool rect = MODE != 0;   // rectangle of P Q^T
    constexpr bool sub = MODE != 1;    // C -= (else C = )
    extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~uintptr_t(1023));
    // stage s: the row tile's box at smem + s * STAGE_BYTES, the column
    // tile's BOX_BYTES after it
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *tfull = empty + STAGES;
    uint64_t *tempty = tfull + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tempty + 2);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Tiles of the lower triangle of the T x T tile grid restricted to tile
    // columns [tk0, tk1), row by row with the column varying fastest, so the
    // CTAs that read the same rows of P run at the same time and share them
    // through L2.  Rows tk0 .. tk1-2 hold 1, 2, ..., nc-1 tiles (the
    // triangle), every later row nc = tk1 - tk0 tiles.
    const bool second = MODE == 0 && sp.first_tiles > 0 && (int64_t)blockIdx.x >= sp.first_tiles;
    if (second) {
        C = sp.C;
        m = sp.m;
        ncol = sp.ncol;
        kp = sp.kp;
        k_off = sp.k_off;
    }
    const CUtensorMap *tma = second ? &tm_b : &tm_a;   // the operand copy of this CTA's update
    const int64_t nc = tk1 - tk0, tri = nc * (nc - 1) / 2;
    const int64_t t = second ? (int64_t)blockIdx.x - sp.first_tiles : (int64_t)blockIdx.x;
    int64_t ti, tk;
    if constexpr (rect) {
        ti = t / nc;
        tk = tk0 + t % nc;
    } else if (t < tri) {
        int64_t r = (int64_t)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
        while (r * (r + 1) / 2 > t) --r;
        while ((r + 1) * (r + 2) / 2 <= t) ++r;
        ti = tk0 + r;
        tk = tk0 + (t - r * (r + 1) / 2);
    } else {
        ti = tk1 - 1 + (t - tri) / nc;
        tk = tk0 + (t - tri) % nc;
    }
    const int64_t i0 = ti * BM, c0 = tk * BN;
    // a diagonal tile of the triangle multiplies its rows by themselves:
    // they are loaded once and serve as both operands
    const bool diag = !rect && ti == tk;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            gpch::tc::mbar_init(&full[s], 1);
            gpch::tc::mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            gpch::tc::mbar_init(&tfull[a], 1);
            gpch::tc::mbar_init(&tempty[a], 4);
        }
        gpch::tc::fence_mbar_init();
    }
    if (warp == 1) gpch::tc::tmem_alloc<TMEM_COLS>(tmem_slot);
    gpch::tc::tc_fence_before();
    __syncthreads();
    gpch::tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int kstage = split ? BOX_K / 2 : BOX_K;   // K columns per stage
    const int spp = panel_k / kstage;            // stages per panel
    const int np = kp / panel_k;                 // panels
    const int NK = np * spp;                     // stages, panel by panel

    if (warp == 0) {
        if (lane == 0) {
            // TMA producer
            gpch::tc::prefetch_tmap(tma);
            if constexpr (rect) gpch::tc::prefetch_tmap(&tm_b);
            const CUtensorMap *mb = rect ? &tm_b : tma;
            const uint32_t bytes = diag ? BOX_BYTES : STAGE_BYTES;
            int issued = 0;
            for (int kc = 0; kc < NK; ++kc) {
                const int s = kc % STAGES;
                if (kc >= STAGES && !gpch::tc::mbar_wait(&empty[s], ((kc / STAGES) - 1) & 1, SPIN_LIMIT)) {
                    atomicExch(err, 1);
                    break;
                }
                const int32_t x = (int32_t)kpos(split, k_off + (kc / spp) * panel_k + (kc % spp) * kstage);
                uint8_t *st = smem + s * STAGE_BYTES;
                gpch::tc::mbar_arrive_expect_tx(&full[s], bytes);
                gpch::tc::tma_load_2d(st, tma, &full[s], x, (int32_t)i0);
                if (!diag) gpch::tc::tma_load_2d(st + BOX_BYTES, mb, &full[s], x, (int32_t)c0);
                ++issued;
            }
            // Every copy this thread started has landed before the CTA may
            // exit (immediate in normal operation: the MMAs consumed them).
            for (int s = 0; s < STAGES && s < issued; ++s) {
                const int uses = (issued - 1 - s) / STAGES + 1;
                if (!gpch::tc::mbar_wait(&full[s], (uses - 1) & 1, SPIN_LIMIT)) atomicExch(err, 4);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer: panel p accumulates into the accumulator once the
            // epilogue has read panel p - 1 out of it
            const uint32_t idesc = f16 ? gpch::tc::idesc_f16_f32(BM, BN) : gpch::tc::idesc_bf16_f32(BM, BN);
            int kc = 0;
            bool ok = true;
            for (int p = 0; p < np && ok; ++p) {
                if (p >= 1 && !gpch::tc::mbar_wait(&tempty[0], (p - 1) & 1, 4 * SPIN_LIMIT)) {
                    atomicExch(err, 2);
                    break;
                }
                gpch::tc::tc_fence_after();
                const uint32_t acc = tmem;
                for (int q = 0; q < spp; ++q, ++kc) {
                    const int s = kc % STAGES;
                    if (!gpch::tc::mbar_wait(&full[s], (kc / STAGES) & 1, SPIN_LIMIT)) {
                        atomicExch(err, 2);
                        ok = false;
                        break;
                    }
                    gpch::tc::tc_fence_after();
                    const uint32_t sa = gpch::tc::smem_u32(smem + s * STAGE_BYTES);
                    const uint64_t a = gpch::tc::sdesc_sw128(sa);
                    const uint64_t b = diag ? a : gpch::tc::sdesc_sw128(sa + BOX_BYTES);
                    // a K step of 16 values advances the start address by 32
                    // bytes (2 in the descriptor); the tail of a split box
                    // row starts 64 bytes (4) after its head
                    if (split) {
#pragma unroll
                        for (int k = 0; k < 2; ++k) {
                            gpch::tc::mma_bf16(acc, a + 2 * k, b + 2 * k, idesc, (q | k) != 0 ? 1u : 0u);
                            gpch::tc::mma_bf16(acc, a + 2 * k, b + 4 + 2 * k, idesc, 1u);
                            gpch::tc::mma_bf16(acc, a + 4 + 2 * k, b + 2 * k, idesc, 1u);
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            gpch::tc::mma_bf16(acc, a + 2 * k, b + 2 * k, idesc, (q | k) != 0 ? 1u : 0u);
                    }
                    gpch::tc::mma_commit(&empty[s]);
                }
                if (ok) gpch::tc::mma_commit(&tfull[0]);
            }
        }
        __syncwarp();
    } else {
        // Epilogue: lane l of warp w holds tile row 32 (w % 4) + l.
        const int qw = warp & 3;
        const int64_t row = i0 + qw * 32 + lane;
        const bool row_ok = row < m;
        // scaled binary16 operands: the products carry 2^(2e); undo it exactly
        const float unscale =
            scale ? __int_as_float((127 - (rect ? scale[1] + scale_b[1] : 2 * scale[1])) << 23) : 1.0f;
        if (prefetch_c && sub) {
            // pull the C tile's columns into L2 while the first MMAs run
            const int64_t rows = (m - i0 < BM) ? m - i0 : BM;
            const uint32_t bytes = (uint32_t)(rows & ~int64_t(3)) * 4u;
            const int64_t col = c0 + (warp - 2) * 32 + lane;
            if (col < (rect ? ncol : m) && bytes > 0)
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(C + i0 + col * ldc), "r"(bytes)
                             : "memory");
        }
        // columns c0 + j with j < jn are in C's lower triangle (and < ncol)
        const int64_t lim = rect ? ncol - c0 : (row < ncol - 1 ? row : ncol - 1) - c0 + 1;
        const int jn = !row_ok ? 0 : (lim > BN ? BN : (lim < 0 ? 0 : (int)lim));
        const uint32_t tacc = tmem + ((uint32_t)(qw * 32) << 16), tsum = tacc + (uint32_t)BN;
        for (int p = 0; p < np; ++p) {
            const bool last = p == np - 1;
            float *crow = C + row + c0 * ldc;
            float cv[32];
            if (last && sub) {
#pragma unroll
                for (int j = 0; j < 32; ++j) cv[j] = (j < jn) ? crow[(int64_t)j * ldc] : 0.0f;
            }
            bool ok = gpch::tc::mbar_wait(&tfull[0], p & 1, 4 * SPIN_LIMIT);
            ok = __all_sync(0xffffffffu, ok);
            gpch::tc::tc_fence_after();
            if (!ok) {
                if (lane == 0) atomicExch(err, 3);
                break;
            }
#pragma unroll 1
            for (int cc = 0; cc < BN / 32; ++cc) {
                float *cb = C + row + (c0 + cc * 32) * ldc;
                // keep the column addresses from living across the loops
                asm volatile("" : "+l"(cb));
                if (last && cc > 0 && sub) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) cv[j] = (cc * 32 + j < jn) ? cb[(int64_t)j * ldc] : 0.0f;
                }
                float v[32];
                gpch::tc::tmem_ld32(tacc + cc * 32, v);
                if (cc == BN / 32 - 1) {
                    // the accumulator is read: the next panel may use it
                    gpch::tc::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) gpch::tc::mbar_arrive(&tempty[0]);
                }
                if (p > 0) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        float s[16];
                        gpch::tc::tmem_ld16(tsum + cc * 32 + h * 16, s);
#pragma unroll
                        for (int j = 0; j < 16; ++j) v[h * 16 + j] += s[j];
                    }
                }
                if (!last) {
                    gpch::tc::tmem_st32_wait(tsum + cc * 32, v);
                    continue;
                }
                asm volatile("" : "+l"(cb));
                if constexpr (!sub) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        v[j] *= unscale;
                        if (cc * 32 + j < jn) cb[(int64_t)j * ldc] = v[j];
                    }
                    if (ohi && jn > 0) {
                        // 16-byte stores: each lane writes its row's 32 values
                        // (64 bytes per copy); columns at or past jn are zero
                        const float osc = __int_as_float((127 + oscale[1]) << 23);
                        uint4 *oh = reinterpret_cast<uint4 *>(ohi + row * ldo + kpos(true, c0 + cc * 32));
                        uint4 *ol = oh + 4;   // the tail, 32 positions later
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            uint32_t hw[4], lw[4];
#pragma unroll
                            for (int h2 = 0; h2 < 4; ++h2) {
                                const int j = 8 * q + 2 * h2;
                                const float x0 = (cc * 32 + j < jn) ? v[j] * osc : 0.0f;
                                const float x1 = (cc * 32 + j + 1 < jn) ? v[j + 1] * osc : 0.0f;
                                const __half a0 = __float2half_rn(x0), a1 = __float2half_rn(x1);
                                const __half b0 = __float2half_rn(x0 - __half2float(a0));
                                const __half b1 = __float2half_rn(x1 - __half2float(a1));
                                hw[h2] = (uint32_t)__half_as_ushort(a0) | ((uint32_t)__half_as_ushort(a1) << 16);
                                lw[h2] = (uint32_t)__half_as_ushort(b0) | ((uint32_t)__half_as_ushort(b1) << 16);
                            }
                            oh[q] = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                            ol[q] = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                        }
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (cc * 32 + j < jn) cb[(int64_t)j * ldc] = cv[j] - v[j] * unscale;
                }
            }
        }
    }
    gpch::tc::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        gpch::tc::tc_fence_after();
        gpch::tc::tmem_dealloc<TMEM_COLS>(tmem);
    }
}

// FP32 column-major panel (m x k, ld ldp) -> bf16 K-major copy of width kp
// (zero-padded beyond k), row r at H + r * ldo: the head alone, or (split)
// head and tail interleaved as kpos() describes.  64 x 64 tiles through
// shared memory so that both the read and the write are coalesced.
__global__ void __launch_bounds__(256) panel_to_bf16_kernel(const float *__restrict__ P, int64_t ldp, int64_t m,
                                                            int k, int kp, __nv_bfloat16 *H, int split, int64_t ldo)
{
    __shared__ float tile[64][65];
    const int64_t r0 = (int64_t)blockIdx.x * 64;
    const int k0 = blockIdx.y * 64;
    for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
        const int r = e % 64, c = e / 64;
        tile[r][c] = (r0 + r < m && k0 + c < k) ? P[(r0 + r) + (int64_t)(k0 + c) * ldp] : 0.0f;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
        const int c = e % 64, r = e / 64;
        if (r0 + r < m && k0 + c < kp) {
            const float v = tile[r][c];
            const __nv_bfloat16 h = __float2bfloat16_rn(v);
            if (split) {
                __nv_bfloat16 *o = H + (r0 + r) * ldo + 2 * k0 + (c >> 5) * 64 + (c & 31);
                o[0] = h;
                o[32] = __float2bfloat16_rn(v - __bfloat162float(h));
            } else {
                H[(r0 + r) * ldo + k0 + c] = h;
            }
        }
    }
}

// Power-of-two scale exponent e of a panel whose largest |entry| has the
// FP32 bit pattern `bits`: the scaled maximum lies in [2^14, 2^15) (below
// binary16's 65504); clamped to [-60, 60].
__device__ inline int f16_scale_exp(unsigned bits)
{
    if (bits == 0) return 0;
    const int e = 14 - ((int)((bits >> 23) & 0xffu) - 127);
    return e < -60 ? -60 : (e > 60 ? 60 : e);
}

// Largest |entry| of the m x k FP32 panel, as FP32 bits (non-negative floats
// order like their bit patterns), into *absmax (zeroed by the caller).
__global__ void __launch_bounds__(256) panel_absmax_kernel(const float *__restrict__ P, int64_t ldp, int64_t m, int k,
                                                           unsigned *absmax)
{
    const int64_t r0 = (int64_t)blockIdx.x * 64;
    const int k0 = blockIdx.y * 64;
    float mx = 0.0f;
    for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
        const int r = e % 64, c = e / 64;
        if (r0 + r < m && k0 + c < k) mx = fmaxf(mx, fabsf(P[(r0 + r) + (int64_t)(k0 + c) * ldp]));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if ((threadIdx.x & 31) == 0) atomicMax(absmax, __float_as_uint(mx));
}

// FP32 panel -> split binary16 K-major copy (head and tail interleaved as
// kpos() describes, row r at H + r * ldo) of the panel scaled by 2^e
// (scale[0]: the panel's largest |entry| as FP32 bits; block (0, 0) writes e
// to scale[1] for the update's epilogue).  The scaling is exact, the head is
// the round-to-nearest binary16 value and the tail that of the (exact)
// remainder.
__global__ void __launch_bounds__(256) panel_to_f16_kernel(const float *__restrict__ P, int64_t ldp, int64_t m, int k,
                                                           int kp, __half *H, int *scale, int64_t ldo)
{
    __shared__ float tile[64][65];
    const int64_t r0 = (int64_t)blockIdx.x * 64;
    const int k0 = blockIdx.y * 64;
    const int e = f16_scale_exp((unsigned)scale[0]);
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) scale[1] = e;
    const float sc = __int_as_float((127 + e) << 23);
    for (int i = threadIdx.x; i < 64 * 64; i += blockDim.x) {
        const int r = i % 64, c = i / 64;
        tile[r][c] = (r0 + r < m && k0 + c < k) ? P[(r0 + r) + (int64_t)(k0 + c) * ldp] : 0.0f;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 64 * 64; i += blockDim.x) {
        const int c = i % 64, r = i / 64;
        if (r0 + r < m && k0 + c < kp) {
            const float v = tile[r][c] * sc;
            const __half h = __float2half_rn(v);
            __half *o = H + (r0 + r) * ldo + 2 * k0 + (c >> 5) * 64 + (c & 31);
            o[0] = h;
            o[32] = __float2half_rn(v - __half2float(h));
        }
    }
}

// Y = L^-1 for the nb x nb lower triangle L (FP32, column-major, ld ldl),
// nb <= 512 with nb % 32 == 0, L and ldl 16-byte aligned, into Y
// (column-major, ld ldy; zero above the diagonal; other sizes are left
// untouched; absmax, if given, gets the largest |entry| of Y as FP32 bits
// by atomicMax, so it must start at 0).  CTA b owns the 8 columns
// 8b .. 8b+7 of Y (L y = e_c, forward
// substitution) and keeps them in shared memory, rows in blocks of 32.
// Block column K of L (rows 32K .. nb-1) arrives as one or two units, 2-D
// TMA boxes of 256 rows x 32 columns through tmL (L as an nb x nb FP32
// tensor; completion on an mbarrier; bounded waits set *err = 5), two
// units ahead of their use (three buffers, about 112 KB in all, so that a
// CTA fits on an SM beside a CTA of the trailing update).  Per block:
// warp w solves the 32 x 32 diagonal block for column w (lane = row; one
// shuffle and one FMA per row), then the later rows are updated as a GEMM,
// rows x 8 columns x 32, in 4 x 4 register tiles (two 16-byte loads feed 16
// FMAs), the rows of each unit as it arrives.
constexpr int TI_COLS = 8;
constexpr int TI_MAXN = 512;
constexpr int TI_THREADS = 256;
constexpr int TI_BUFS = 3;
constexpr int TI_BOX = 256;                     // rows of one TMA box (one unit)
constexpr size_t TI_SMEM = 128 + (size_t)(TI_BUFS * TI_BOX * 32 + TI_MAXN * TI_COLS) * sizeof(float);
static_assert(2 * TI_BOX >= TI_MAXN, "a block column is at most two units");
__global__ void __launch_bounds__(TI_THREADS) tri_inv_f32_kernel(const __grid_constant__ CUtensorMap tmL, int nb,
                                                                 float *Y, int64_t ldy, int *err, unsigned *absmax)
{
    extern __shared__ __align__(128) float ti_smem_raw[];
    float *ti_smem = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(ti_smem_raw) + 127) & ~uintptr_t(127));
    __shared__ __align__(8) uint64_t bar[TI_BUFS];
    if (nb % 32 != 0 || nb > TI_MAXN) return;
    float *Ts = ti_smem + TI_BUFS * TI_BOX * 32;   // Ts[r * TI_COLS + c]: row r of this CTA's columns
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int c0 = blockIdx.x * TI_COLS;
    const int nK = nb / 32, K0 = c0 / 32;
    if (tid == 0) {
        for (int b = 0; b < TI_BUFS; ++b) gpch::tc::mbar_init(&bar[b], 1);
        gpch::tc::fence_mbar_init();
    }
    __syncthreads();
    // unit (K, h): rows 32K + 256h .. 32K + 256h + 255 of block column K
    // (h = 1 only when the column has more than 256 rows; rows past nb read
    // as zeros), in buffer u % 3 for the u-th unit, row q of column 32K + kk
    // at kk * 256 + q
    auto next_unit = [&](int &K, int &h) {
        if (h == 0 && 32 * K + TI_BOX < nb) {
            h = 1;
        } else {
            ++K;
            h = 0;
        }
    };
    int sK = K0, sh = 0, nstaged = 0;   // the next unit to stage (every thread tracks it)
    auto stage_next = [&]() {
        if (sK >= nK) return;
        if (tid == 0) {
            const int b = nstaged % TI_BUFS;
            gpch::tc::mbar_arrive_expect_tx(&bar[b], TI_BOX * 32u * 4u);
            gpch::tc::tma_load_2d(ti_smem + b * TI_BOX * 32, &tmL, &bar[b], 32 * sK + TI_BOX * sh, 32 * sK);
        }
        ++nstaged;
        next_unit(sK, sh);
    };
    uint32_t phases = 0;   // bit b: parity of buffer b's next phase
    bool ok = true;
    stage_next();
    stage_next();
    for (int e = tid; e < TI_MAXN * TI_COLS; e += TI_THREADS) {
        const int r = e / TI_COLS, cc = e % TI_COLS;
        Ts[e] = (r == c0 + cc) ? 1.0f : 0.0f;
    }
    int K = K0, h = 0, ncons = 0;
    while (K < nK) {
        stage_next();
        const int bk = ncons % TI_BUFS;
        ok = gpch::tc::mbar_wait(&bar[bk], (phases >> bk) & 1u, 1u << 24);
        phases ^= 1u << bk;
        ok = __syncthreads_and(ok);
        if (!ok) {
            if (tid == 0) atomicExch(err, 5);
            // let every copy this CTA started land before it exits
            gpch::tc::mbar_wait(&bar[bk], ((phases >> bk) & 1u) ^ 1u, 1u << 24);
            for (int u = ncons + 1; u < nstaged; ++u)
                gpch::tc::mbar_wait(&bar[u % TI_BUFS], (phases >> (u % TI_BUFS)) & 1u, 1u << 24);
            break;
        }
        const float *Ls = ti_smem + bk * TI_BOX * 32;
        if (h == 0) {
            // diagonal block, column c0 + warp, row 32K + lane
            const int r = 32 * K + lane;
            float t = Ts[r * TI_COLS + warp];
            const float rp = 1.0f / Ls[lane * TI_BOX + lane];
#pragma unroll 8
            for (int kk = 0; kk < 32; ++kk) {
                const float l = Ls[kk * TI_BOX + lane];
                const float y = __shfl_sync(0xffffffffu, t * rp, kk);
                const float tn = fmaf(-l, y, t);
                t = (lane == kk) ? y : ((lane > kk) ? tn : t);
            }
            Ts[r * TI_COLS + warp] = t;
            __syncthreads();
        }
        // this unit's later rows: T[r][:] -= L[r][32K..32K+31] Y[32K..32K+31][:]
        const int ubase = 32 * K + TI_BOX * h;
        const int rbeg = h == 0 ? 32 * (K + 1) : ubase, rend = (ubase + TI_BOX < nb) ? ubase + TI_BOX : nb;
        const int ntiles = (rend > rbeg ? rend - rbeg : 0) / 4 * (TI_COLS / 4);
        for (int tile = tid; tile < ntiles; tile += TI_THREADS) {
            const int r0 = rbeg + 4 * (tile / (TI_COLS / 4)), cg = 4 * (tile % (TI_COLS / 4));
            float acc[4][4] = {};
#pragma unroll 8
            for (int kk = 0; kk < 32; ++kk) {
                const float4 lv = *reinterpret_cast<const float4 *>(Ls + kk * TI_BOX + (r0 - ubase));
                const float4 yv = *reinterpret_cast<const float4 *>(Ts + (32 * K + kk) * TI_COLS + cg);
                const float la[4] = {lv.x, lv.y, lv.z, lv.w}, ya[4] = {yv.x, yv.y, yv.z, yv.w};
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(la[a], ya[b], acc[a][b]);
            }
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                float4 *tp = reinterpret_cast<float4 *>(Ts + (r0 + a) * TI_COLS + cg);
                float4 v = *tp;
                v.x -= acc[a][0];
                v.y -= acc[a][1];
                v.z -= acc[a][2];
                v.w -= acc[a][3];
                *tp = v;
            }
        }
        __syncthreads();   // the buffer is refilled two units on; Ts rows are read by later units
        ++ncons;
        next_unit(K, h);
    }
    float mx = 0.0f;
    for (int e = tid; e < nb * TI_COLS; e += TI_THREADS) {
        const int r = e % nb, cc = e / nb;
        const float v = Ts[r * TI_COLS + cc];
        Y[r + (int64_t)(c0 + cc) * ldy] = v;
        mx = fmaxf(mx, fabsf(v));
    }
    if (absmax) {
        // largest |entry| as FP32 bits (non-negative floats order like their bits)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        if (lane == 0) atomicMax(absmax, __float_as_uint(mx));
    }
}

// Scale word of a whole split-f16 factor from the a-priori bound
// |L_ij| <= sqrt(max_i W_ii) (W = A + shift I, SPD): scale[0] = FP32 bits of
// sqrt(max_i W_ii), from which the conversions derive the exponent.
// pscale (optional): the same for the panels before their solve, bounded
// by max_i W_ii.
__global__ void __launch_bounds__(256) factor_scale_kernel(int64_t n, const float *__restrict__ W, int64_t ldw,
                                                           int *scale, int *pscale)
{
    __shared__ float red[8];
    float mx = 0.0f;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) mx = fmaxf(mx, W[i + i * ldw]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) mx = fmaxf(mx, red[w]);
        mx = fmaxf(mx, red[0]);
        const float r = sqrtf(mx);
        scale[0] = (int)__float_as_uint(r);
        scale[1] = f16_scale_exp(__float_as_uint(r));
        if (pscale) {
            // entries of an SPD trailing matrix S obey |S_ij| <= max_i S_ii <= max_i W_ii
            pscale[0] = (int)__float_as_uint(mx);
            pscale[1] = f16_scale_exp(__float_as_uint(mx));
        }
    }
}

// The same scale words from A's diagonal: W_ii = fl32(A_ii + shift), the
// value the input pass writes, so that the scale need not wait for it.
__global__ void __launch_bounds__(256) factor_scale_from_a_kernel(int64_t n, const double *__restrict__ A, int64_t lda,
                                                                  double shift, int *scale, int *pscale)
{
    __shared__ float red[8];
    float mx = 0.0f;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) mx = fmaxf(mx, (float)(A[i + i * lda] + shift));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) mx = fmaxf(mx, red[w]);
        mx = fmaxf(mx, red[0]);
        const float r = sqrtf(mx);
        scale[0] = (int)__float_as_uint(r);
        scale[1] = f16_scale_exp(__float_as_uint(r));
        if (pscale) {
            pscale[0] = (int)__float_as_uint(mx);
            pscale[1] = f16_scale_exp(__float_as_uint(mx));
        }
    }
}

// FP32 inverses of the 64 x 64 diagonal blocks of the factored FP64 tile D
// (nj x nj, ld ldd), for the FP32 panel solve: block b of the grid inverts
// rows/columns [64b, 64b + 64), unit-padded, by right-looking substitution
// on all columns of the identity (thread (tx, ty) keeps entries (tx + 16i,
// ty + 16jj)).  Stored widened to FP64 (column-major, ld 64).
__global__ void __launch_bounds__(256) inv_blocks_f32_kernel(const double *__restrict__ D, int64_t ldd, int64_t nj,
                                                             double *Linv, float *Linv32)
{
    __shared__ float S[LEAF][LEAF + 1];
    __shared__ float dinv[LEAF];
    __shared__ float xrow[2][LEAF];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int64_t o = (int64_t)blockIdx.x * LEAF;
    const int nb = (int)((nj - o < LEAF) ? nj - o : LEAF);
    for (int e = tid; e < LEAF * LEAF; e += blockDim.x) {
        const int r = e % LEAF, c = e / LEAF;
        float v;
        if (r < nb && c < nb) v = (r >= c) ? (float)D[(o + r) + (o + c) * ldd] : 0.0f;
        else v = (r == c) ? 1.0f : 0.0f;
        S[r][c] = v;
    }
    __syncthreads();
    if (tid < LEAF) dinv[tid] = 1.0f / S[tid][tid];
    float x[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) x[i][jj] = (tx + 16 * i == ty + 16 * jj) ? 1.0f : 0.0f;
    __syncthreads();
    for (int j = 0; j < LEAF; ++j) {
        float *xr = xrow[j & 1];
        if (tx == j % 16) {
            // row j is x[j / 16]: selected with compile-time indices so that
            // x stays in registers
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (i != j / 16) continue;
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const int c = ty + 16 * jj;
                    if (c <= j) {
                        x[i][jj] *= dinv[j];
                        xr[c] = x[i][jj];
                    }
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = tx + 16 * i;
            if (r <= j) continue;
            const float l = S[r][j];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                const int c = ty + 16 * jj;
                if (c <= j) x[i][jj] -= l * xr[c];
            }
        }
    }
    double *dst = Linv + (int64_t)blockIdx.x * LEAF * LEAF;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            dst[(tx + 16 * i) + (ty + 16 * jj) * LEAF] = (double)x[i][jj];
            Linv32[(int64_t)blockIdx.x * LEAF * LEAF + (tx + 16 * i) + (ty + 16 * jj) * LEAF] = x[i][jj];
        }
}

// Step 2 of the mixed factor for a whole block column in one launch:
// X = P L_jj^-T on the m x nj panel P (nj <= PN_MAXK), FP32.  Each CTA owns
// PN_ROWS rows of the panel, keeps them in shared memory and runs the
// blocked substitution over the 64-column chunks of L_jj:
//   for c: X_c = P_c inv(L_cc)^T;  for d > c: P_d -= X_c L_dc^T
// (inv(L_cc): the FP32 inverses of the 64 x 64 diagonal blocks, computed
// from the FP64 factor).  The 64 x 64 blocks of L are read through L2 and
// double-buffered in shared memory with cp.async; thread (tr, tc) keeps a
// 4 x 4 register tile (rows 4 tr.., columns 4 tc..) of every block product.
// A warp covers 8 values of tr and 4 of tc, so per k its two 16-byte
// shared-memory loads touch 128 B (rows) and 64 B (columns).  32 rows per
// CTA keep its shared memory (96 KB) small enough to share an SM with a CTA
// of the tensor-core update running on the other stream.
constexpr int PN_ROWS = 32;
constexpr int PN_THREADS = 128;
constexpr int PN_MAXK = 512;
constexpr size_t PN_SMEM = (size_t)(PN_MAXK * PN_ROWS + 2 * LEAF * LEAF) * sizeof(float);

__device__ __forceinline__ void cp_async16(void *dst, const void *src, int src_bytes)
{
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}

__global__ void __launch_bounds__(PN_THREADS, 2) panel_trsm_f32_kernel(float *P, int64_t ldp, int64_t m, int nj,
                                                                const float *__restrict__ L, int64_t ldl,
                                                                const float *__restrict__ Linv32,
                                                                const int64_t *info)
{
    extern __shared__ __align__(16) float pn_smem[];
    float *Xs = pn_smem;                         // Xs[k * PN_ROWS + r]
    float *Lb = pn_smem + PN_MAXK * PN_ROWS;     // 2 buffers, [k * 64 + j]
    if (info && *info != 0) return;
    const int tid = threadIdx.x, warp = tid / 32;
    const int tr = tid % 8, tc = (tid / 8) % 4 + 4 * warp;
    const int64_t r0 = (int64_t)blockIdx.x * PN_ROWS;
    const int nch = (nj + LEAF - 1) / LEAF;
    const int nops = nch + nch * (nch - 1) / 2;

    // op q -> (c, d): d == c is the inverse product of chunk c, d > c the
    // update of chunk d by chunk c; ops run c-major.
    auto op_cd = [&](int q, int &c, int &d) {
        c = 0;
        int left = q;
        while (left >= nch - c) {
            left -= nch - c;
            ++c;
        }
        d = c + left;
    };
    auto stage = [&](int q, int buf) {
        int c, d;
        op_cd(q, c, d);
        float *dst = Lb + buf * LEAF * LEAF;
        for (int e = tid; e < LEAF * LEAF / 4; e += PN_THREADS) {
            const int j4 = (e % 16) * 4, k = e / 16;
            if (c == d) {
                cp_async16(dst + k * LEAF + j4, Linv32 + (int64_t)c * LEAF * LEAF + j4 + k * LEAF, 16);
            } else {
                const int row = d * LEAF + j4;   // rows of L_dc; columns of chunk c are all inside L_jj
                const int valid = nj - row;
                const float *src = L + row + (int64_t)(c * LEAF + k) * ldl;
                cp_async16(dst + k * LEAF + j4, valid > 0 ? src : L, valid >= 4 ? 16 : (valid > 0 ? valid * 4 : 0));
            }
        }
    };

    // the CTA's rows, 16 bytes at a time (rows past m and columns past nj
    // are zero-filled)
    for (int e = tid; e < nch * LEAF * (PN_ROWS / 4); e += PN_THREADS) {
        const int r4 = (e % (PN_ROWS / 4)) * 4, k = e / (PN_ROWS / 4);
        const int64_t rows = m - r0 - r4;
        const int bytes = (k >= nj || rows <= 0) ? 0 : (rows >= 4 ? 16 : (int)rows * 4);
        cp_async16(Xs + k * PN_ROWS + r4, bytes ? P + (r0 + r4) + (int64_t)k * ldp : P, bytes);
    }
    stage(0, 0);
    asm volatile("cp.async.commit_group;" ::: "memory");
    for (int q = 0; q < nops; ++q) {
        int c, d;
        op_cd(q, c, d);
        if (q + 1 < nops) stage(q + 1, (q + 1) & 1);
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        __syncthreads();
        const float *Lq = Lb + (q & 1) * LEAF * LEAF;
        const float *xc = Xs + (c * LEAF) * PN_ROWS + 4 * tr;
        float acc[4][4] = {};
#pragma unroll 8
        for (int k = 0; k < LEAF; ++k) {
            const float4 x = *reinterpret_cast<const float4 *>(xc + k * PN_ROWS);
            const float4 l = *reinterpret_cast<const float4 *>(Lq + k * LEAF + 4 * tc);
            const float xv[4] = {x.x, x.y, x.z, x.w}, lv[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) acc[i][jj] = fmaf(xv[i], lv[jj], acc[i][jj]);
        }
        float *xd = Xs + (d * LEAF + 4 * tc) * PN_ROWS + 4 * tr;
        if (c == d) {
            __syncthreads();   // every thread has read chunk c
#pragma unroll
            for (int jj = 0; jj < 4; ++jj)
                *reinterpret_cast<float4 *>(xd + jj * PN_ROWS) =
                    make_float4(acc[0][jj], acc[1][jj], acc[2][jj], acc[3][jj]);
        } else {
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                float4 v = *reinterpret_cast<float4 *>(xd + jj * PN_ROWS);
                v.x -= acc[0][jj];
                v.y -= acc[1][jj];
                v.z -= acc[2][jj];
                v.w -= acc[3][jj];
                *reinterpret_cast<float4 *>(xd + jj * PN_ROWS) = v;
            }
        }
        __syncthreads();
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    for (int e = tid; e < nch * LEAF * PN_ROWS; e += PN_THREADS) {
        const int r = e % PN_ROWS, k = e / PN_ROWS;
        if (r0 + r < m && k < nj) P[(r0 + r) + (int64_t)k * ldp] = Xs[e];
    }
}

// W (FP32, lower triangle) = A (FP64) + shift * I.  One CTA per column j;
// the threads walk rows j.. of it, four at a time per thread.
// W = A + shift I on the lower triangle (FP32), one CTA per column.
__global__ void __launch_bounds__(256) init_w_kernel(int64_t n, const double *__restrict__ A, int64_t lda, float *W,
                                                     int64_t ldw, double shift)
{
    const int64_t j = blockIdx.x;
    const double *a = A + j * lda;
    float *w = W + j * ldw;
    if (threadIdx.x == 0) w[j] = (float)(a[j] + shift);
    int64_t i = j + 1 + threadIdx.x;
    for (; i + 3 * 256 < n; i += 4 * 256) {
        const double v0 = a[i], v1 = a[i + 256], v2 = a[i + 512], v3 = a[i + 768];
        w[i] = (float)v0;
        w[i + 256] = (float)v1;
        w[i + 512] = (float)v2;
        w[i + 768] = (float)v3;
    }
    for (; i < n; i += 256) w[i] = (float)a[i];
}

// W = A + shift I on the lower triangle (FP32) together with the pieces of
// ||A||_inf (= max_i sum_j |A_ij| for symmetric A), from the lower triangle
// only: row i's sum is its part left of and on the diagonal plus, by
// symmetry, column i's part below the diagonal.  CTA (b, q) covers the
// NW_COLS columns of strip b (c0 = NW_COLS b ..) and the NW_ROWS rows of
// chunk q (r0 = NW_ROWS q ..), walking the strip column by column so that
// each column piece streams contiguously from HBM; thread t owns the rows
// r0 + t + 256 k.
// * part[b * n + row]: the row's sum over the strip (registers across the
//   columns);
// * colpart[q * n + col]: the column's sum over the chunk's rows below the
//   diagonal (a fixed-order CTA reduction).
// CTAs whose chunk lies above the strip leave at once.  The magnitudes come
// from the FP32 values written to W (one conversion per entry, which the
// FP64 pipe performs); the norm only scales the refinement's stopping test
// and reported backward error.  Strips from strip0 on (a block column's at a
// time when the factor runs the pass).  With packed, each entry of the lower
// triangle is also cut into the head and tail of 2^-ea A_ij (df_split_a,
// ebias = 896 + ea) and stored in the refinement's packed copy.
constexpr int NW_COLS = 64;
constexpr int NW_ROWS = 1024;   // short CTAs: the factor runs the pass beside its own kernels
constexpr int NW_THREADS = 256;
constexpr int NW_PER = NW_ROWS / NW_THREADS;   // rows of a thread
__global__ void __launch_bounds__(NW_THREADS) init_w_norm_kernel(int64_t n, const double *__restrict__ A,
                                                                 int64_t lda, float *W, int64_t ldw, double shift,
                                                                 float *part, float *colpart, int64_t strip0,
                                                                 float2 *packed, unsigned ebias)
{
    __shared__ float red[NW_THREADS / 32][NW_COLS];
    const int64_t strip = strip0 + (int64_t)blockIdx.x;   // strips strip0.. (a block column's at a time)
    const int64_t c0 = strip * NW_COLS, r0 = (int64_t)blockIdx.y * NW_ROWS;
    if (r0 + NW_ROWS <= c0) return;   // the chunk lies above the strip
    const int cw = (int)((n - c0 < NW_COLS) ? n - c0 : NW_COLS);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float racc[NW_PER];
#pragma unroll
    for (int k = 0; k < NW_PER; ++k) racc[k] = 0.0f;
    const int64_t n2 = (n + 1) & ~int64_t(1);
    for (int c = 0; c < cw; ++c) {
        const int64_t col = c0 + c;
        const double *a = A + col * lda;
        float *w = W + col * ldw;
        // with packed: this column of the refinement's packed copy, by row
        const int64_t pj = col / gpch::SYM_STRIP, ps = pj * gpch::SYM_STRIP;
        float2 *pc = packed ? packed + gpch::sy_off(n, pj) + (col - ps) * (n2 - ps) - ps : nullptr;
        double v[NW_PER];
#pragma unroll
        for (int k = 0; k < NW_PER; ++k) {
            const int64_t row = r0 + threadIdx.x + NW_THREADS * k;
            v[k] = (row >= col && row < n) ? a[row] : 0.0;
        }
        float cacc = 0.0f;
#pragma unroll
        for (int k = 0; k < NW_PER; ++k) {
            const int64_t row = r0 + threadIdx.x + NW_THREADS * k;
            if (row > col && row < n) {
                const float f = (float)v[k];
                w[row] = f;
                racc[k] += fabsf(f);
                cacc += fabsf(f);
            } else if (row == col) {
                w[row] = (float)(v[k] + shift);
                racc[k] += fabsf((float)v[k]);
            }
            if (pc && row >= col && row < n) {
                float h, t;
                gpch::df_split_a(v[k], ebias, h, t);
                pc[row] = make_float2(h, t);
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) cacc += __shfl_xor_sync(0xffffffffu, cacc, off);
        if (lane == 0) red[warp][c] = cacc;
    }
    float *prow = part + strip * n;
#pragma unroll
    for (int k = 0; k < NW_PER; ++k) {
        const int64_t row = r0 + threadIdx.x + NW_THREADS * k;
        if (row < n) prow[row] = racc[k];
    }
    __syncthreads();
    if (threadIdx.x < cw) {
        float t = 0.0f;
        for (int w2 = 0; w2 < NW_THREADS / 32; ++w2) t += red[w2][threadIdx.x];
        colpart[(int64_t)blockIdx.y * n + c0 + threadIdx.x] = t;
    }
}

// *anorm = max_i (sum over the strips b <= i / NW_COLS of part[b * n + i]
// + sum over the chunks q >= (NW_COLS (i / NW_COLS)) / NW_ROWS of
// colpart[q * n + i]), each row summed in a fixed order; *anorm holds a
// non-negative double compared through its bit pattern (zeroed by the
// caller).
__global__ void __launch_bounds__(256) norm_reduce_kernel(int64_t n, const float *__restrict__ part,
                                                          const float *__restrict__ colpart, double *anorm)
{
    __shared__ double red[8];
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    double m = 0.0;
    if (i < n) {
        float s = 0.0f;
        const int64_t nb = i / NW_COLS, nq = (n + NW_ROWS - 1) / NW_ROWS;
        for (int64_t b = 0; b <= nb; ++b) s += part[b * n + i];
        for (int64_t q = (nb * NW_COLS) / NW_ROWS; q < nq; ++q) s += colpart[q * n + i];
        m = (double)s;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w2 = 1; w2 < 8; ++w2) m = fmax(m, red[w2]);
        m = fmax(m, red[0]);
        atomicMax(reinterpret_cast<unsigned long long *>(anorm), (unsigned long long)__double_as_longlong(m));
    }
}

// Step 1 in FP32, left-looking, one launch per 32-column block of the
// diagonal tile T (nb x nb, ld ldt): the launch for the block column at
// c0 = 32 s forms, in every CTA b,
//   D = T(c0.., c0..) - L(c0.., 0:c0) L(c0.., 0:c0)^T   (the 32 x 32 diagonal block)
//   X = T(R.., c0..)  - L(R.., 0:c0)  L(c0.., 0:c0)^T   (its 32 rows, R = c0 + 32 (b + 1))
// (warps 0-3 form D, warps 4-7 form X, 4 x 4 outputs per thread over
// half of each chunk's K columns, the halves added at the end; the
// columns 0:c0 of both row sets staged k-major in shared memory 32 at a
// time by cp.async, three chunks in flight), factors D on one warp (each
// pivot column broadcast through shared memory), inverts L_ss on all eight
// warps (four columns each) and forms X L_ss^-T as one 32 x 32 product.
// Every CTA forms and factors D itself, so the launch needs no
// communication between CTAs.  Launched as a programmatic dependent of the
// previous block column's launch: what does not depend on it (the entries
// of block column s, and K columns before the previous block column) is
// loaded before the wait.  L_ss may not be written into T while other CTAs
// of the launch may still read T's block there as D's input: with one CTA
// it is written at once, otherwise CTA 0 leaves it in `lss` (32 x 32, ld
// 32) and the launch of the next block column (which reads no entry of
// that block) copies it into T (prev_c0 >= 0).  A pivot that is not
// positive sets *info = col0 + c0 + (its column) + 1 (CTA 0) and ends
// every CTA.  The 32 x 32 blocks used after the K loop share the stages'
// shared memory, so that a CTA (about 25 KB) fits on an SM beside two
// CTAs of the trailing update, which run meanwhile on other streams.
__device__ __forceinline__ void cp_async_f32(float *dst, const float *src)
{
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
// wait until at most `pending` of this thread's cp.async groups are in flight
__device__ __forceinline__ void cp_async_wait_upto(int pending)
{
    if (pending <= 0) asm volatile("cp.async.wait_group 0;" ::: "memory");
    else if (pending == 1) asm volatile("cp.async.wait_group 1;" ::: "memory");
    else if (pending == 2) asm volatile("cp.async.wait_group 2;" ::: "memory");
    else if (pending == 3) asm volatile("cp.async.wait_group 3;" ::: "memory");
    else if (pending == 4) asm volatile("cp.async.wait_group 4;" ::: "memory");
    else asm volatile("cp.async.wait_group 5;" ::: "memory");
}

constexpr int DS_THREADS = 256;
constexpr int DS_KC = 32;       // K columns per staged chunk (one block column)
constexpr int DS_STAGES = 3;    // chunks in flight (cp_async_wait_upto covers up to 5 pending)
constexpr int DS_STAGE_FLOATS = DS_STAGES * DS_KC * 32;
static_assert(3 * 32 * 33 <= 2 * DS_STAGE_FLOATS, "the post-loop blocks fit in the stages");
__global__ void __launch_bounds__(DS_THREADS) diag_step_kernel(float *T, int64_t ldt, int nb, int c0, int64_t col0,
                                                               int64_t *info, float *lss, int prev_c0)
{
    __shared__ __align__(16) float stg[2 * DS_STAGE_FLOATS];
    // K loop: Ad[.][k][i] = L(c0 + i, k0 + k), Ar[.][k][r] = L(R + r, k0 + k)
    float(*Ad)[DS_KC][32] = reinterpret_cast<float(*)[DS_KC][32]>(stg);
    float(*Ar)[DS_KC][32] = reinterpret_cast<float(*)[DS_KC][32]>(stg + DS_STAGE_FLOATS);
    // after it: D, then L_ss (zero above the diagonal); X; L_ss^-1
    float(*Ds)[33] = reinterpret_cast<float(*)[33]>(stg);
    float(*Xs)[33] = reinterpret_cast<float(*)[33]>(stg + 32 * 33);
    float(*Ys)[33] = reinterpret_cast<float(*)[33]>(stg + 2 * 32 * 33);
    __shared__ float rd[32];
    __shared__ __align__(16) float colb[32];   // the pivot column being broadcast
    __shared__ int bad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nc = (nb - c0 < 32) ? nb - c0 : 32;
    const int R = c0 + 32 * ((int)blockIdx.x + 1);
    const int nr = (nb - R < 0) ? 0 : ((nb - R < 32) ? nb - R : 32);
    // threads 0-127 form D, 128-255 X; within each, the first 64 take the
    // even halves of every chunk's K columns and the last 64 the odd halves
    // (4 x 4 outputs per thread), added together once after the K loop
    const bool isD = tid < DS_THREADS / 2;
    const int u = isD ? tid : tid - DS_THREADS / 2;
    const int kh = u / 64, v = u % 64;
    const int ri = 4 * (v % 8), cj = 4 * (v / 8);   // this thread's rows ri.., columns cj..
    const int row0 = isD ? c0 : R, nrow = isD ? nc : nr;
    const int nchunk = c0 / DS_KC;
    float acc[4][4];
    auto init_acc = [&]() {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int i = ri + a, j = cj + b;
                // D: its lower triangle only (the tile's upper triangle is not read)
                const bool in = kh == 0 && i < nrow && j < nc && (!isD || j <= i);
                acc[a][b] = in ? T[(row0 + i) + (int64_t)(c0 + j) * ldt] : 0.0f;
            }
    };
    // chunk ch (K columns 32 ch ..) into stage ch % DS_STAGES, one commit group
    auto stage = [&](int ch) {
        const int k0 = ch * DS_KC, sb = ch % DS_STAGES;
        for (int e = tid; e < DS_KC * 32; e += DS_THREADS) {
            const int r = e & 31, k = e >> 5;
            const float *col = T + (int64_t)(k0 + k) * ldt;
            if (r < nc) cp_async_f32(&Ad[sb][k][r], col + c0 + r);
            else Ad[sb][k][r] = 0.0f;
            if (r < nr) cp_async_f32(&Ar[sb][k][r], col + R + r);
            else Ar[sb][k][r] = 0.0f;
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    int issued = 0;
    const bool early = c0 > 0;   // the previous launch is this tile's block column s - 1
    if (early) {
        init_acc();
        // K columns before the previous block column (32 wide) only
        while (issued < DS_STAGES - 1 && issued < nchunk - 32 / DS_KC) stage(issued++);
    }
    gpch::pdl_wait();
    gpch::pdl_trigger();
    if (*info != 0) {   // the same value in every thread
        asm volatile("cp.async.wait_all;" ::: "memory");
        return;
    }
    if (prev_c0 >= 0 && blockIdx.x == 0) {
        // the previous block column's diagonal block (32 columns: it was not the last)
        for (int e = tid; e < 32 * 32; e += DS_THREADS) {
            const int i = e % 32, j = e / 32;
            if (j <= i) T[(prev_c0 + i) + (int64_t)(prev_c0 + j) * ldt] = lss[i + 32 * j];
        }
    }
    if (!early) init_acc();
    while (issued < DS_STAGES - 1 && issued < nchunk) stage(issued++);
    for (int ch = 0; ch < nchunk; ++ch) {
        if (issued < nchunk && issued < ch + DS_STAGES) stage(issued++);
        cp_async_wait_upto(issued - 1 - ch);
        __syncthreads();
        const int sb = ch % DS_STAGES;
        const float(*Ao)[32] = isD ? Ad[sb] : Ar[sb];
        const float(*Bo)[32] = Ad[sb];
#pragma unroll 4
        for (int k = kh * (DS_KC / 2); k < (kh + 1) * (DS_KC / 2); ++k) {
            const float4 av = *reinterpret_cast<const float4 *>(&Ao[k][ri]);
            const float4 bv = *reinterpret_cast<const float4 *>(&Bo[k][cj]);
            const float x[4] = {av.x, av.y, av.z, av.w}, y[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(-x[a], y[b], acc[a][b]);
        }
        __syncthreads();   // the stage is refilled by a later chunk
    }
    // the two K halves: the odd halves' sums first, then the even halves add theirs
    float(*Os)[33] = isD ? Ds : Xs;
    if (kh == 1) {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) Os[ri + a][cj + b] = acc[a][b];
    }
    __syncthreads();
    if (kh == 0) {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) Os[ri + a][cj + b] += acc[a][b];
    }
    if (tid == 0) bad = 0;
    __syncthreads();
    if (warp == 0) {
        // the leaf: lane i holds row i of D
        float a[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) a[j] = (j <= lane && lane < nc && j < nc) ? Ds[lane][j] : 0.0f;
        int fail = 0;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            if (j < nc && fail == 0) {
                const float d = __shfl_sync(0xffffffffu, a[j], j);
                if (!(d > 0.0f)) {
                    fail = j + 1;
                } else {
                    const float r = rsqrtf(d), ljj = d * r;
                    const float l = (lane == j) ? ljj : ((lane > j) ? a[j] * r : 0.0f);
                    a[j] = (lane >= j) ? l : 0.0f;
                    if (lane == j) rd[j] = r;
                    __syncwarp();   // the previous column's broadcast has been read
                    colb[lane] = l;
                    __syncwarp();
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        if (4 * q + 3 > j) {
                            const float4 v = *reinterpret_cast<const float4 *>(&colb[4 * q]);
                            const float c[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                if (4 * q + e > j) a[4 * q + e] = fmaf(-l, c[e], a[4 * q + e]);
                        }
                    }
                }
            }
        }
        if (fail != 0) {
            if (lane == 0) {
                bad = 1;
                if (blockIdx.x == 0) *info = col0 + c0 + fail;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) Ds[lane][j] = a[j];
        }
    }
    __syncthreads();
    if (bad) return;
    if (blockIdx.x == 0 && tid < nc) {
        if (gridDim.x == 1) {
            for (int j = 0; j <= tid; ++j) T[(c0 + tid) + (int64_t)(c0 + j) * ldt] = Ds[tid][j];
        } else {
            for (int j = 0; j <= tid; ++j) lss[tid + 32 * j] = Ds[tid][j];
        }
    }
    if (nr == 0) return;   // (a block column with rows below it is 32 wide)
    {
        // Y = L_ss^-1: warp w solves L y = e_c for c = 4w .. 4w + 3, lane = row
        float lrow[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) lrow[k] = Ds[lane][k];
        float y[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) y[q] = (lane == 4 * warp + q) ? 1.0f : 0.0f;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const float rj = rd[j];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (lane == j) y[q] *= rj;
                const float yj = __shfl_sync(0xffffffffu, y[q], j);
                if (lane > j) y[q] = fmaf(-lrow[j], yj, y[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) Ys[lane][4 * warp + q] = y[q];
    }
    __syncthreads();
    {
        // X L_ss^-T: thread (row r, columns 4 jg ..)
        const int r = tid & 31, jg = tid >> 5;
        float o[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll 8
        for (int k = 0; k < 32; ++k) {
            const float x = Xs[r][k];
#pragma unroll
            for (int q = 0; q < 4; ++q) o[q] = fmaf(x, Ys[4 * jg + q][k], o[q]);
        }
        if (r < nr) {
#pragma unroll
            for (int q = 0; q < 4; ++q) T[(R + r) + (int64_t)(c0 + 4 * jg + q) * ldt] = o[q];
        }
    }
}

// Copy the nb x nb lower block of FP32 W into FP64 D (ld ldd).
__global__ void tile_f32_to_f64(int64_t nb, const float *__restrict__ W, int64_t ldw, double *D, int64_t ldd)
{
    const int64_t j = blockIdx.y;
    for (int64_t i = j + threadIdx.x; i < nb; i += blockDim.x) D[i + j * ldd] = (double)W[i + j * ldw];
}

// Tensor map over a K-major 16-bit panel copy of m rows, `width` positions
// per row (kpos() of the K columns used) and row stride ld positions (both
// multiples of 64): 128-row boxes of BOX_K positions with 128-byte
// swizzling.  Every TMA x coordinate used is a multiple of 64 positions.
gpch_status make_panel_map(gpch_ctx *ctx, CUtensorMap *map, const void *base, int64_t m, int64_t width, int64_t ld,
                           bool f16)
{
    auto enc = gpch::tc::tmap_encoder();
    if (!enc) return gpch::fail(ctx, GPCH_CUDA_ERROR, "cuTensorMapEncodeTiled not available");
    cuuint64_t dims[2] = {(cuuint64_t)width, (cuuint64_t)m};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)BOX_K, (cuuint32_t)BM};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return gpch::fail(ctx, GPCH_CUDA_ERROR, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return GPCH_OK;
}

// Tensor map over the nb x nb FP32 tile at L (column-major, ld ldl; L and
// ldl * 4 multiples of 16 bytes) in boxes of TI_BOX rows x 32 columns, no
// swizzle; rows and columns past nb read as zeros.
gpch_status make_tile_map_f32(gpch_ctx *ctx, CUtensorMap *map, const float *L, int64_t nb, int64_t ldl)
{
    auto enc = gpch::tc::tmap_encoder();
    if (!enc) return gpch::fail(ctx, GPCH_CUDA_ERROR, "cuTensorMapEncodeTiled not available");
    cuuint64_t dims[2] = {(cuuint64_t)nb, (cuuint64_t)nb};
    cuuint64_t strides[1] = {(cuuint64_t)ldl * 4};
    cuuint32_t box[2] = {(cuuint32_t)TI_BOX, 32u};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(L), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return gpch::fail(ctx, GPCH_CUDA_ERROR, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return GPCH_OK;
}

struct LowprecBuffers {
    __nv_bfloat16 *hi = nullptr;   // the 16-bit copy (binary16 data under SPLIT_F16), layout of kpos()
    int *err = nullptr;
    int *scale = nullptr;   // SPLIT_F16: [0] largest |entry| (FP32 bits), [1] scale exponent
    int64_t ld = 0;         // row stride (positions) of hi
    bool fixed_scale = false;   // scale[0] already holds the bound; do not rescan the panel
};

// Round the FP32 panel P (m x k) to its 16-bit K-major copy: row i, K
// column col0 + c at position kpos(col0 + c) of hi + i * buf.ld
// (zero-padded up to a multiple of 64 columns; col0 a multiple of 64).
gpch_status panel_convert(gpch_ctx *ctx, int64_t m, int k, const float *P, int64_t ldp, int prec,
                          const LowprecBuffers &buf, int64_t col0, cudaStream_t st)
{
    const int kp = (k + BK - 1) / BK * BK;
    dim3 grid((unsigned)((m + 63) / 64), (unsigned)(kp / 64));
    if (prec == GPCH_PREC_SPLIT_F16) {
        if (!buf.fixed_scale) {
            GPCH_CUDA(ctx, cudaMemsetAsync(buf.scale, 0, 2 * sizeof(int), st));
            panel_absmax_kernel<<<grid, 256, 0, st>>>(P, ldp, m, k, reinterpret_cast<unsigned *>(buf.scale));
            GPCH_LAUNCH_CHECK(ctx);
        }
        panel_to_f16_kernel<<<grid, 256, 0, st>>>(P, ldp, m, k, kp, reinterpret_cast<__half *>(buf.hi) + 2 * col0,
                                                  buf.scale, buf.ld);
        GPCH_LAUNCH_CHECK(ctx);
        return GPCH_OK;
    }
    const bool split = prec == GPCH_PREC_SPLIT_BF16;
    panel_to_bf16_kernel<<<grid, 256, 0, st>>>(P, ldp, m, k, kp, buf.hi + kpos(split, col0), split ? 1 : 0, buf.ld);
    GPCH_LAUNCH_CHECK(ctx);
    return GPCH_OK;
}

// C_lower (m x m FP32) -= P P^T on the tile columns [tk0, tk1) of the
// 128 x 128 tile grid (tk1 < 0: to the end), from the 16-bit copy in buf:
// rows 0 .. m-1 (row stride buf.ld), K columns [k_off, k_off + k);
// only C columns below ncol (< 0: m) are written.  panel_k > 0: the K range
// is a sequence of panels of that many columns, subtracted one at a time
// (panel_k must divide the padded k).
// One update of the lower trapezoid restricted to tile columns [tk0, tk1)
// (see syrk_tc_kernel), for syrk_tc_launch.
struct SyrkUpdate {
    int64_t m;
    int k;
    int64_t k_off;
    float *C;
    LowprecBuffers buf;
    int64_t ncol = -1;   // columns at or past ncol are not written (-1: m)
};

// C_lower -= P P^T for one update u, or for u and a second update u2 of
// another block column in the same grid (with u2.m > 0; the same ldc, tile
// columns and panel_k).
gpch_status syrk_tc_launch_pair(gpch_ctx *ctx, const SyrkUpdate &u, const SyrkUpdate &u2, int64_t ldc, int prec,
                                int64_t tk0, int64_t tk1, cudaStream_t st, int panel_k)
{
    const bool split = prec != GPCH_PREC_BF16;
    const bool f16 = prec == GPCH_PREC_SPLIT_F16;
    struct Shape {
        int64_t tiles = 0, t1 = 0, ncol = 0;
        int kp = 0;
        double work = 0.0;
        CUtensorMap map;
    };
    auto shape = [&](const SyrkUpdate &v, Shape &o) -> gpch_status {
        o.kp = (v.k + BK - 1) / BK * BK;
        const int64_t T = (v.m + BM - 1) / BM;
        const int64_t t1 = (tk1 < 0 || tk1 > T) ? T : tk1;
        o.t1 = t1;
        if (tk0 >= t1) return GPCH_OK;
        GPCH_CHECK(make_panel_map(ctx, &o.map, v.buf.hi, v.m, kpos(split, v.k_off + o.kp), v.buf.ld, f16));
        auto offset = [&](int64_t c) { return c * T - c * (c - 1) / 2; };
        o.tiles = offset(t1) - offset(tk0);
        // algorithmic work: the lower-triangle entries of the updated columns
        o.ncol = (v.ncol < 0 || v.ncol > v.m) ? v.m : v.ncol;
        const int64_t cA = tk0 * BN, cB = (t1 * BN < o.ncol) ? t1 * BN : o.ncol;
        const double cols_entries =
            (double)(cB - cA) * (double)v.m - ((double)cB * (cB - 1) - (double)cA * (cA - 1)) / 2.0;
        o.work = 2.0 * (double)v.k * cols_entries * (split ? 3.0 : 1.0);
        return GPCH_OK;
    };
    Shape a, b;
    GPCH_CHECK(shape(u, a));
    if (u2.m > 0) GPCH_CHECK(shape(u2, b));
    if (a.tiles == 0 && b.tiles == 0) return GPCH_OK;
    static gpch::DeviceOnce attr_once;
    GPCH_CHECK(gpch::once_per_device(ctx, attr_once, [&]() -> gpch_status {
        GPCH_CUDA(ctx, cudaFuncSetAttribute(syrk_tc_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
        return GPCH_OK;
    }));
    gpch::PhaseScope ph(ctx, GPCH_PHASE_MIXED_TRAILING, st, a.work + b.work);
    // the C-tile prefetch needs 16-byte aligned columns
    const bool al = (uintptr_t)u.C % 16 == 0 && (u2.m <= 0 || (uintptr_t)u2.C % 16 == 0);
    const int prefetch_c = (al && ldc % 4 == 0) ? 1 : 0;
    // a first update without tiles hands the whole grid to the second
    const bool only2 = a.tiles == 0;
    const SyrkUpdate &f = only2 ? u2 : u;
    const Shape &fa = only2 ? b : a;
    const SyrkSecond sp = (only2 || b.tiles == 0) ? SyrkSecond{nullptr, 0, 0, 0, 0, 0}
                                                  : SyrkSecond{u2.C, u2.m, b.ncol, a.tiles, b.kp, (int)u2.k_off};
    // tile columns of the enumeration: the wider of the two (an update with
    // fewer tile rows than that has all its tiles in the leading triangle,
    // which the enumeration lays out the same way for any width)
    const int64_t tk1k = (a.t1 > b.t1) ? a.t1 : b.t1;
    syrk_tc_kernel<0><<<(unsigned)(a.tiles + b.tiles), TC_THREADS, TC_SMEM, st>>>(
        fa.map, (only2 || b.tiles == 0) ? fa.map : b.map, f.m, fa.kp, split ? 1 : 0, f.C, ldc, tk0, tk1k, f.buf.err,
        prefetch_c, f16 ? 1 : 0, f16 ? f.buf.scale : nullptr, (int)f.k_off, fa.ncol, panel_k > 0 ? panel_k : fa.kp,
        nullptr, nullptr, 0, nullptr, sp);
    GPCH_LAUNCH_CHECK(ctx);
    return GPCH_OK;
}

gpch_status syrk_tc_launch(gpch_ctx *ctx, int64_t m, int k, int64_t k_off, float *C, int64_t ldc, int prec,
                           const LowprecBuffers &buf, int64_t tk0, int64_t tk1, cudaStream_t st, int64_t ncol = -1,
                           int panel_k = 0)
{
    return syrk_tc_launch_pair(ctx, SyrkUpdate{m, k, k_off, C, buf, ncol}, SyrkUpdate{0, 0, 0, nullptr, buf}, ldc,
                               prec, tk0, tk1, st, panel_k);
}

// C (m x nq FP32, ldc) = P Q^T on tensor cores from split-f16 copies: P in
// pb (rows 0 .. m-1, K columns 0 .. k-1, row stride pb.ld, scale word
// pb.scale), Q in qb likewise (nq rows); nq <= k.  One CTA per 128 x 128
// tile of C.  out (optional): C's own split-f16 copy, row r and column c at
// position kpos(out_col + c) of out->hi + r * out->ld (out_col a multiple of
// 32), scaled by out->scale.  subtract:
// C -= P Q^T instead (no copy is written).  acc_k > 0 (dividing the padded
// k): products summed in the tensor-core accumulator per piece of acc_k
// before the FP32 running sum.
gpch_status panel_gemm_tc_launch(gpch_ctx *ctx, int64_t m, int64_t nq, int k, float *C, int64_t ldc,
                                 const LowprecBuffers &pb, const LowprecBuffers &qb, cudaStream_t st,
                                 const LowprecBuffers *out = nullptr, int64_t out_col = 0, bool subtract = false,
                                 int acc_k = 0)
{
    if (m <= 0 || nq <= 0) return GPCH_OK;
    const int kp = (k + BK - 1) / BK * BK;
    CUtensorMap mp, mq;
    GPCH_CHECK(make_panel_map(ctx, &mp, pb.hi, m, kpos(true, kp), pb.ld, true));
    GPCH_CHECK(make_panel_map(ctx, &mq, qb.hi, nq, kpos(true, kp), qb.ld, true));
    static gpch::DeviceOnce attr_once;
    GPCH_CHECK(gpch::once_per_device(ctx, attr_once, [&]() -> gpch_status {
        GPCH_CUDA(ctx, cudaFuncSetAttribute(syrk_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
        GPCH_CUDA(ctx, cudaFuncSetAttribute(syrk_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
        return GPCH_OK;
    }));
    const int64_t tr = (m + BM - 1) / BM, tc = (nq + BN - 1) / BN;
    auto kern = subtract ? syrk_tc_kernel<2> : syrk_tc_kernel<1>;
    const int prefetch_c = (subtract && (uintptr_t)C % 16 == 0 && ldc % 4 == 0) ? 1 : 0;
    kern<<<(unsigned)(tr * tc), TC_THREADS, TC_SMEM, st>>>(
        mp, mq, m, kp, 1, C, ldc, 0, tc, pb.err, prefetch_c, 1, pb.scale, 0, nq,
        (acc_k > 0 && kp % acc_k == 0) ? acc_k : kp, qb.scale,
        out ? reinterpret_cast<__half *>(out->hi) + kpos(true, out_col) : nullptr, out ? out->ld : 0,
        out ? out->scale : nullptr, SyrkSecond{nullptr, 0, 0, 0, 0, 0});
    GPCH_LAUNCH_CHECK(ctx);
    return GPCH_OK;
}

// C_lower (m x m FP32) -= P P^T with P (m x k FP32) on tensor cores.
gpch_status syrk_lowprec_enqueue(gpch_ctx *ctx, int64_t m, int k, const float *P, int64_t ldp, float *C,
                                 int64_t ldc, int prec, const LowprecBuffers &buf, cudaStream_t st)
{
    if (m <= 0 || k <= 0) return GPCH_OK;
    GPCH_CHECK(panel_convert(ctx, m, k, P, ldp, prec, buf, 0, st));
    return syrk_tc_launch(ctx, m, k, 0, C, ldc, prec, buf, 0, -1, st);
}

}  // namespace

namespace gpch {

// Workspace layout of the mixed factor for n, tile.
struct MixedWs {
    double *D, *Linv;
    float *lss;   // step 1: a diagonal 32 x 32 block on its way into W
    float *Linv32;
    int64_t *info;
    __nv_bfloat16 *hi;        // 16-bit copies of all panels: row i, K column c at kpos(c) of hi + i * kpos(kpa)
    int *err;
    int *scale;               // SPLIT_F16 scale word of the whole factor
    // step 2 on tensor cores (SPLIT_F16): L_jj^-T, 16-bit copies of its
    // transpose's rows and of the panel before the solve, their scale words
    float *Tid;
    __nv_bfloat16 *thi, *phi;   // split-f16 copies, row stride 2 * tile
    int *tscale, *pscale;
};

static MixedWs carve_mixed(Carver &cv, int64_t n, int tile)
{
    MixedWs w;
    w.info = cv.take<int64_t>(1);
    w.err = cv.take<int>(4);
    w.D = cv.take<double>((size_t)tile * tile);
    w.lss = cv.take<float>(32 * 32);
    w.Linv = cv.take<double>((size_t)(tile / LEAF) * LEAF * LEAF);
    w.Linv32 = cv.take<float>((size_t)(tile / LEAF) * LEAF * LEAF);
    const int64_t kpa = (n + BK - 1) / BK * BK;
    w.hi = cv.take<__nv_bfloat16>((size_t)n * 2 * kpa);
    w.scale = cv.take<int>(2);
    w.Tid = cv.take<float>((size_t)tile * tile);
    w.thi = cv.take<__nv_bfloat16>((size_t)tile * 2 * tile);
    w.phi = cv.take<__nv_bfloat16>((size_t)n * 2 * tile);
    w.tscale = cv.take<int>(2);
    w.pscale = cv.take<int>(2);
    return w;
}

size_t mixed_ws_bytes(int64_t n, int tile)
{
    Carver dry(nullptr);
    carve_mixed(dry, n, tile);
    return dry.off;
}

// Enqueue the low-precision factorization of W (FP32, n x n lower, ldw),
// which already holds A + shift I.  info/err live in the workspace; the
// caller reads them after the stream synchronizes.
//
// Step 3 is applied left-looking, one block column at a time, split over two
// streams.  Block column J+1 receives panel J's product on the critical
// stream (highest priority) right after that panel is solved and copied, so
// that its diagonal tile can be factored next.  Block column J+2 receives
// the products of all panels 0..J in one long-K pass on the second stream
// (lowest priority), which runs while the critical stream factors and
// solves block column J+1.  Every panel's 16-bit copy stays in one buffer
// of n rows (row i, K column c at kpos(c) of row i), so a pass reads the panels it
// needs as one K range.  Each entry of C is read and written twice (once per
// stream) instead of once per panel, and the critical stream waits only for
// the block it needs next.
gpch_status mixed_factor_enqueue(gpch_ctx *ctx, int64_t n, int tile, float *W, int64_t ldw, int prec, void *wsbase,
                                 int64_t **info_out, int **err_out, cudaStream_t st, const MixedInit *init)
{
    Carver cv(wsbase);
    MixedWs w = carve_mixed(cv, n, tile);
    *info_out = w.info;
    *err_out = w.err;
    GPCH_CHECK(aux_stream(ctx));
    cudaStream_t caller = st, sb = ctx->aux;
    st = ctx->crit;   // the critical chain runs at the highest priority
    GPCH_CUDA(ctx, cudaMemsetAsync(w.info, 0, sizeof(int64_t), caller));
    GPCH_CUDA(ctx, cudaMemsetAsync(w.err, 0, 4 * sizeof(int), caller));
    const int64_t ncols = (n + tile - 1) / tile;
    const int64_t kpa = (n + BK - 1) / BK * BK;
    const bool split = prec != GPCH_PREC_BF16;
    LowprecBuffers all;
    all.hi = w.hi;
    all.err = w.err;
    all.scale = w.scale;
    all.ld = kpos(split, kpa);
    if (prec == GPCH_PREC_SPLIT_F16) {
        // one scale for every panel, from |L_ij| <= sqrt(max_i W_ii)
        if (init)
            factor_scale_from_a_kernel<<<1, 256, 0, caller>>>(n, init->A, init->lda, init->shift, w.scale, w.pscale);
        else
            factor_scale_kernel<<<1, 256, 0, caller>>>(n, W, ldw, w.scale, w.pscale);
        GPCH_LAUNCH_CHECK(ctx);
        all.fixed_scale = true;
    }
    // the fused panel kernel needs 16-byte aligned columns of W
    const bool panel_fused = ((uintptr_t)W % 16 == 0) && (ldw % 4 == 0);
    // step 2 as a tensor-core product (SPLIT_F16; the identity solve uses
    // the fused panel kernel, and the 16-bit panel copies have a row stride
    // of `tile` elements, a multiple of 64)
    const bool tc_panel = prec == GPCH_PREC_SPLIT_F16 && panel_fused && tile <= TI_MAXN && tile % BK == 0;
    if (tc_panel) {
        static gpch::DeviceOnce inv_once;
        GPCH_CHECK(gpch::once_per_device(ctx, inv_once, [&]() -> gpch_status {
            GPCH_CUDA(ctx, cudaFuncSetAttribute(tri_inv_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)TI_SMEM));
            return GPCH_OK;
        }));
    }
    if (panel_fused) {
        static gpch::DeviceOnce pn_once;
        GPCH_CHECK(gpch::once_per_device(ctx, pn_once, [&]() -> gpch_status {
            GPCH_CUDA(ctx, cudaFuncSetAttribute(panel_trsm_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)PN_SMEM));
            return GPCH_OK;
        }));
    }
    cudaEvent_t ev_conv = ctx->aux_ev[0], ev_start = ctx->aux_ev[2], ev_done = ctx->aux_ev[3],
                ev_side = ctx->aux_ev[4], ev_pan1 = ctx->aux_ev[5];
    // ev_ready[X % 2]: the second stream's passes over block column X are done
    cudaEvent_t ev_ready[2] = {ctx->aux_ev[1], ctx->aux_ev[6]};
    cudaStream_t sc = ctx->side;
    bool side_pending = false, next_pre_conv = false;
    GPCH_CUDA(ctx, cudaEventRecord(ev_start, caller));
    GPCH_CUDA(ctx, cudaStreamWaitEvent(st, ev_start, 0));
    GPCH_CUDA(ctx, cudaStreamWaitEvent(sb, ev_start, 0));
    GPCH_CUDA(ctx, cudaStreamWaitEvent(sc, ev_start, 0));
    // the input pass, block column by block column on its own stream:
    // block column J is in W once pre_ev[J] has fired (the critical stream
    // waits for J + 1 at step J, the second stream for J + 3)
    const int64_t nbc = (n + tile - 1) / tile;
    if (init) {
        if ((int64_t)ctx->pre_ev.size() < nbc + 1) {
            ctx->pre_ev.reserve((size_t)(nbc + 1));
            while ((int64_t)ctx->pre_ev.size() < nbc + 1) {
                cudaEvent_t e = nullptr;
                GPCH_CUDA(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
                ctx->pre_ev.push_back(e);
            }
        }
        cudaStream_t sp = ctx->pre;
        GPCH_CUDA(ctx, cudaStreamWaitEvent(sp, ev_start, 0));
        GPCH_CUDA(ctx, cudaMemsetAsync(init->anorm, 0, sizeof(double), sp));
        const int64_t nchunk = (n + NW_ROWS - 1) / NW_ROWS, nstrip_all = (n + NW_COLS - 1) / NW_COLS;
        float *part = init->norm_ws, *colpart = init->norm_ws + nstrip_all * n;
        for (int64_t J = 0; J < nbc; ++J) {
            const int64_t j0 = J * tile, j1 = (n < j0 + tile) ? n : j0 + tile;
            const int64_t s0 = j0 / NW_COLS, s1 = (j1 + NW_COLS - 1) / NW_COLS;
            init_w_norm_kernel<<<dim3((unsigned)(s1 - s0), (unsigned)nchunk), NW_THREADS, 0, sp>>>(
                n, init->A, init->lda, W, ldw, init->shift, part, colpart, s0, init->packed, init->ebias);
            GPCH_LAUNCH_CHECK(ctx);
            GPCH_CUDA(ctx, cudaEventRecord(ctx->pre_ev[J], sp));
        }
        norm_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, sp>>>(n, part, colpart, init->anorm);
        GPCH_LAUNCH_CHECK(ctx);
        GPCH_CUDA(ctx, cudaEventRecord(ctx->pre_ev[nbc], sp));
    }
    auto wait_cols = [&](cudaStream_t s, int64_t J) -> gpch_status {
        if (init) GPCH_CUDA(ctx, cudaStreamWaitEvent(s, ctx->pre_ev[J < nbc ? J : nbc - 1], 0));
        return GPCH_OK;
    };
    const int64_t blk_cols = (tile + BN - 1) / BN;   // tile columns of one block column
    // K columns (whole panels) per launch of the long pass: longer launches
    // read and write C fewer times and leave fewer partial waves (at
    // n = 32768, 2 panels: 76.7 ms per solve, 4: 69, 8 to 64: 65-68), while
    // a bound keeps a CTA's lifetime, and so the wait of the critical
    // stream's tensor-core launches for a free slot, bounded at large n
    const int64_t LEFT_K = 16 * (int64_t)tile;
    // products summed in the tensor-core accumulator before they are added
    // (in FP32, rounding to nearest) to the running sum: half a panel when
    // that is a whole number of 64-column K blocks
    const int acc_k = (tile % (2 * BK) == 0) ? tile / 2 : tile;
    for (int64_t J = 0; J < ncols; ++J) {
        const int64_t j0 = J * tile;
        const int64_t nj = (n - j0 < tile) ? n - j0 : tile;
        float *Wjj = W + j0 + j0 * ldw;
        GPCH_CHECK(wait_cols(st, J + 1));
        {
            // step 1 in FP32: one left-looking launch per 32-column block
            PhaseScope ph1(ctx, GPCH_PHASE_DIAG, st, (double)nj * nj * nj / 3.0);
            int prev = -1;   // block column whose diagonal block waits in w.lss
            for (int c0 = 0; c0 < (int)nj; c0 += 32) {
                const int64_t mr = nj - c0 - ((nj - c0 < 32) ? nj - c0 : 32);
                const unsigned grid = mr > 0 ? (unsigned)((mr + 31) / 32) : 1u;
                GPCH_CUDA(ctx, gpch::launch_pdl(diag_step_kernel, dim3(grid), dim3(DS_THREADS), 0, st, Wjj, ldw,
                                                (int)nj, c0, j0, w.info, w.lss, prev));
                GPCH_LAUNCH_CHECK(ctx);
                prev = grid > 1 ? c0 : -1;
            }
        }
        if (!tc_panel) {
            // FP64 copy of the factored tile for the FP32 inverses of its 64 x 64 blocks
            tile_f32_to_f64<<<dim3(1, (unsigned)nj), 256, 0, st>>>(nj, Wjj, ldw, w.D, tile);
            GPCH_LAUNCH_CHECK(ctx);
        }
        const int64_t m = n - j0 - nj;
        if (m <= 0) continue;
        float *Pan = W + (j0 + nj) + j0 * ldw;
        // the panel's rows below block column J's... the side stream's part
        // of step J-1 (block column J below its tile) must be complete
        if (side_pending) GPCH_CUDA(ctx, cudaStreamWaitEvent(st, ev_side, 0));
        side_pending = false;
        const bool pre_conv = next_pre_conv;   // the side stream made this panel's first 16-bit rows
        next_pre_conv = false;
        // tensor-core panel with look-ahead: rows [0, m1) of the panel (the
        // rows of block column J+1) on the critical stream, the others on
        // the side stream
        const int64_t m1 = tc_panel ? (m < nj ? m : nj) : m, mr = m - m1;
        {
            // step 2 in FP32 against FP32 inverses of the tile's 64 x 64
            // diagonal blocks (computed from the FP64 factor)
            PhaseScope ph2(ctx, GPCH_PHASE_PANEL, st, (double)m * nj * nj);
            if (!tc_panel) {
                inv_blocks_f32_kernel<<<(unsigned)((nj + LEAF - 1) / LEAF), 256, 0, st>>>(w.D, tile, nj, w.Linv,
                                                                                         w.Linv32);
                GPCH_LAUNCH_CHECK(ctx);
            }
            if (tc_panel) {
                // X = P L_jj^-T as one tensor-core product: L_jj^-T by the
                // FP32 solve of the identity (column-major, so its columns
                // are the rows of L_jj^-1, the K-major right operand), both
                // operands split into scaled binary16 head and tail
                const int kpj = (int)((nj + BK - 1) / BK * BK);
                CUtensorMap tmT;
                GPCH_CHECK(make_tile_map_f32(ctx, &tmT, Wjj, nj, ldw));
                // the inverse's scale word starts at 0 (cleared by the side
                // stream at the end of the previous step when it ran)
                if (!pre_conv) GPCH_CUDA(ctx, cudaMemsetAsync(w.tscale, 0, 2 * sizeof(int), st));
                tri_inv_f32_kernel<<<(unsigned)((nj + TI_COLS - 1) / TI_COLS), TI_THREADS, TI_SMEM, st>>>(
                    tmT, (int)nj, w.Tid, tile, w.err, reinterpret_cast<unsigned *>(w.tscale));
                GPCH_LAUNCH_CHECK(ctx);
                // rows of L_jj^-1 (stored column-major) become the K-major rows
                panel_to_f16_kernel<<<dim3((unsigned)((nj + 63) / 64), (unsigned)(kpj / 64)), 256, 0, st>>>(
                    w.Tid, tile, nj, (int)nj, kpj, reinterpret_cast<__half *>(w.thi), w.tscale, 2 * tile);
                GPCH_LAUNCH_CHECK(ctx);
                if (!pre_conv) {
                    panel_to_f16_kernel<<<dim3((unsigned)((m1 + 63) / 64), (unsigned)(kpj / 64)), 256, 0, st>>>(
                        Pan, ldw, m1, (int)nj, kpj, reinterpret_cast<__half *>(w.phi), w.pscale, 2 * tile);
                    GPCH_LAUNCH_CHECK(ctx);
                }
                LowprecBuffers pbuf = all, qbuf = all;
                pbuf.hi = w.phi;
                pbuf.scale = w.pscale;
                pbuf.ld = 2 * tile;
                qbuf.hi = w.thi;
                qbuf.scale = w.tscale;
                qbuf.ld = 2 * tile;
                LowprecBuffers obuf = all;   // the panel's 16-bit copy, written by the product
                obuf.hi = all.hi + (j0 + nj) * all.ld;
                GPCH_CHECK(panel_gemm_tc_launch(ctx, m1, nj, (int)nj, Pan, ldw, pbuf, qbuf, st, &obuf, j0));
                if (mr > 0) {
                    // side stream: the other rows of the panel, then their
                    // product with block column J+1 (after the second
                    // stream's update of that block column, which writes
                    // the same entries)
                    GPCH_CUDA(ctx, cudaEventRecord(ev_pan1, st));
                    GPCH_CUDA(ctx, cudaStreamWaitEvent(sc, ev_pan1, 0));
                    PhaseScope phs(ctx, GPCH_PHASE_PANEL, sc, (double)mr * nj * nj);
                    panel_to_f16_kernel<<<dim3((unsigned)((mr + 63) / 64), (unsigned)(kpj / 64)), 256, 0, sc>>>(
                        Pan + m1, ldw, mr, (int)nj, kpj, reinterpret_cast<__half *>(w.phi) + m1 * 2 * tile, w.pscale,
                        2 * tile);
                    GPCH_LAUNCH_CHECK(ctx);
                    LowprecBuffers pr = pbuf, orr = obuf;
                    pr.hi = w.phi + m1 * 2 * tile;
                    orr.hi = obuf.hi + m1 * all.ld;
                    GPCH_CHECK(panel_gemm_tc_launch(ctx, mr, nj, (int)nj, Pan + m1, ldw, pr, qbuf, sc, &orr, j0));
                    if (J >= 1) GPCH_CUDA(ctx, cudaStreamWaitEvent(sc, ev_ready[(J + 1) % 2], 0));
                    // block column J+1, rows below its tile, -= (panel rows m1..) (panel rows 0..m1)^T
                    LowprecBuffers rb = all, cb = all;
                    rb.hi = all.hi + (j0 + nj + m1) * all.ld + kpos(true, j0);
                    cb.hi = all.hi + (j0 + nj) * all.ld + kpos(true, j0);
                    GPCH_CHECK(panel_gemm_tc_launch(ctx, mr, m1, (int)nj, W + (j0 + nj + m1) + (j0 + nj) * ldw, ldw,
                                                    rb, cb, sc, nullptr, 0, true, acc_k));
                    // block column J+1 below its tile is final now: the
                    // 16-bit copy of its first rows (panel J+1 before the
                    // solve) and the clearing of the next inverse's scale
                    // word leave the critical stream
                    const int64_t j1 = j0 + nj, nj1 = (n - j1 < tile) ? n - j1 : tile, mn = n - j1 - nj1;
                    next_pre_conv = mn > 0;
                    if (next_pre_conv) {
                        const int64_t m1n = (mn < nj1) ? mn : nj1;
                        const int kpn = (int)((nj1 + BK - 1) / BK * BK);
                        GPCH_CUDA(ctx, cudaMemsetAsync(w.tscale, 0, 2 * sizeof(int), sc));
                        panel_to_f16_kernel<<<dim3((unsigned)((m1n + 63) / 64), (unsigned)(kpn / 64)), 256, 0, sc>>>(
                            W + (j1 + nj1) + j1 * ldw, ldw, m1n, (int)nj1, kpn, reinterpret_cast<__half *>(w.phi),
                            w.pscale, 2 * tile);
                        GPCH_LAUNCH_CHECK(ctx);
                    }
                    GPCH_CUDA(ctx, cudaEventRecord(ev_side, sc));
                    side_pending = true;
                }
            } else if (panel_fused && nj <= PN_MAXK) {
                panel_trsm_f32_kernel<<<(unsigned)((m + PN_ROWS - 1) / PN_ROWS), PN_THREADS, PN_SMEM, st>>>(
                    Pan, ldw, m, (int)nj, Wjj, ldw, w.Linv32, w.info);
                GPCH_LAUNCH_CHECK(ctx);
            } else for (int64_t c0 = 0; c0 < nj; c0 += LEAF) {
                const int nc = (int)((nj - c0 < LEAF) ? nj - c0 : LEAF);
                float *Xc = Pan + c0 * ldw;
                GPCH_CHECK(launch_trsm<float>(ctx, Xc, ldw, m, nc, w.Linv + (c0 / LEAF) * LEAF * LEAF, w.info, st));
                const int64_t rest = nj - c0 - nc;
                if (rest > 0)
                    GPCH_CHECK(launch_gemm<float>(ctx, false, m, rest, nc, Xc, ldw, Wjj + (c0 + nc) + c0 * ldw, ldw,
                                                  Pan + (c0 + nc) * ldw, ldw, w.info, st));
            }
        }
        // step 3: the panel's 16-bit copy (rows j0 + nj.., K columns j0..)
        LowprecBuffers pb = all;
        pb.hi = all.hi + (j0 + nj) * all.ld;
        if (!tc_panel) GPCH_CHECK(panel_convert(ctx, m, (int)nj, Pan, ldw, prec, pb, j0, st));
        GPCH_CUDA(ctx, cudaEventRecord(ev_conv, side_pending ? sc : st));
        // block column J+1 <- panel J, after it received panels 0..J-1 (with
        // the look-ahead only its diagonal tile here; the side stream does
        // the rows below)
        if (J >= 1) GPCH_CUDA(ctx, cudaStreamWaitEvent(st, ev_ready[(J + 1) % 2], 0));
        GPCH_CHECK(syrk_tc_launch(ctx, m1, (int)nj, j0, W + (j0 + nj) * (1 + ldw), ldw, prec, pb, 0, blk_cols, st,
                                  tile, acc_k));
        // second stream, two block columns ahead of the critical stream:
        // block column J+2 <- panel J (it already has panels 0..J-1), then
        // block column J+3 <- panels 0..J in one long-K pass
        if (m > tile) {
            GPCH_CUDA(ctx, cudaStreamWaitEvent(sb, ev_conv, 0));
            GPCH_CHECK(wait_cols(sb, J + 3));
            const int64_t r2 = j0 + nj + tile, m2 = n - r2;
            LowprecBuffers qb = all;
            qb.hi = all.hi + r2 * all.ld;
            const SyrkUpdate short_pass{m2, (int)nj, j0, W + r2 * (1 + ldw), qb, tile};
            if (m > 2 * tile) {
                // the short pass shares one grid with the first piece of the
                // long pass, whose tiles fill the waves the short tiles leave
                const int64_t r3 = r2 + tile, m3 = n - r3, K = j0 + nj;
                LowprecBuffers qb3 = all;
                qb3.hi = all.hi + r3 * all.ld;
                const int64_t kk0 = (K < LEFT_K) ? K : LEFT_K;
                GPCH_CHECK(syrk_tc_launch_pair(ctx, short_pass,
                                               SyrkUpdate{m3, (int)kk0, 0, W + r3 * (1 + ldw), qb3, tile}, ldw, prec, 0,
                                               blk_cols, sb, acc_k));
                GPCH_CUDA(ctx, cudaEventRecord(ev_ready[(J + 2) % 2], sb));
                for (int64_t k0 = kk0; k0 < K; k0 += LEFT_K) {
                    const int64_t kk = (K - k0 < LEFT_K) ? K - k0 : LEFT_K;
                    GPCH_CHECK(syrk_tc_launch(ctx, m3, (int)kk, k0, W + r3 * (1 + ldw), ldw, prec, qb3, 0, blk_cols,
                                              sb, tile, acc_k));
                }
            } else {
                GPCH_CHECK(syrk_tc_launch(ctx, m2, (int)nj, j0, W + r2 * (1 + ldw), ldw, prec, qb, 0, blk_cols, sb,
                                          tile, acc_k));
                GPCH_CUDA(ctx, cudaEventRecord(ev_ready[(J + 2) % 2], sb));
            }
        }
    }
    // the second stream's last pass (and the side stream, and the input
    // pass's norm) before the caller
    if (init) GPCH_CUDA(ctx, cudaStreamWaitEvent(caller, ctx->pre_ev[nbc], 0));
    GPCH_CUDA(ctx, cudaEventRecord(ev_ready[0], sb));
    GPCH_CUDA(ctx, cudaStreamWaitEvent(caller, ev_ready[0], 0));
    if (side_pending) GPCH_CUDA(ctx, cudaStreamWaitEvent(caller, ev_side, 0));
    GPCH_CUDA(ctx, cudaEventRecord(ev_done, st));
    GPCH_CUDA(ctx, cudaStreamWaitEvent(caller, ev_done, 0));
    return GPCH_OK;
}

size_t anorm_ws_floats(int64_t n)
{
    return (size_t)((n + NW_COLS - 1) / NW_COLS + (n + NW_ROWS - 1) / NW_ROWS) * (size_t)n;
}

// W = A + shift I (FP32 lower triangle); with anorm and norm_ws, also
// ||A||_inf into *anorm (zeroed here), through norm_ws (anorm_ws_floats(n)
// floats).
gpch_status mixed_init_enqueue(gpch_ctx *ctx, int64_t n, const double *A, int64_t lda, float *W, int64_t ldw,
                               double shift, cudaStream_t st, double *anorm, float *norm_ws)
{
    if ((anorm == nullptr) != (norm_ws == nullptr))
        return gpch::fail(ctx, GPCH_INVALID_ARG, "the norm needs both its output and its workspace");
    if (anorm) {
        GPCH_CUDA(ctx, cudaMemsetAsync(anorm, 0, sizeof(double), st));
        const int64_t nstrip = (n + NW_COLS - 1) / NW_COLS, nchunk = (n + NW_ROWS - 1) / NW_ROWS;
        float *part = norm_ws, *colpart = norm_ws + nstrip * n;
        init_w_norm_kernel<<<dim3((unsigned)nstrip, (unsigned)nchunk), NW_THREADS, 0, st>>>(n, A, lda, W, ldw, shift,
                                                                                           part, colpart, 0, nullptr,
                                                                                           0u);
        GPCH_LAUNCH_CHECK(ctx);
        norm_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, part, colpart, anorm);
        GPCH_LAUNCH_CHECK(ctx);
        return GPCH_OK;
    }
    init_w_kernel<<<(unsigned)n, 256, 0, st>>>(n, A, lda, W, ldw, shift);
    GPCH_LAUNCH_CHECK(ctx);
    return GPCH_OK;
}

}  // namespace gpch

extern "C" gpch_status gpch_syrk_lowprec(gpch_ctx *ctx, int64_t m, int64_t k, const float *P, int64_t ldp, float *C,
                                         int64_t ldc, gpch_prec prec, void *stream)
{
    GPCH_ARG(ctx, ctx != nullptr, "null context");
    GPCH_ARG(ctx, m >= 0 && k >= 0 && k <= 4096, "need m >= 0 and 0 <= k <= 4096");
    GPCH_ARG(ctx, ldp >= (m > 0 ? m : 1) && ldc >= (m > 0 ? m : 1), "ld < m");
    GPCH_ARG(ctx, prec == GPCH_PREC_BF16 || prec == GPCH_PREC_SPLIT_BF16 || prec == GPCH_PREC_SPLIT_F16,
             "prec must be BF16, SPLIT_BF16 or SPLIT_F16");
    GPCH_ARG(ctx, m < (int64_t)1 << 31, "m too large");
    if (m == 0 || k == 0) return GPCH_OK;
    GPCH_ARG(ctx, P && C, "null pointer");
    GPCH_CUDA(ctx, cudaSetDevice(ctx->device));
    const int kp = (int)((k + BK - 1) / BK * BK);
    gpch::Carver dry(nullptr);
    dry.take<int>(4);
    dry.take<__nv_bfloat16>((size_t)m * 2 * kp);
    dry.take<int>(2);
    GPCH_CHECK(gpch::ws_reserve(ctx, dry.off));
    gpch::Carver cv(ctx->ws);
    LowprecBuffers buf;
    buf.err = cv.take<int>(4);
    buf.hi = cv.take<__nv_bfloat16>((size_t)m * 2 * kp);
    buf.scale = cv.take<int>(2);
    buf.ld = kpos(prec != GPCH_PREC_BF16, kp);
    cudaStream_t st = (cudaStream_t)stream;
    GPCH_CUDA(ctx, cudaMemsetAsync(buf.err, 0, 4 * sizeof(int), st));
    GPCH_CHECK(syrk_lowprec_enqueue(ctx, m, (int)k, P, ldp, C, ldc, prec, buf, st));
    int *h = static_cast<int *>(ctx->pinned);
    GPCH_CUDA(ctx, cudaMemcpyAsync(h, buf.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    GPCH_CUDA(ctx, cudaStreamSynchronize(st));
    if (*h != 0) return gpch::fail(ctx, GPCH_TIMEOUT, "tensor-core pipeline wait gave up (code %d)", *h);
    return GPCH_OK;
}

extern "C" gpch_status gpch_chol_factor_mixed(gpch_ctx *ctx, int64_t n, int tile, const double *A, int64_t lda,
                                              gpch_prec prec, double shift, float *L, int64_t ldl, void *stream,
                                              int64_t *info)
{
    GPCH_ARG(ctx, ctx != nullptr, "null context");
    GPCH_ARG(ctx, info != nullptr, "info must not be NULL");
    *info = 0;
    GPCH_ARG(ctx, n >= 0 && lda >= (n > 0 ? n : 1) && ldl >= (n > 0 ? n : 1), "bad n / lda / ldl");
    GPCH_ARG(ctx, tile >= LEAF && tile <= 1024 && tile % LEAF == 0, "tile must be a multiple of 64 in [64, 1024]");
    GPCH_ARG(ctx, prec == GPCH_PREC_BF16 || prec == GPCH_PREC_SPLIT_BF16 || prec == GPCH_PREC_SPLIT_F16,
             "prec must be BF16, SPLIT_BF16 or SPLIT_F16");
    GPCH_ARG(ctx, shift >= 0.0, "shift must be >= 0");
    GPCH_ARG(ctx, n < (int64_t)1 << 31, "n too large");
    if (n == 0) return GPCH_OK;
    GPCH_ARG(ctx, A && L, "null pointer");
    GPCH_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    GPCH_CHECK(gpch::ws_reserve(ctx, gpch::mixed_ws_bytes(n, tile)));
    GPCH_CHECK(gpch::mixed_init_enqueue(ctx, n, A, lda, L, ldl, shift, st));
    int64_t *d_info;
    int *d_err;
    GPCH_CHECK(gpch::mixed_factor_enqueue(ctx, n, tile, L, ldl, (int)prec, ctx->ws, &d_info, &d_err, st));
    int64_t *h = static_cast<int64_t *>(ctx->pinned);
    GPCH_CUDA(ctx, cudaMemcpyAsync(h, d_info, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    GPCH_CUDA(ctx, cudaMemcpyAsync(h + 1, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    GPCH_CUDA(ctx, cudaStreamSynchronize(st));
    const int e = (int)(reinterpret_cast<int *>(h + 1)[0]);
    if (e != 0) return gpch::fail(ctx, GPCH_TIMEOUT, "tensor-core pipeline wait gave up (code %d)", e);
    *info = h[0];
    if (*info != 0) return gpch::fail(ctx, GPCH_NOT_SPD, "pivot %lld not positive", (long long)*info);
    return GPCH_OK;
}
