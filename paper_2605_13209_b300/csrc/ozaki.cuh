// ozaki.cuh -- pieces of the FP64-accurate tensor-core product (the
// error-free splitting of ozaki.cu) shared by its users: the digit layout,
// the exact rounding of a combined class sum, and the tensor map over a
// digit copy.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include "internal.cuh"
#include "tc_ptx.cuh"

namespace gpch {

// Position of digit p of K column c in a row of the digit copy: 4 boxes of
// rows; box p / 2; inside a box row, 32-column chunks of 64 positions with
// digit p % 2 at offset 32 (p % 2) -- the head/tail interleave of the
// split copies of mixed.cu, with two digits in place of head and tail.
__host__ __device__ constexpr int64_t oz_pos(int p, int64_t c) { return (c / 32) * 64 + (p & 1) * 32 + c % 32; }


// The FP64 value nearest to T 2^s for a signed integer T = H 2^28 + L
// (|H|, |L| < 2^48), rounded to nearest even, from integer operations only
// (this part runs FP64 conversions on its slow FP64 pipe).  Results outside
// FP64's normal range take the FP64 route (never for a product of two
// normal operands' digits; kept for completeness).
__device__ __forceinline__ double oz_round_scaled(long long H, long long L, int s)
{
    const __int128 T = (__int128)H * ((__int128)1 << 28) + (__int128)L;
    if (T == 0) return 0.0;
    const bool neg = T < 0;
    const unsigned __int128 U = neg ? (unsigned __int128)(-T) : (unsigned __int128)T;
    const unsigned long long hi = (unsigned long long)(U >> 64), lo = (unsigned long long)U;
    const int lz = hi ? __clzll((long long)hi) : 64 + __clzll((long long)lo);
    const int msb = 127 - lz;                       // U in [2^msb, 2^(msb+1))
    const int ex = msb + s;                         // unbiased exponent of the result
    if (ex < -1022 || ex > 1023)
        return neg ? -ldexp((double)U, s) : ldexp((double)U, s);
    // top 53 bits of U, then round to nearest even on the rest
    unsigned long long mant;
    bool round_up = false;
    if (msb <= 52) {
        mant = lo << (52 - msb);
    } else {
        const int sh = msb - 52;                    // bits below the 53
        const unsigned __int128 q = U >> sh;
        mant = (unsigned long long)q;
        const unsigned __int128 rem = U - (q << sh);
        const unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
        round_up = rem > half || (rem == half && (mant & 1ull));
    }
    unsigned long long bits = ((unsigned long long)(ex + 1023) << 52) + (mant & 0xfffffffffffffull);
    bits += round_up ? 1ull : 0ull;                 // a carry into the exponent is the right rounding
    if (neg) bits |= 0x8000000000000000ull;
    return __longlong_as_double((long long)bits);
}


// Tensor map over a digit copy: `rows` rows of `width` bf16 positions,
// boxes of 64 positions (128 bytes, 128-byte swizzle) by box_rows rows, or
// with narrow, of 32 positions (64 bytes, 64-byte swizzle).
inline gpch_status oz_map(gpch_ctx *ctx, CUtensorMap *map, const void *base, int64_t rows, int64_t width,
                          uint32_t box_rows, bool narrow = false)
{
    auto enc = gpch::tc::tmap_encoder();
    if (!enc) return gpch::fail(ctx, GPCH_CUDA_ERROR, "cuTensorMapEncodeTiled not available");
    cuuint64_t dims[2] = {(cuuint64_t)width, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)width * 2};
    cuuint32_t box[2] = {narrow ? 32u : 64u, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, narrow ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return gpch::fail(ctx, GPCH_CUDA_ERROR, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return GPCH_OK;
}

}  // namespace gpch
