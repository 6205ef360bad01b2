// dense_fp64.cuh -- FP64 device building blocks used by the blocked
// Cholesky (Algorithm 1, right) and by the triangular solves.
//
// Leaf size is 64: a 64 x 64 FP64 block (32 KB) fits one CTA's shared
// memory, so the diagonal tile of any size is factored as a nest of 64-wide
// leaf steps.  On this GPU one SM retires two FP64 FMAs per clock, so these
// kernels are bound by the FP64 pipe, not by memory; they keep that pipe
// busy with 4 x 4 register tiles per thread and several CTAs per SM.
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
