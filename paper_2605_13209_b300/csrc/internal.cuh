// internal.cuh -- context, workspace arena and error plumbing shared by the
// CUDA translation units of libgpchol.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <cstdarg>
#include <cstdint>
#include <cstdio>

#include "../../include/gpchol.h"

struct gpch_ctx {
    int device = 0;
    size_t budget = 0;          // 0 = no cap
    void *ws = nullptr;         // workspace arena (device)
    size_t ws_bytes = 0;
    void *pinned = nullptr;     // small pinned host block for flags / stats
    size_t pinned_bytes = 0;
    char err[512] = {0};
};

namespace gpch {

gpch_status fail(gpch_ctx *ctx, gpch_status st, const char *fmt, ...);

// Make sure the arena holds at least `bytes`; grows it (after a device
// synchronize) if needed.  Respects the context's HBM budget.
gpch_status ws_reserve(gpch_ctx *ctx, size_t bytes);

// Bump allocator over the arena for one call: carve(bytes) returns 256-byte
// aligned slices.  Sizes are computed first (dry run), then reserved.
struct Carver {
    char *base;
    size_t off = 0;
    explicit Carver(void *b) : base(static_cast<char *>(b)) {}
    template <typename T>
    T *take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T *p = reinterpret_cast<T *>(base ? base + off : nullptr);
        off += count * sizeof(T);
        return p;
    }
};

inline int ceil_div(int64_t a, int64_t b) { return static_cast<int>((a + b - 1) / b); }

}  // namespace gpch

#define GPCH_CUDA(ctx, call)                                                        \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess)                                                      \
            return gpch::fail((ctx), GPCH_CUDA_ERROR, "%s: %s (%s:%d)", #call,      \
                              cudaGetErrorString(e_), __FILE__, __LINE__);          \
    } while (0)

#define GPCH_LAUNCH_CHECK(ctx)                                                      \
    do {                                                                            \
        cudaError_t e_ = cudaGetLastError();                                        \
        if (e_ != cudaSuccess)                                                      \
            return gpch::fail((ctx), GPCH_CUDA_ERROR, "kernel launch: %s (%s:%d)",  \
                              cudaGetErrorString(e_), __FILE__, __LINE__);          \
    } while (0)

#define GPCH_CHECK(expr)                                                            \
    do {                                                                            \
        gpch_status s_ = (expr);                                                    \
        if (s_ != GPCH_OK) return s_;                                               \
    } while (0)

#define GPCH_ARG(ctx, cond, msg)                                                    \
    do {                                                                            \
        if (!(cond)) return gpch::fail((ctx), GPCH_INVALID_ARG, "%s", (msg));       \
    } while (0)
