// internal.cuh -- context, workspace arena and error plumbing shared by the
// CUDA translation units of libgpchol.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <mutex>
#include <vector>

#include "../../include/gpchol.h"

struct gpch_timed_launch {
    cudaEvent_t start, stop;
    double work;
};

struct gpch_ctx {
    int device = 0;
    size_t budget = 0;          // 0 = no cap
    void *ws = nullptr;         // workspace arena (device)
    size_t ws_bytes = 0;
    void *pinned = nullptr;     // small pinned host block for flags / stats
    size_t pinned_bytes = 0;
    char err[512] = {0};
    int64_t launches = 0;       // kernels launched through this context
    bool timing = false;
    std::vector<gpch_timed_launch> pending[GPCH_PHASE_COUNT];
    std::vector<cudaEvent_t> event_pool;
    double phase_ms[GPCH_PHASE_COUNT] = {0};
    int64_t phase_launches[GPCH_PHASE_COUNT] = {0};
    double phase_work[GPCH_PHASE_COUNT] = {0};
    cudaStream_t aux = nullptr;          // low-priority stream for bulk overlapped work
    cudaStream_t crit = nullptr;         // high-priority stream for the critical chain
    cudaStream_t side = nullptr;         // middle priority: work the critical chain needs one step later
    cudaStream_t pre = nullptr;          // low priority: the factor's input pass, block column by block column
    std::vector<cudaEvent_t> pre_ev;     // one per block column of that pass (no timing)
    cudaEvent_t aux_ev[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
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
    // Reserve `bytes` (256-byte aligned); returns the offset from the base.
    size_t reserve(size_t bytes) {
        off = (off + 255) & ~size_t(255);
        const size_t o = off;
        off += bytes;
        return o;
    }
    template <typename T>
    T *take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T *p = reinterpret_cast<T *>(base ? base + off : nullptr);
        off += count * sizeof(T);
        return p;
    }
};

inline int ceil_div(int64_t a, int64_t b) { return static_cast<int>((a + b - 1) / b); }

cudaEvent_t take_event(gpch_ctx *ctx);

// Create the context's two internal streams (bulk at the lowest priority,
// critical chain at the highest) and their ordering events (once).
gpch_status aux_stream(gpch_ctx *ctx);

// Tile choices, by problem size: the refined solve's tile and the batched
// factors' trailing-update tile (32 or 64 rows and columns per CTA; the
// result does not depend on it, only the speed).  Defaults until the
// autotuner (autotune.cu) has measured this device or loaded its cache.
constexpr int TUNE_BUCKETS = 9;   // n <= 512, 1024, ..., 65536, larger
struct TuneTable {
    int refined_tile[TUNE_BUCKETS];
    int batch_bt[2][TUNE_BUCKETS];   // [0] FP64 batch, [1] mixed batch
    int tuned;                       // 0 defaults, 1 measured, 2 loaded
};
int tune_bucket(int64_t n);
TuneTable tune_table(int device);
void tune_set(int device, const TuneTable &t);

// Free the batched solvers' cached plans of a context (batched.cu,
// batched_mixed.cu).
void batched_release(gpch_ctx *ctx);
void batched_mixed_release(gpch_ctx *ctx);

// Batched FP64 solve launched directly, tables in the context workspace.
gpch_status batched_solve_direct(gpch_ctx *ctx, int count, const gpch_system *systems, cudaStream_t st,
                                 int64_t *info);

// Records an event pair around the launches made while it is alive, when
// timing is on; `work` is their algorithmic flops (or bytes).
struct PhaseScope {
    gpch_ctx *ctx;
    int phase;
    cudaStream_t st;
    double work;
    cudaEvent_t start = nullptr;
    PhaseScope(gpch_ctx *c, int ph, cudaStream_t s, double w) : ctx(c), phase(ph), st(s), work(w)
    {
        if (ctx->timing) {
            start = take_event(ctx);
            if (start) cudaEventRecord(start, st);
        }
    }
    ~PhaseScope()
    {
        if (start) {
            cudaEvent_t stop = take_event(ctx);
            if (stop) {
                cudaEventRecord(stop, st);
                ctx->pending[phase].push_back({start, stop, work});
            }
        }
    }
};

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
        ++(ctx)->launches;                                                          \
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

namespace gpch {

// One-time set-up per device for one call site (a kernel's shared-memory
// limit, say): cudaFuncSetAttribute applies to the current device only,
// and contexts on several host threads may reach the site together.  set()
// runs under the site's mutex the first time a context of a device gets
// here (every time for device numbers past 63); a failure leaves the device
// unmarked.
struct DeviceOnce {
    std::mutex mu;
    bool done[64] = {};
};

template <typename F>
inline gpch_status once_per_device(gpch_ctx *ctx, DeviceOnce &once, F &&set)
{
    std::lock_guard<std::mutex> lock(once.mu);
    const int d = ctx->device;
    const bool tracked = d >= 0 && d < 64;
    if (tracked && once.done[d]) return GPCH_OK;
    GPCH_CHECK(set());
    if (tracked) once.done[d] = true;
    return GPCH_OK;
}

}  // namespace gpch
