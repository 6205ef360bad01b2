// api.cu -- context lifetime, workspace arena, status strings.
#include <cstring>

#include "internal.cuh"

namespace gpch {

gpch_status fail(gpch_ctx *ctx, gpch_status st, const char *fmt, ...)
{
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
        va_end(ap);
    }
    return st;
}

gpch_status ws_reserve(gpch_ctx *ctx, size_t bytes)
{
    if (bytes <= ctx->ws_bytes) return GPCH_OK;
    if (ctx->budget && bytes > ctx->budget)
        return fail(ctx, GPCH_OOM_BUDGET, "workspace of %zu bytes exceeds the budget of %zu bytes",
                    bytes, ctx->budget);
    GPCH_CUDA(ctx, cudaSetDevice(ctx->device));
    if (ctx->ws) {
        // Work queued on any stream may still use the old arena.
        GPCH_CUDA(ctx, cudaDeviceSynchronize());
        GPCH_CUDA(ctx, cudaFree(ctx->ws));
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
    }
    size_t sz = bytes + (bytes >> 3);   // grow with some slack
    if (ctx->budget && sz > ctx->budget) sz = ctx->budget;
    cudaError_t e = cudaMalloc(&ctx->ws, sz);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->ws = nullptr;
        return fail(ctx, GPCH_OOM_BUDGET, "cudaMalloc(%zu) failed: %s", sz, cudaGetErrorString(e));
    }
    ctx->ws_bytes = sz;
    return GPCH_OK;
}

gpch_status aux_stream(gpch_ctx *ctx)
{
    if (ctx->aux) return GPCH_OK;
    int least = 0, greatest = 0;
    GPCH_CUDA(ctx, cudaDeviceGetStreamPriorityRange(&least, &greatest));
    GPCH_CUDA(ctx, cudaStreamCreateWithPriority(&ctx->aux, cudaStreamNonBlocking, least));
    GPCH_CUDA(ctx, cudaStreamCreateWithPriority(&ctx->crit, cudaStreamNonBlocking, greatest));
    GPCH_CUDA(ctx, cudaStreamCreateWithPriority(&ctx->pre, cudaStreamNonBlocking, least));
    GPCH_CUDA(ctx, cudaStreamCreateWithPriority(&ctx->side, cudaStreamNonBlocking,
                                                greatest < least ? greatest + 1 : greatest));
    for (auto &e : ctx->aux_ev) GPCH_CUDA(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return GPCH_OK;
}

cudaEvent_t take_event(gpch_ctx *ctx)
{
    if (!ctx->event_pool.empty()) {
        cudaEvent_t e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

}  // namespace gpch

extern "C" {

gpch_status gpch_create(gpch_ctx **out, int device, size_t hbm_budget_bytes)
{
    if (!out) return GPCH_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || count == 0) {
        cudaGetLastError();
        return GPCH_CUDA_ERROR;
    }
    if (device < 0 || device >= count) return GPCH_INVALID_ARG;
    gpch_ctx *ctx = new gpch_ctx();
    ctx->device = device;
    ctx->budget = hbm_budget_bytes;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaMallocHost(&ctx->pinned, 4096) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return GPCH_CUDA_ERROR;
    }
    ctx->pinned_bytes = 4096;
    *out = ctx;
    return GPCH_OK;
}

gpch_status gpch_destroy(gpch_ctx *ctx)
{
    if (!ctx) return GPCH_OK;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    gpch::batched_release(ctx);
    gpch::batched_mixed_release(ctx);
    for (auto &v : ctx->pending)
        for (auto &t : v) {
            cudaEventDestroy(t.start);
            cudaEventDestroy(t.stop);
        }
    for (auto e : ctx->event_pool) cudaEventDestroy(e);
    for (auto e : ctx->aux_ev)
        if (e) cudaEventDestroy(e);
    if (ctx->aux) cudaStreamDestroy(ctx->aux);
    if (ctx->crit) cudaStreamDestroy(ctx->crit);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    if (ctx->pre) cudaStreamDestroy(ctx->pre);
    for (auto e : ctx->pre_ev) cudaEventDestroy(e);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    delete ctx;
    return GPCH_OK;
}

const char *gpch_status_string(gpch_status s)
{
    switch (s) {
    case GPCH_OK: return "GPCH_OK";
    case GPCH_INVALID_ARG: return "GPCH_INVALID_ARG";
    case GPCH_NOT_SPD: return "GPCH_NOT_SPD";
    case GPCH_NOT_CONVERGED: return "GPCH_NOT_CONVERGED";
    case GPCH_OOM_BUDGET: return "GPCH_OOM_BUDGET";
    case GPCH_TIMEOUT: return "GPCH_TIMEOUT";
    case GPCH_CUDA_ERROR: return "GPCH_CUDA_ERROR";
    }
    return "GPCH_UNKNOWN";
}

const char *gpch_last_error(const gpch_ctx *ctx) { return ctx ? ctx->err : "no context"; }

int gpch_version(void) { return GPCH_VERSION; }

size_t gpch_workspace_bytes(const gpch_ctx *ctx) { return ctx ? ctx->ws_bytes : 0; }

int64_t gpch_launch_count(const gpch_ctx *ctx) { return ctx ? ctx->launches : 0; }

static gpch_status drain_phase(gpch_ctx *ctx, int ph)
{
    for (auto &t : ctx->pending[ph]) {
        float ms = 0.f;
        GPCH_CUDA(ctx, cudaEventSynchronize(t.stop));
        GPCH_CUDA(ctx, cudaEventElapsedTime(&ms, t.start, t.stop));
        ctx->phase_ms[ph] += ms;
        ctx->phase_launches[ph] += 1;
        ctx->phase_work[ph] += t.work;
        ctx->event_pool.push_back(t.start);
        ctx->event_pool.push_back(t.stop);
    }
    ctx->pending[ph].clear();
    return GPCH_OK;
}

gpch_status gpch_timing_enable(gpch_ctx *ctx, int enable)
{
    if (!ctx) return GPCH_INVALID_ARG;
    GPCH_CUDA(ctx, cudaSetDevice(ctx->device));
    for (int ph = 0; ph < GPCH_PHASE_COUNT; ++ph) {
        GPCH_CHECK(drain_phase(ctx, ph));
        ctx->phase_ms[ph] = 0.0;
        ctx->phase_launches[ph] = 0;
        ctx->phase_work[ph] = 0.0;
    }
    ctx->timing = enable != 0;
    return GPCH_OK;
}

gpch_status gpch_timing_read(gpch_ctx *ctx, int phase, double *total_ms, int64_t *launches, double *work)
{
    if (!ctx) return GPCH_INVALID_ARG;
    if (phase < 0 || phase >= GPCH_PHASE_COUNT) return gpch::fail(ctx, GPCH_INVALID_ARG, "bad phase %d", phase);
    GPCH_CUDA(ctx, cudaSetDevice(ctx->device));
    GPCH_CHECK(drain_phase(ctx, phase));
    if (total_ms) *total_ms = ctx->phase_ms[phase];
    if (launches) *launches = ctx->phase_launches[phase];
    if (work) *work = ctx->phase_work[phase];
    return GPCH_OK;
}

}  // extern "C"
