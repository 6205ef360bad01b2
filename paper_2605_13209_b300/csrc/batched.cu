// batched.cu -- A10: many independent GP systems factored and solved
// together (FP64 blocked Cholesky, Algorithm 1 right, with 64-wide blocks,
// then forward/back substitution).
//
// The batch runs level-synchronously: step k of every system whose matrix
// has more than k block columns is done by one grouped launch per kernel
// kind (leaf POTRF + inverse of block (k,k), panel solve below it, SYRK/GEMM
// update of the trailing lower triangle), and likewise one grouped launch
// per block of each substitution sweep.  A per-step prefix table maps a CTA
// to (system, local task), found by binary search.  Every system is cut into
// tiles by its own size only, so its arithmetic does not depend on the
// other systems in the batch.  The whole launch sequence of a batch is
// captured once as a CUDA graph and replayed on later calls with the same
// systems.
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "dense_fp64.cuh"

namespace {

using gpch::LEAF;

struct BSys {
    double *A;
    int64_t lda;
    int64_t n;
    double *B;
    int64_t ldb;
    int nrhs;
    double *Linv;    // nblocks x 64 x 64
    double *Y;       // n x nrhs
    int64_t *info;
};

// Per-step task table: `cnt` active systems, their indices, and prefix sums
// of their task counts (length cnt + 1).
struct StepTable {
    const int *sys;
    const int64_t *pref;
    int cnt;
};

__device__ inline int find_task(const StepTable &t, int64_t task, int64_t &local)
{
    int lo = 0, hi = t.cnt - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (t.pref[mid] <= task) lo = mid;
        else hi = mid - 1;
    }
    local = task - t.pref[lo];
    return t.sys[lo];
}

__device__ inline int64_t block_rows(int64_t n, int64_t k) { return (n - k * LEAF < LEAF) ? n - k * LEAF : LEAF; }

__global__ void __launch_bounds__(256) bpotrf_kernel(const BSys *sys, StepTable t, int k)
{
    extern __shared__ double bsmem[];
    int64_t local;
    const BSys &S = sys[find_task(t, blockIdx.x, local)];
    if (*S.info != 0) return;
    const int64_t o = (int64_t)k * LEAF;
    potrf_leaf_body<LEAF>(S.A + o + o * S.lda, S.lda, (int)block_rows(S.n, k), nullptr,
                          S.Linv + (int64_t)k * LEAF * LEAF, o, S.info, bsmem);
}

__global__ void __launch_bounds__(256) btrsm_kernel(const BSys *sys, StepTable t, int k)
{
    extern __shared__ __align__(16) unsigned char btsmem[];
    int64_t local;
    const BSys &S = sys[find_task(t, blockIdx.x, local)];
    if (*S.info != 0) return;
    const int64_t o = (int64_t)k * LEAF, m = S.n - o - LEAF;
    trsm_inv_body<double, 64>(S.A + (o + LEAF) + o * S.lda, S.lda, m, LEAF, S.Linv + (int64_t)k * LEAF * LEAF,
                              local * 64, btsmem);
}

// Step 3: one BT x BT lower tile of the trailing matrix (BT = 32 or 64,
// chosen per system size by the autotuner; every entry sums its products
// in the same order for either tile, so the result does not depend on it).
template <int BT>
__global__ void __launch_bounds__(256, 3) bgemm_kernel(const BSys *sys, StepTable t, int k)
{
    int64_t local;
    const BSys &S = sys[find_task(t, blockIdx.x, local)];
    if (*S.info != 0) return;
    const int64_t o = (int64_t)k * LEAF, m = S.n - o - LEAF;
    int64_t ti, tj;
    tri_index(local, ti, tj);
    const double *P = S.A + (o + LEAF) + o * S.lda;
    gemm_nt_minus_body<double, true, BT>(m, m, LEAF, P, S.lda, P, S.lda, S.A + (o + LEAF) * (1 + S.lda), S.lda,
                                         ti, tj);
}

// Forward step k: y_k = inv(L_kk) b_k (each CTA recomputes it), CTA 0 of the
// system stores it in Y, every CTA updates 256 rows below the block.
__global__ void __launch_bounds__(256) bfwd_kernel(const BSys *sys, StepTable t, int k)
{
    __shared__ double bj[LEAF], yj[LEAF];
    int64_t local;
    const BSys &S = sys[find_task(t, blockIdx.x, local)];
    if (*S.info != 0) return;
    const int tid = threadIdx.x;
    const int64_t o = (int64_t)k * LEAF;
    const int nb = (int)block_rows(S.n, k);
    const double *Li = S.Linv + (int64_t)k * LEAF * LEAF;
    const int64_t row = o + nb + local * 256 + tid;
    for (int r = 0; r < S.nrhs; ++r) {
        if (tid < LEAF) bj[tid] = (tid < nb) ? S.B[o + tid + r * S.ldb] : 0.0;
        __syncthreads();
        if (tid < LEAF) {
            double s = 0.0;
            for (int q = 0; q <= tid; ++q) s = fma(Li[tid + q * LEAF], bj[q], s);
            yj[tid] = s;
            if (local == 0 && tid < nb) S.Y[o + tid + r * S.n] = s;
        }
        __syncthreads();
        if (row < S.n) {
            double s = S.B[row + r * S.ldb];
            for (int q = 0; q < nb; ++q) s = fma(-S.A[row + (o + q) * S.lda], yj[q], s);
            S.B[row + r * S.ldb] = s;
        }
        __syncthreads();
    }
}

// Back step k: x_k = inv(L_kk)^T w_k (w = Y), CTA 0 of the system stores it
// in B, every CTA updates 64 earlier entries of w, one warp per entry.
__global__ void __launch_bounds__(256) bbwd_kernel(const BSys *sys, StepTable t, int k)
{
    __shared__ double wj[LEAF], xj[LEAF];
    int64_t local;
    const BSys &S = sys[find_task(t, blockIdx.x, local)];
    if (*S.info != 0) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t o = (int64_t)k * LEAF;
    const int nb = (int)block_rows(S.n, k);
    const double *Li = S.Linv + (int64_t)k * LEAF * LEAF;
    for (int r = 0; r < S.nrhs; ++r) {
        if (tid < LEAF) wj[tid] = (tid < nb) ? S.Y[o + tid + r * S.n] : 0.0;
        __syncthreads();
        if (tid < LEAF) {
            double s = 0.0;
            for (int q = tid; q < LEAF; ++q) s = fma(Li[q + tid * LEAF], wj[q], s);
            xj[tid] = s;
            if (local == 0 && tid < nb) S.B[o + tid + r * S.ldb] = s;
        }
        __syncthreads();
        for (int cc = warp; cc < LEAF; cc += 8) {
            const int64_t c = local * LEAF + cc;
            if (c >= o) break;
            double s = 0.0;
            if (lane < nb) s = S.A[(o + lane) + c * S.lda] * xj[lane];
            if (lane + 32 < nb) s = fma(S.A[(o + lane + 32) + c * S.lda], xj[lane + 32], s);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            if (lane == 0) S.Y[c + r * S.n] -= s;
        }
        __syncthreads();
    }
}

constexpr size_t BPOTRF_SMEM = 2 * LEAF * (LEAF + 1) * sizeof(double);
constexpr size_t BTRSM_SMEM = trsm_smem_bytes<double, 64>();

// One captured batch: device tables, per-system workspace, the graph.
struct BatchPlan {
    void *dev = nullptr;          // all device memory of the plan
    size_t bytes = 0;
    BSys *d_sys = nullptr;
    int64_t *d_info = nullptr;
    int count = 0;
    int64_t launches = 0;
    cudaGraphExec_t exec = nullptr;
    std::vector<int64_t> flops;   // per system n^3/3
};

struct PlanKey {
    std::vector<int64_t> v;
    bool operator<(const PlanKey &o) const { return v < o.v; }
};

struct PlanCache {
    std::map<PlanKey, BatchPlan> plans;
};

std::map<gpch_ctx *, PlanCache> g_caches;   // per context
std::mutex g_caches_mu;

void free_plan(BatchPlan &p)
{
    if (p.exec) cudaGraphExecDestroy(p.exec);
    if (p.dev) cudaFree(p.dev);
    p = BatchPlan();
}

// Host-side layout of all step tables, built from the sizes only.
struct HostTables {
    std::vector<int> sys;
    std::vector<int64_t> pref;
    struct Step {
        size_t sys_off, pref_off;
        int cnt;
        int64_t tasks;
    };
    std::vector<Step> potrf, trsm, gemm64, gemm32, fwd, bwd;
};

template <typename F>
HostTables::Step add_step(HostTables &h, int count, const int64_t *ns, F tasks_of)
{
    HostTables::Step st{h.sys.size(), h.pref.size(), 0, 0};
    h.pref.push_back(0);
    for (int s = 0; s < count; ++s) {
        const int64_t t = tasks_of(ns[s]);
        if (t <= 0) continue;
        h.sys.push_back(s);
        st.tasks += t;
        h.pref.push_back(st.tasks);
        ++st.cnt;
    }
    return st;
}

// Sizes-only plan of a batch: the step tables and the device layout.
struct Layout {
    HostTables h;
    std::vector<int64_t> ns;
    int64_t kmax = 0;
    gpch::TuneTable tune{};
    // trailing-update tile of a system of size n (autotuned, else 64)
    int bt_of(int64_t n) const { return tune.batch_bt[0][gpch::tune_bucket(n)] == 32 ? 32 : 64; }
    size_t o_sys = 0, o_info = 0, o_tsys = 0, o_pref = 0, bytes = 0;
    std::vector<size_t> o_linv, o_y;
};

Layout make_layout(int count, const gpch_system *systems, const gpch::TuneTable &tune)
{
    Layout L;
    L.tune = tune;
    L.ns.resize(count);
    for (int s = 0; s < count; ++s) {
        L.ns[s] = systems[s].n;
        const int64_t nb = (L.ns[s] + LEAF - 1) / LEAF;
        if (nb > L.kmax) L.kmax = nb;
    }
    HostTables &h = L.h;
    const int64_t *ns = L.ns.data();
    for (int64_t k = 0; k < L.kmax; ++k) {
        h.potrf.push_back(add_step(h, count, ns, [&](int64_t n) { return n > k * LEAF ? 1 : 0; }));
        h.trsm.push_back(add_step(h, count, ns, [&](int64_t n) {
            const int64_t m = n - (k + 1) * LEAF;
            return m > 0 ? (m + 63) / 64 : 0;
        }));
        for (int bt : {64, 32}) {
            auto &dst = bt == 64 ? h.gemm64 : h.gemm32;
            dst.push_back(add_step(h, count, ns, [&](int64_t n) {
                if (L.bt_of(n) != bt) return (int64_t)0;
                const int64_t m = n - (k + 1) * LEAF;
                const int64_t T = m > 0 ? (m + bt - 1) / bt : 0;
                return T * (T + 1) / 2;
            }));
        }
        h.fwd.push_back(add_step(h, count, ns, [&](int64_t n) {
            if (n <= k * LEAF) return (int64_t)0;
            const int64_t below = n - (k + 1) * LEAF;
            return below > 0 ? (below + 255) / 256 : (int64_t)1;
        }));
        h.bwd.push_back(add_step(h, count, ns, [&](int64_t n) {
            if (n <= k * LEAF) return (int64_t)0;
            return k > 0 ? k : (int64_t)1;   // k*64 columns above, 64 per CTA
        }));
    }
    gpch::Carver dry(nullptr);
    L.o_sys = dry.reserve(count * sizeof(BSys));
    L.o_info = dry.reserve(count * sizeof(int64_t));
    L.o_tsys = dry.reserve(h.sys.size() * sizeof(int));
    L.o_pref = dry.reserve(h.pref.size() * sizeof(int64_t));
    L.o_linv.resize(count);
    L.o_y.resize(count);
    for (int s = 0; s < count; ++s) {
        L.o_linv[s] = dry.reserve((size_t)((ns[s] + LEAF - 1) / LEAF) * LEAF * LEAF * sizeof(double));
        L.o_y[s] = dry.reserve((size_t)ns[s] * systems[s].nrhs * sizeof(double));
    }
    L.bytes = dry.off;
    return L;
}

struct DevTables {
    BSys *sys;
    int64_t *info;
    int *tsys;
    int64_t *pref;
};

// Copy descriptors and tables to `base` (L.bytes of device memory) on st.
gpch_status upload(gpch_ctx *ctx, const Layout &L, int count, const gpch_system *systems, char *base, DevTables &d,
                   cudaStream_t st)
{
    d.sys = reinterpret_cast<BSys *>(base + L.o_sys);
    d.info = reinterpret_cast<int64_t *>(base + L.o_info);
    d.tsys = reinterpret_cast<int *>(base + L.o_tsys);
    d.pref = reinterpret_cast<int64_t *>(base + L.o_pref);
    std::vector<BSys> hs(count);
    for (int s = 0; s < count; ++s)
        hs[s] = BSys{systems[s].A, systems[s].lda, L.ns[s], systems[s].B, systems[s].ldb, systems[s].nrhs,
                     reinterpret_cast<double *>(base + L.o_linv[s]), reinterpret_cast<double *>(base + L.o_y[s]),
                     d.info + s};
    GPCH_CUDA(ctx, cudaMemcpyAsync(d.sys, hs.data(), count * sizeof(BSys), cudaMemcpyHostToDevice, st));
    if (!L.h.sys.empty())
        GPCH_CUDA(ctx, cudaMemcpyAsync(d.tsys, L.h.sys.data(), L.h.sys.size() * sizeof(int), cudaMemcpyHostToDevice,
                                       st));
    GPCH_CUDA(ctx, cudaMemcpyAsync(d.pref, L.h.pref.data(), L.h.pref.size() * sizeof(int64_t),
                                   cudaMemcpyHostToDevice, st));
    GPCH_CUDA(ctx, cudaStreamSynchronize(st));   // the host vectors go out of scope
    return GPCH_OK;
}

gpch_status set_attrs(gpch_ctx *ctx)
{
    static gpch::DeviceOnce attr_once;
    GPCH_CHECK(gpch::once_per_device(ctx, attr_once, [&]() -> gpch_status {
        GPCH_CUDA(ctx, cudaFuncSetAttribute(bpotrf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)BPOTRF_SMEM));
        GPCH_CUDA(ctx, cudaFuncSetAttribute(btrsm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)BTRSM_SMEM));
        return GPCH_OK;
    }));
    return GPCH_OK;
}

// Enqueue the whole batch on st (directly or into a capturing stream);
// returns the number of kernel launches.
int64_t enqueue_batch(const Layout &L, const DevTables &d, int count, cudaStream_t st)
{
    const HostTables &h = L.h;
    auto table = [&](const HostTables::Step &x) { return StepTable{d.tsys + x.sys_off, d.pref + x.pref_off, x.cnt}; };
    int64_t launches = 0;
    cudaMemsetAsync(d.info, 0, count * sizeof(int64_t), st);
    for (int64_t k = 0; k < L.kmax; ++k) {
        if (h.potrf[k].tasks) {
            bpotrf_kernel<<<(unsigned)h.potrf[k].tasks, 256, BPOTRF_SMEM, st>>>(d.sys, table(h.potrf[k]), (int)k);
            ++launches;
        }
        if (h.trsm[k].tasks) {
            btrsm_kernel<<<(unsigned)h.trsm[k].tasks, 256, BTRSM_SMEM, st>>>(d.sys, table(h.trsm[k]), (int)k);
            ++launches;
        }
        if (h.gemm64[k].tasks) {
            bgemm_kernel<64><<<(unsigned)h.gemm64[k].tasks, 256, 0, st>>>(d.sys, table(h.gemm64[k]), (int)k);
            ++launches;
        }
        if (h.gemm32[k].tasks) {
            bgemm_kernel<32><<<(unsigned)h.gemm32[k].tasks, 256, 0, st>>>(d.sys, table(h.gemm32[k]), (int)k);
            ++launches;
        }
    }
    for (int64_t k = 0; k < L.kmax; ++k)
        if (h.fwd[k].tasks) {
            bfwd_kernel<<<(unsigned)h.fwd[k].tasks, 256, 0, st>>>(d.sys, table(h.fwd[k]), (int)k);
            ++launches;
        }
    for (int64_t k = L.kmax - 1; k >= 0; --k)
        if (h.bwd[k].tasks) {
            bbwd_kernel<<<(unsigned)h.bwd[k].tasks, 256, 0, st>>>(d.sys, table(h.bwd[k]), (int)k);
            ++launches;
        }
    return launches;
}

gpch_status build_plan(gpch_ctx *ctx, int count, const gpch_system *systems, BatchPlan &plan, cudaStream_t st)
{
    Layout L = make_layout(count, systems, gpch::tune_table(ctx->device));
    if (ctx->budget && ctx->ws_bytes + L.bytes > ctx->budget)
        return gpch::fail(ctx, GPCH_OOM_BUDGET, "batch plan of %zu bytes exceeds the HBM budget", L.bytes);
    GPCH_CUDA(ctx, cudaMalloc(&plan.dev, L.bytes));
    plan.bytes = L.bytes;
    DevTables d;
    gpch_status s0 = upload(ctx, L, count, systems, static_cast<char *>(plan.dev), d, st);
    if (s0 != GPCH_OK) {
        free_plan(plan);
        return s0;
    }
    plan.d_sys = d.sys;
    plan.d_info = d.info;
    GPCH_CHECK(set_attrs(ctx));
    cudaStream_t cs;
    GPCH_CUDA(ctx, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    int64_t launches = 0;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        launches = enqueue_batch(L, d, count, cs);
        e = cudaStreamEndCapture(cs, &graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&plan.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_plan(plan);
        return gpch::fail(ctx, GPCH_CUDA_ERROR, "batch graph capture failed: %s", cudaGetErrorString(e));
    }
    plan.count = count;
    plan.launches = launches;
    plan.flops.resize(count);
    for (int s = 0; s < count; ++s) plan.flops[s] = L.ns[s] * L.ns[s] * L.ns[s] / 3;
    return GPCH_OK;
}

}  // namespace

namespace gpch {

// A batch launched directly on `st` with its tables in the context's
// workspace (no graph, nothing cached): the form a serving loop uses for
// batches that are each seen once.  info: host array of count entries.
gpch_status batched_solve_direct(gpch_ctx *ctx, int count, const gpch_system *systems, cudaStream_t st,
                                 int64_t *info)
{
    Layout L = make_layout(count, systems, gpch::tune_table(ctx->device));
    GPCH_CHECK(ws_reserve(ctx, L.bytes));
    DevTables d;
    GPCH_CHECK(upload(ctx, L, count, systems, static_cast<char *>(ctx->ws), d, st));
    GPCH_CHECK(set_attrs(ctx));
    double work = 0.0;
    for (int s = 0; s < count; ++s) work += (double)L.ns[s] * L.ns[s] * L.ns[s] / 3.0;
    {
        PhaseScope ph(ctx, GPCH_PHASE_BATCHED, st, work);
        ctx->launches += enqueue_batch(L, d, count, st);
    }
    GPCH_LAUNCH_CHECK(ctx);
    --ctx->launches;
    std::vector<int64_t> h(count);
    GPCH_CUDA(ctx, cudaMemcpyAsync(h.data(), d.info, count * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    GPCH_CUDA(ctx, cudaStreamSynchronize(st));
    for (int s = 0; s < count; ++s) info[s] = h[s];
    return GPCH_OK;
}

void batched_release(gpch_ctx *ctx)
{
    std::lock_guard<std::mutex> lock(g_caches_mu);
    auto it = g_caches.find(ctx);
    if (it == g_caches.end()) return;
    for (auto &kv : it->second.plans) free_plan(kv.second);
    g_caches.erase(it);
}

}  // namespace gpch

extern "C" gpch_status gpch_batched_solve(gpch_ctx *ctx, int count, const gpch_system *systems, void *stream,
                                          int64_t *info)
{
    GPCH_ARG(ctx, ctx != nullptr, "null context");
    GPCH_ARG(ctx, count >= 0, "count < 0");
    if (count == 0) return GPCH_OK;
    GPCH_ARG(ctx, systems != nullptr && info != nullptr, "null pointer");
    for (int s = 0; s < count; ++s) {
        const gpch_system &y = systems[s];
        GPCH_ARG(ctx, y.n >= 1 && y.nrhs >= 1 && y.lda >= y.n && y.ldb >= y.n && y.A && y.B,
                 "each system needs n >= 1, nrhs >= 1, lda >= n, ldb >= n and non-null A, B");
        GPCH_ARG(ctx, y.n < ((int64_t)1 << 31), "n too large");
    }
    GPCH_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    PlanKey key;
    key.v.reserve(count * 6 + gpch::TUNE_BUCKETS);
    {
        const gpch::TuneTable tt = gpch::tune_table(ctx->device);   // plans differ by their update tiles
        for (int b = 0; b < gpch::TUNE_BUCKETS; ++b) key.v.push_back(tt.batch_bt[0][b]);
    }
    for (int s = 0; s < count; ++s) {
        const gpch_system &y = systems[s];
        key.v.insert(key.v.end(), {y.n, (int64_t)(uintptr_t)y.A, y.lda, (int64_t)(uintptr_t)y.B, y.ldb, y.nrhs});
    }
    std::lock_guard<std::mutex> lock(g_caches_mu);
    PlanCache &cache = g_caches[ctx];
    auto it = cache.plans.find(key);
    if (it == cache.plans.end()) {
        if (cache.plans.size() >= 8) {   // bounded cache: drop the oldest-keyed plan
            GPCH_CUDA(ctx, cudaStreamSynchronize(st));
            free_plan(cache.plans.begin()->second);
            cache.plans.erase(cache.plans.begin());
        }
        BatchPlan plan;
        GPCH_CHECK(build_plan(ctx, count, systems, plan, st));
        it = cache.plans.emplace(key, plan).first;
    }
    BatchPlan &plan = it->second;
    double work = 0.0;
    for (int64_t f : plan.flops) work += (double)f;
    {
        gpch::PhaseScope ph(ctx, GPCH_PHASE_BATCHED, st, work);
        GPCH_CUDA(ctx, cudaGraphLaunch(plan.exec, st));
    }
    ctx->launches += plan.launches;
    int64_t *h = static_cast<int64_t *>(ctx->pinned);
    const int chunk = (int)(ctx->pinned_bytes / sizeof(int64_t));
    bool any_bad = false;
    for (int s0 = 0; s0 < count; s0 += chunk) {
        const int c = (count - s0 < chunk) ? count - s0 : chunk;
        GPCH_CUDA(ctx, cudaMemcpyAsync(h, plan.d_info + s0, c * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        GPCH_CUDA(ctx, cudaStreamSynchronize(st));
        for (int s = 0; s < c; ++s) {
            info[s0 + s] = h[s];
            if (h[s] != 0) any_bad = true;
        }
    }
    if (any_bad) return gpch::fail(ctx, GPCH_NOT_SPD, "at least one system of the batch is not SPD (see info)");
    return GPCH_OK;
}
