// batched_mixed.cu -- A10, mixed precision: many independent GP systems
// factored in FP32 with FP64 diagonal leaves, then refined to an FP64
// backward error, all systems together.
//
// Per system (n <= 65536, at most 16 right-hand sides):
//   set-up   L = fl32(A) (lower triangle), ||A||_inf, ||b_r||_inf, x = 0
//   factor   Algorithm 1 (right) on L with 64-wide blocks: step 1 in FP64
//            (the 64 x 64 diagonal block widened, factored by the FP64
//            leaf, its inverse kept in FP64, the factor rounded back to
//            FP32), step 2 as the product with that inverse and step 3 as
//            an FP32 SYRK/GEMM on the CUDA cores
//   refine   iterative refinement in FP64: r = b - A x (FP64 products,
//            A intact), stop per column when
//            ||r||_inf / (||A||_inf ||x||_inf + ||b||_inf) <= tol,
//            else x += L^-T L^-1 r (forward/back substitution with the
//            FP32 factor, FP64 vectors)
// Refinement converges when kappa(A) times FP32's unit roundoff is well
// below one, the regime of the batched GP systems; a column whose error
// stops falling is reported as not converged.
//
// Like the FP64 batch, every step of every system is one grouped launch
// per kernel kind (task tables map a CTA to (system, local task)), each
// system is cut by its own size only, so its arithmetic does not depend on
// its batch-mates, and the launch sequence (set-up, factor, first solve,
// REFINE_STEPS refinement steps) is captured once as a CUDA graph; a batch
// that needs more steps replays a captured single step.  Converged systems
// skip their work inside every kernel.
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "dense_fp64.cuh"

namespace {

using gpch::LEAF;

constexpr int MAXR = 16;
constexpr int REFINE_STEPS = 4;

// Per-system device state (doubles first).
struct MState {
    double anorm;
    double binf[MAXR], xinf[MAXR], rinf[MAXR], bwd[MAXR], prev[MAXR];
    int active;          // 1 while some column is refining
    int colact[MAXR];    // per column
    int iters;           // refinement steps taken
    int stalled;         // a column's error stopped falling
};

struct MSys {
    const double *A;
    int64_t lda;
    int64_t n;
    const double *B;
    int64_t ldb;
    double *X;
    int64_t ldx;
    int nrhs;
    float *L;            // n x n (ld n), FP32 factor
    double *Linv;        // nblocks x 64 x 64
    double *stage;       // 64 x 64 FP64 staging of a diagonal block
    double *W;           // n x nrhs: residual, then the correction (in place)
    double *Y;           // n x nrhs: forward-substitution result
    int64_t *info;
    MState *ms;
};

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

__device__ inline void atomic_max_nonneg(double *addr, double v)
{
    atomicMax(reinterpret_cast<unsigned long long *>(addr), (unsigned long long)__double_as_longlong(v));
}

__device__ inline double warp_max(double v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}

// Set-up, one CTA per 64 columns: L[:, cols] = fl32(A) on and below the
// diagonal, column sums |A| (= row sums, A symmetric) into ||A||_inf, and
// for CTA 0 of a system ||b_r||_inf and x = 0.
__global__ void __launch_bounds__(256) bm_setup_kernel(const MSys *sys, StepTable t)
{
    int64_t local;
    const MSys &S = sys[find_task(t, blockIdx.x, local)];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t c0 = local * LEAF;
    for (int cc = warp; cc < LEAF; cc += 8) {
        const int64_t c = c0 + cc;
        if (c >= S.n) break;
        double s = 0.0;
        for (int64_t i = lane; i < S.n; i += 32) {
            const double a = S.A[i + c * S.lda];
            s += fabs(a);
            if (i >= c) S.L[i + c * S.n] = (float)a;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) atomic_max_nonneg(&S.ms->anorm, s);
    }
    if (local == 0) {
        for (int r = 0; r < S.nrhs; ++r) {
            double m = 0.0;
            for (int64_t i = tid; i < S.n; i += 256) {
                m = fmax(m, fabs(S.B[i + r * S.ldb]));
                S.X[i + r * S.ldx] = 0.0;
                S.W[i + r * S.n] = S.B[i + r * S.ldb];
            }
            m = warp_max(m);
            if (lane == 0) atomic_max_nonneg(&S.ms->binf[r], m);
        }
    }
}

// Step 1 of block column k: the 64 x 64 diagonal block in FP64.
__global__ void __launch_bounds__(256) bm_potrf_kernel(const MSys *sys, StepTable t, int k)
{
    extern __shared__ double bm_smem[];
    int64_t local;
    const MSys &S = sys[find_task(t, blockIdx.x, local)];
    if (*S.info != 0) return;
    const int64_t o = (int64_t)k * LEAF;
    const int nb = (int)block_rows(S.n, k);
    const float *Lk = S.L + o + o * S.n;
    for (int e = threadIdx.x; e < LEAF * LEAF; e += blockDim.x) {
        const int r = e % LEAF, c = e / LEAF;
        S.stage[e] = (r < nb && c < nb && r >= c) ? (double)Lk[r + c * S.n] : 0.0;
    }
    __syncthreads();
    potrf_leaf_body<LEAF>(S.stage, LEAF, nb, nullptr, S.Linv + (int64_t)k * LEAF * LEAF, o, S.info, bm_smem);
    __syncthreads();
    if (*S.info != 0) return;
    float *Lw = S.L + o + o * S.n;
    for (int e = threadIdx.x; e < LEAF * LEAF; e += blockDim.x) {
        const int r = e % LEAF, c = e / LEAF;
        if (r < nb && c < nb && r >= c) Lw[r + c * S.n] = (float)S.stage[e];
    }
}

// Step 2: rows below the block times inv(L_kk)^T, 64 rows per CTA.
__global__ void __launch_bounds__(256) bm_trsm_kernel(const MSys *sys, StepTable t, int k)
{
    extern __shared__ __align__(16) unsigned char bm_tsmem[];
    int64_t local;
    const MSys &S = sys[find_task(t, blockIdx.x, local)];
    if (*S.info != 0) return;
    const int64_t o = (int64_t)k * LEAF, m = S.n - o - LEAF;
    trsm_inv_body<float, 64>(S.L + (o + LEAF) + o * S.n, S.n, m, LEAF, S.Linv + (int64_t)k * LEAF * LEAF,
                             local * 64, bm_tsmem);
}

// Step 3: one BT x BT lower tile of the trailing matrix, FP32 (BT = 32 or
// 64, chosen per system size by the autotuner; the result does not depend
// on it).
template <int BT>
__global__ void __launch_bounds__(256, 3) bm_gemm_kernel(const MSys *sys, StepTable t, int k)
{
    int64_t local;
    const MSys &S = sys[find_task(t, blockIdx.x, local)];
    if (*S.info != 0) return;
    const int64_t o = (int64_t)k * LEAF, m = S.n - o - LEAF;
    int64_t ti, tj;
    tri_index(local, ti, tj);
    const float *P = S.L + (o + LEAF) + o * S.n;
    gemm_nt_minus_body<float, true, BT>(m, m, LEAF, P, S.n, P, S.n, S.L + (o + LEAF) * (1 + S.n), S.n, ti, tj);
}

// Forward step k on W (in place): y_k = inv(L_kk) w_k (every CTA of the
// system recomputes it), CTA 0 stores it in Y, every CTA updates 256 rows
// below the block.  FP32 factor entries, FP64 vectors.
__global__ void __launch_bounds__(256) bm_fwd_kernel(const MSys *sys, StepTable t, int k)
{
    __shared__ double bj[LEAF], yj[LEAF];
    int64_t local;
    const MSys &S = sys[find_task(t, blockIdx.x, local)];
    if (*S.info != 0 || !S.ms->active) return;
    const int tid = threadIdx.x;
    const int64_t o = (int64_t)k * LEAF;
    const int nb = (int)block_rows(S.n, k);
    const double *Li = S.Linv + (int64_t)k * LEAF * LEAF;
    const int64_t row = o + nb + local * 256 + tid;
    for (int r = 0; r < S.nrhs; ++r) {
        if (!S.ms->colact[r]) continue;
        if (tid < LEAF) bj[tid] = (tid < nb) ? S.W[o + tid + r * S.n] : 0.0;
        __syncthreads();
        if (tid < LEAF) {
            double s = 0.0;
            for (int q = 0; q <= tid; ++q) s = fma(Li[tid + q * LEAF], bj[q], s);
            yj[tid] = s;
            if (local == 0 && tid < nb) S.Y[o + tid + r * S.n] = s;
        }
        __syncthreads();
        if (row < S.n) {
            double s = S.W[row + r * S.n];
            for (int q = 0; q < nb; ++q) s = fma(-(double)S.L[row + (o + q) * S.n], yj[q], s);
            S.W[row + r * S.n] = s;
        }
        __syncthreads();
    }
}

// Back step k: x_k = inv(L_kk)^T y_k, CTA 0 of the system stores it in W,
// every CTA updates 64 earlier entries of Y, one warp per entry.
__global__ void __launch_bounds__(256) bm_bwd_kernel(const MSys *sys, StepTable t, int k)
{
    __shared__ double wj[LEAF], xj[LEAF];
    int64_t local;
    const MSys &S = sys[find_task(t, blockIdx.x, local)];
    if (*S.info != 0 || !S.ms->active) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t o = (int64_t)k * LEAF;
    const int nb = (int)block_rows(S.n, k);
    const double *Li = S.Linv + (int64_t)k * LEAF * LEAF;
    for (int r = 0; r < S.nrhs; ++r) {
        if (!S.ms->colact[r]) continue;
        if (tid < LEAF) wj[tid] = (tid < nb) ? S.Y[o + tid + r * S.n] : 0.0;
        __syncthreads();
        if (tid < LEAF) {
            double s = 0.0;
            for (int q = tid; q < LEAF; ++q) s = fma(Li[q + tid * LEAF], wj[q], s);
            xj[tid] = s;
            if (local == 0 && tid < nb) S.W[o + tid + r * S.n] = s;
        }
        __syncthreads();
        for (int cc = warp; cc < LEAF; cc += 8) {
            const int64_t c = local * LEAF + cc;
            if (c >= o) break;
            double s = 0.0;
            if (lane < nb) s = (double)S.L[(o + lane) + c * S.n] * xj[lane];
            if (lane + 32 < nb) s = fma((double)S.L[(o + lane + 32) + c * S.n], xj[lane + 32], s);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            if (lane == 0) S.Y[c + r * S.n] -= s;
        }
        __syncthreads();
    }
}

// x += w on the refining columns (w = the correction), one CTA per 256 rows.
__global__ void __launch_bounds__(256) bm_axpy_kernel(const MSys *sys, StepTable t)
{
    int64_t local;
    const MSys &S = sys[find_task(t, blockIdx.x, local)];
    if (*S.info != 0 || !S.ms->active) return;
    const int64_t i = local * 256 + threadIdx.x;
    if (i >= S.n) return;
    for (int r = 0; r < S.nrhs; ++r)
        if (S.ms->colact[r]) S.X[i + r * S.ldx] += S.W[i + r * S.n];
}

// r = b - A x on the refining columns (FP64, A symmetric: r_j is a dot
// product down column j), one CTA per 8 columns, a warp per column; the
// maxima of |r| and |x| per column go to the system's state.  W <- r.
__global__ void __launch_bounds__(256) bm_resid_kernel(const MSys *sys, StepTable t)
{
    int64_t local;
    const MSys &S = sys[find_task(t, blockIdx.x, local)];
    if (*S.info != 0 || !S.ms->active) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t j = local * 8 + warp;
    if (j >= S.n) return;
    for (int r = 0; r < S.nrhs; ++r) {
        if (!S.ms->colact[r]) continue;
        double s = 0.0;
        for (int64_t i = lane; i < S.n; i += 32) s = fma(S.A[i + j * S.lda], S.X[i + r * S.ldx], s);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) {
            const double rj = S.B[j + r * S.ldb] - s;
            S.W[j + r * S.n] = rj;
            atomic_max_nonneg(&S.ms->rinf[r], fabs(rj));
            atomic_max_nonneg(&S.ms->xinf[r], fabs(S.X[j + r * S.ldx]));
        }
    }
}

// Per system: the backward error of every refining column, its stop, the
// stall test (the error has not halved over the last step, after the
// first two steps), and the reset of the maxima.  One thread per system.
__global__ void bm_check_kernel(const MSys *sys, int count, double tol, int maxit)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= count) return;
    const MSys &S = sys[s];
    MState *m = S.ms;
    if (*S.info != 0 || !m->active) return;
    int any = 0;
    for (int r = 0; r < S.nrhs; ++r) {
        if (m->colact[r]) {
            const double den = m->anorm * m->xinf[r] + m->binf[r];
            const double bwd = den > 0.0 ? m->rinf[r] / den : 0.0;
            m->bwd[r] = bwd;
            if (bwd <= tol) {
                m->colact[r] = 0;
            } else if (m->iters >= 2 && bwd > 0.5 * m->prev[r]) {
                m->colact[r] = 0;
                m->stalled = 1;
            }
            m->prev[r] = bwd;
        }
        m->rinf[r] = 0.0;
        m->xinf[r] = 0.0;
        any |= m->colact[r];
    }
    m->iters += 1;
    if (m->iters > maxit) {
        for (int r = 0; r < S.nrhs; ++r)
            if (m->colact[r]) m->stalled = 1;
        any = 0;
    }
    m->active = any;
}

__global__ void bm_state_init_kernel(const MSys *sys, int count)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= count) return;
    MState *m = sys[s].ms;
    m->anorm = 0.0;
    for (int r = 0; r < MAXR; ++r) {
        m->binf[r] = m->xinf[r] = m->rinf[r] = m->bwd[r] = 0.0;
        m->prev[r] = 1e300;
        m->colact[r] = r < sys[s].nrhs ? 1 : 0;
    }
    m->active = 1;
    m->iters = 0;
    m->stalled = 0;
    *sys[s].info = 0;
}

constexpr size_t BM_POTRF_SMEM = 2 * LEAF * (LEAF + 1) * sizeof(double);
constexpr size_t BM_TRSM_SMEM = trsm_smem_bytes<float, 64>();

struct HostTables {
    std::vector<int> sys;
    std::vector<int64_t> pref;
    struct Step {
        size_t sys_off, pref_off;
        int cnt;
        int64_t tasks;
    };
    std::vector<Step> potrf, trsm, gemm64, gemm32, fwd, bwd;
    Step setup{}, rows{}, cols{};
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

struct Layout {
    HostTables h;
    std::vector<int64_t> ns;
    int64_t kmax = 0;
    gpch::TuneTable tune{};
    // trailing-update tile of a system of size n (autotuned, else 64)
    int bt_of(int64_t n) const { return tune.batch_bt[1][gpch::tune_bucket(n)] == 32 ? 32 : 64; }
    size_t o_sys = 0, o_info = 0, o_state = 0, o_tsys = 0, o_pref = 0, bytes = 0;
    std::vector<size_t> o_L, o_linv, o_stage, o_w, o_y;
};

Layout make_layout(int count, const gpch_msystem *systems, const gpch::TuneTable &tune)
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
    h.setup = add_step(h, count, ns, [](int64_t n) { return (n + LEAF - 1) / LEAF; });
    h.rows = add_step(h, count, ns, [](int64_t n) { return (n + 255) / 256; });
    h.cols = add_step(h, count, ns, [](int64_t n) { return (n + 7) / 8; });
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
            return k > 0 ? k : (int64_t)1;
        }));
    }
    gpch::Carver dry(nullptr);
    L.o_sys = dry.reserve(count * sizeof(MSys));
    L.o_info = dry.reserve(count * sizeof(int64_t));
    L.o_state = dry.reserve(count * sizeof(MState));
    L.o_tsys = dry.reserve(h.sys.size() * sizeof(int));
    L.o_pref = dry.reserve(h.pref.size() * sizeof(int64_t));
    L.o_L.resize(count);
    L.o_linv.resize(count);
    L.o_stage.resize(count);
    L.o_w.resize(count);
    L.o_y.resize(count);
    for (int s = 0; s < count; ++s) {
        const size_t n = (size_t)ns[s];
        L.o_L[s] = dry.reserve(n * n * sizeof(float));
        L.o_linv[s] = dry.reserve((size_t)((n + LEAF - 1) / LEAF) * LEAF * LEAF * sizeof(double));
        L.o_stage[s] = dry.reserve(LEAF * LEAF * sizeof(double));
        L.o_w[s] = dry.reserve(n * systems[s].nrhs * sizeof(double));
        L.o_y[s] = dry.reserve(n * systems[s].nrhs * sizeof(double));
    }
    L.bytes = dry.off;
    return L;
}

struct DevTables {
    MSys *sys;
    int64_t *info;
    MState *state;
    int *tsys;
    int64_t *pref;
};

gpch_status upload(gpch_ctx *ctx, const Layout &L, int count, const gpch_msystem *systems, char *base, DevTables &d,
                   cudaStream_t st)
{
    d.sys = reinterpret_cast<MSys *>(base + L.o_sys);
    d.info = reinterpret_cast<int64_t *>(base + L.o_info);
    d.state = reinterpret_cast<MState *>(base + L.o_state);
    d.tsys = reinterpret_cast<int *>(base + L.o_tsys);
    d.pref = reinterpret_cast<int64_t *>(base + L.o_pref);
    std::vector<MSys> hs(count);
    for (int s = 0; s < count; ++s) {
        const gpch_msystem &y = systems[s];
        hs[s] = MSys{y.A, y.lda, L.ns[s], y.B, y.ldb, y.X, y.ldx, y.nrhs,
                     reinterpret_cast<float *>(base + L.o_L[s]), reinterpret_cast<double *>(base + L.o_linv[s]),
                     reinterpret_cast<double *>(base + L.o_stage[s]), reinterpret_cast<double *>(base + L.o_w[s]),
                     reinterpret_cast<double *>(base + L.o_y[s]), d.info + s, d.state + s};
    }
    GPCH_CUDA(ctx, cudaMemcpyAsync(d.sys, hs.data(), count * sizeof(MSys), cudaMemcpyHostToDevice, st));
    if (!L.h.sys.empty())
        GPCH_CUDA(ctx, cudaMemcpyAsync(d.tsys, L.h.sys.data(), L.h.sys.size() * sizeof(int), cudaMemcpyHostToDevice,
                                       st));
    GPCH_CUDA(ctx, cudaMemcpyAsync(d.pref, L.h.pref.data(), L.h.pref.size() * sizeof(int64_t),
                                   cudaMemcpyHostToDevice, st));
    GPCH_CUDA(ctx, cudaStreamSynchronize(st));
    return GPCH_OK;
}

gpch_status set_attrs(gpch_ctx *ctx)
{
    static gpch::DeviceOnce attr_once;
    return gpch::once_per_device(ctx, attr_once, [&]() -> gpch_status {
        GPCH_CUDA(ctx, cudaFuncSetAttribute(bm_potrf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)BM_POTRF_SMEM));
        GPCH_CUDA(ctx, cudaFuncSetAttribute(bm_trsm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)BM_TRSM_SMEM));
        return GPCH_OK;
    });
}

// One refinement step: r = b - A x and the stop test; x += L^-T L^-1 r.
int64_t enqueue_refine_step(const Layout &L, const DevTables &d, int count, double tol, int maxit, cudaStream_t st)
{
    const HostTables &h = L.h;
    auto table = [&](const HostTables::Step &x) { return StepTable{d.tsys + x.sys_off, d.pref + x.pref_off, x.cnt}; };
    int64_t launches = 0;
    bm_resid_kernel<<<(unsigned)h.cols.tasks, 256, 0, st>>>(d.sys, table(h.cols));
    bm_check_kernel<<<(unsigned)((count + 127) / 128), 128, 0, st>>>(d.sys, count, tol, maxit);
    launches += 2;
    for (int64_t k = 0; k < L.kmax; ++k)
        if (h.fwd[k].tasks) {
            bm_fwd_kernel<<<(unsigned)h.fwd[k].tasks, 256, 0, st>>>(d.sys, table(h.fwd[k]), (int)k);
            ++launches;
        }
    for (int64_t k = L.kmax - 1; k >= 0; --k)
        if (h.bwd[k].tasks) {
            bm_bwd_kernel<<<(unsigned)h.bwd[k].tasks, 256, 0, st>>>(d.sys, table(h.bwd[k]), (int)k);
            ++launches;
        }
    bm_axpy_kernel<<<(unsigned)h.rows.tasks, 256, 0, st>>>(d.sys, table(h.rows));
    return launches + 1;
}

// Set-up, factor, first solve (x = L^-T L^-1 b) and REFINE_STEPS steps.
int64_t enqueue_batch(const Layout &L, const DevTables &d, int count, double tol, int maxit, cudaStream_t st)
{
    const HostTables &h = L.h;
    auto table = [&](const HostTables::Step &x) { return StepTable{d.tsys + x.sys_off, d.pref + x.pref_off, x.cnt}; };
    int64_t launches = 0;
    bm_state_init_kernel<<<(unsigned)((count + 127) / 128), 128, 0, st>>>(d.sys, count);
    bm_setup_kernel<<<(unsigned)h.setup.tasks, 256, 0, st>>>(d.sys, table(h.setup));
    launches += 2;
    for (int64_t k = 0; k < L.kmax; ++k) {
        if (h.potrf[k].tasks) {
            bm_potrf_kernel<<<(unsigned)h.potrf[k].tasks, 256, BM_POTRF_SMEM, st>>>(d.sys, table(h.potrf[k]), (int)k);
            ++launches;
        }
        if (h.trsm[k].tasks) {
            bm_trsm_kernel<<<(unsigned)h.trsm[k].tasks, 256, BM_TRSM_SMEM, st>>>(d.sys, table(h.trsm[k]), (int)k);
            ++launches;
        }
        if (h.gemm64[k].tasks) {
            bm_gemm_kernel<64><<<(unsigned)h.gemm64[k].tasks, 256, 0, st>>>(d.sys, table(h.gemm64[k]), (int)k);
            ++launches;
        }
        if (h.gemm32[k].tasks) {
            bm_gemm_kernel<32><<<(unsigned)h.gemm32[k].tasks, 256, 0, st>>>(d.sys, table(h.gemm32[k]), (int)k);
            ++launches;
        }
    }
    // first solve: W = b was set up; x = 0, so x += L^-T L^-1 b
    for (int64_t k = 0; k < L.kmax; ++k)
        if (h.fwd[k].tasks) {
            bm_fwd_kernel<<<(unsigned)h.fwd[k].tasks, 256, 0, st>>>(d.sys, table(h.fwd[k]), (int)k);
            ++launches;
        }
    for (int64_t k = L.kmax - 1; k >= 0; --k)
        if (h.bwd[k].tasks) {
            bm_bwd_kernel<<<(unsigned)h.bwd[k].tasks, 256, 0, st>>>(d.sys, table(h.bwd[k]), (int)k);
            ++launches;
        }
    bm_axpy_kernel<<<(unsigned)h.rows.tasks, 256, 0, st>>>(d.sys, table(h.rows));
    ++launches;
    for (int q = 0; q < REFINE_STEPS; ++q) launches += enqueue_refine_step(L, d, count, tol, maxit, st);
    return launches;
}

struct MPlan {
    void *dev = nullptr;
    size_t bytes = 0;
    DevTables d{};
    int count = 0;
    int64_t launches = 0, step_launches = 0;
    cudaGraphExec_t exec = nullptr, step = nullptr;
    double work = 0.0;
};

struct MKey {
    std::vector<int64_t> v;
    bool operator<(const MKey &o) const { return v < o.v; }
};

std::map<gpch_ctx *, std::map<MKey, MPlan>> g_mcaches;
std::mutex g_mcaches_mu;

void free_mplan(MPlan &p)
{
    if (p.exec) cudaGraphExecDestroy(p.exec);
    if (p.step) cudaGraphExecDestroy(p.step);
    if (p.dev) cudaFree(p.dev);
    p = MPlan();
}

template <typename F>
cudaError_t capture(cudaGraphExec_t *exec, F &&enqueue)
{
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        enqueue(cs);
        e = cudaStreamEndCapture(cs, &graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    return e;
}

gpch_status build_mplan(gpch_ctx *ctx, int count, const gpch_msystem *systems, double tol, int maxit, MPlan &plan,
                        cudaStream_t st)
{
    Layout L = make_layout(count, systems, gpch::tune_table(ctx->device));
    if (ctx->budget && ctx->ws_bytes + L.bytes > ctx->budget)
        return gpch::fail(ctx, GPCH_OOM_BUDGET, "batch plan of %zu bytes exceeds the HBM budget", L.bytes);
    GPCH_CUDA(ctx, cudaMalloc(&plan.dev, L.bytes));
    plan.bytes = L.bytes;
    gpch_status s0 = upload(ctx, L, count, systems, static_cast<char *>(plan.dev), plan.d, st);
    if (s0 == GPCH_OK) s0 = set_attrs(ctx);
    if (s0 != GPCH_OK) {
        free_mplan(plan);
        return s0;
    }
    int64_t launches = 0, step_launches = 0;
    cudaError_t e = capture(&plan.exec, [&](cudaStream_t cs) {
        launches = enqueue_batch(L, plan.d, count, tol, maxit, cs);
    });
    if (e == cudaSuccess)
        e = capture(&plan.step, [&](cudaStream_t cs) {
            step_launches = enqueue_refine_step(L, plan.d, count, tol, maxit, cs);
        });
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_mplan(plan);
        return gpch::fail(ctx, GPCH_CUDA_ERROR, "batch graph capture failed: %s", cudaGetErrorString(e));
    }
    plan.count = count;
    plan.launches = launches;
    plan.step_launches = step_launches;
    for (int s = 0; s < count; ++s) plan.work += (double)L.ns[s] * L.ns[s] * L.ns[s] / 3.0;
    return GPCH_OK;
}

}  // namespace

namespace gpch {

void batched_mixed_release(gpch_ctx *ctx)
{
    std::lock_guard<std::mutex> lock(g_mcaches_mu);
    auto it = g_mcaches.find(ctx);
    if (it == g_mcaches.end()) return;
    for (auto &kv : it->second) free_mplan(kv.second);
    g_mcaches.erase(it);
}

}  // namespace gpch

extern "C" gpch_status gpch_batched_solve_mixed(gpch_ctx *ctx, int count, const gpch_msystem *systems,
                                                double bwd_tol, int maxit, void *stream, int64_t *info,
                                                gpch_batch_stats *stats)
{
    GPCH_ARG(ctx, ctx != nullptr, "null context");
    if (stats) *stats = gpch_batch_stats{0, 0, 0.0};
    GPCH_ARG(ctx, count >= 0, "count < 0");
    GPCH_ARG(ctx, bwd_tol > 0.0 && maxit >= REFINE_STEPS, "need bwd_tol > 0 and maxit >= 4");
    if (count == 0) return GPCH_OK;
    GPCH_ARG(ctx, systems != nullptr && info != nullptr, "null pointer");
    for (int s = 0; s < count; ++s) {
        const gpch_msystem &y = systems[s];
        GPCH_ARG(ctx, y.n >= 1 && y.nrhs >= 1 && y.nrhs <= MAXR && y.lda >= y.n && y.ldb >= y.n && y.ldx >= y.n &&
                          y.A && y.B && y.X,
                 "each system needs n >= 1, 1 <= nrhs <= 16, lda, ldb, ldx >= n and non-null A, B, X");
        GPCH_ARG(ctx, y.n <= 65536, "n above 65536");
    }
    GPCH_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    MKey key;
    key.v.reserve(count * 8 + 2 + gpch::TUNE_BUCKETS);
    {
        const gpch::TuneTable tt = gpch::tune_table(ctx->device);   // plans differ by their update tiles
        for (int b = 0; b < gpch::TUNE_BUCKETS; ++b) key.v.push_back(tt.batch_bt[1][b]);
    }
    key.v.push_back((int64_t)maxit);
    int64_t tbits;
    std::memcpy(&tbits, &bwd_tol, sizeof(tbits));
    key.v.push_back(tbits);
    for (int s = 0; s < count; ++s) {
        const gpch_msystem &y = systems[s];
        key.v.insert(key.v.end(), {y.n, (int64_t)(uintptr_t)y.A, y.lda, (int64_t)(uintptr_t)y.B, y.ldb,
                                   (int64_t)(uintptr_t)y.X, y.ldx, y.nrhs});
    }
    std::lock_guard<std::mutex> lock(g_mcaches_mu);
    auto &cache = g_mcaches[ctx];
    auto it = cache.find(key);
    if (it == cache.end()) {
        if (cache.size() >= 8) {
            GPCH_CUDA(ctx, cudaStreamSynchronize(st));
            free_mplan(cache.begin()->second);
            cache.erase(cache.begin());
        }
        MPlan plan;
        GPCH_CHECK(build_mplan(ctx, count, systems, bwd_tol, maxit, plan, st));
        it = cache.emplace(key, plan).first;
    }
    MPlan &plan = it->second;
    std::vector<MState> hs(count);
    std::vector<int64_t> hi(count);
    int steps = REFINE_STEPS;
    {
        gpch::PhaseScope ph(ctx, GPCH_PHASE_BATCHED, st, plan.work);
        GPCH_CUDA(ctx, cudaGraphLaunch(plan.exec, st));
        ctx->launches += plan.launches;
        while (true) {
            GPCH_CUDA(ctx, cudaMemcpyAsync(hs.data(), plan.d.state, count * sizeof(MState), cudaMemcpyDeviceToHost, st));
            GPCH_CUDA(ctx, cudaStreamSynchronize(st));
            bool any = false;
            for (int s = 0; s < count; ++s) any |= hs[s].active != 0;
            if (!any || steps > maxit) break;
            GPCH_CUDA(ctx, cudaGraphLaunch(plan.step, st));
            ctx->launches += plan.step_launches;
            ++steps;
        }
    }
    GPCH_CUDA(ctx, cudaMemcpyAsync(hi.data(), plan.d.info, count * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    GPCH_CUDA(ctx, cudaStreamSynchronize(st));
    bool not_spd = false, not_conv = false;
    int it_max = 0;
    double bwd_max = 0.0;
    for (int s = 0; s < count; ++s) {
        info[s] = hi[s];
        if (hi[s] != 0) {
            not_spd = true;
            continue;
        }
        // iters counts the stop tests; the last one found the error small
        const int refine = hs[s].iters > 0 ? hs[s].iters - 1 : 0;
        if (refine > it_max) it_max = refine;
        bool conv = !hs[s].stalled;
        for (int r = 0; r < systems[s].nrhs; ++r) {
            if (hs[s].bwd[r] > bwd_max) bwd_max = hs[s].bwd[r];
            if (hs[s].colact[r] || hs[s].bwd[r] > bwd_tol) conv = false;
        }
        if (!conv) {
            info[s] = -1;
            not_conv = true;
        }
    }
    if (stats) *stats = gpch_batch_stats{it_max, steps, bwd_max};
    if (not_spd) return gpch::fail(ctx, GPCH_NOT_SPD, "the FP32 factor of at least one system broke down (see info)");
    if (not_conv)
        return gpch::fail(ctx, GPCH_NOT_CONVERGED, "refinement of at least one system missed %.1e (info = -1)",
                          bwd_tol);
    return GPCH_OK;
}
