// server.cu -- A11: a serving loop for GP solves with continuous batching.
//
// Requests (points X, SE hyper-parameters, right-hand sides B, all in host
// memory) are admitted as device memory and GPU lanes free up:
//   - a dispatcher thread scans the queue in arrival order and admits every
//     request that fits the HBM budget (first fit), so small requests do
//     not wait behind a large one that does not fit yet;
//   - admitted requests with n <= batch_max_n are grouped (up to
//     batch_max_count per group) and solved by one batched FP64 launch
//     sequence; larger ones run alone, by the mixed-precision refined solve
//     (or the FP64 factor + solve when solo_prec is FP64);
//   - each lane is a host thread with its own library context (workspace)
//     and CUDA stream, so the work of different lanes overlaps on the GPU.
// A request's result depends only on its own data and the path its size
// selects, never on what else is in flight.  Latency = completion time minus
// submission time; gpch_server_get_stats reports p50/p99 over completed
// requests.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.cuh"

namespace {

using clk = std::chrono::steady_clock;

struct Req {
    uint64_t ticket;
    gpch_request r;
    clk::time_point t_submit, t_start, t_end;
    gpch_status status = GPCH_OK;
    int path = 0;            // 1 batched FP64, 2 solo mixed, 3 solo FP64
    int iterations = 0;
    double backward_error = 0.0;
    size_t mem = 0;
    bool done = false;
};

struct Lane;

}  // namespace

struct gpch_server {
    int device = 0;
    gpch_server_opts o{};
    std::mutex mu;
    std::condition_variable cv_dispatch, cv_done;
    std::deque<Req *> queue;
    std::unordered_map<uint64_t, Req *> reqs;
    std::vector<Lane *> lanes;
    std::thread dispatcher;
    bool stop = false;
    uint64_t next_ticket = 1;
    size_t mem_reserved = 0;      // device bytes of admitted, unfinished requests
    size_t mem_peak = 0;
    std::vector<double> latencies_ms;
    int64_t completed = 0, failed = 0, batches = 0, batched_requests = 0;
    clk::time_point t_first_submit, t_last_done;
    bool any_submit = false;
};

namespace {

struct Lane {
    gpch_server *srv = nullptr;
    gpch_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    std::thread th;
    std::vector<Req *> job;   // empty = idle
    bool busy = false;
    // device buffers, grown on demand
    void *buf = nullptr;
    size_t cap = 0;
};

size_t round_up(size_t x) { return (x + 255) & ~size_t(255); }

// Device bytes a request holds while in flight: its matrix, points and
// right-hand sides, plus (solo mixed path) the FP32 factor and panel copies.
size_t request_bytes(const gpch_request &r, bool solo_mixed, int tile)
{
    const size_t n = (size_t)r.n;
    size_t b = round_up(n * n * 8) + round_up(n * (size_t)r.d * 8) + 2 * round_up(n * (size_t)r.nrhs * 8);
    // mixed solo path: FP32 factor, 16-bit head and tail copies of every
    // panel (n x n each), vectors
    if (solo_mixed)
        b += round_up(((n + 31) / 32 * 32) * n * 4) + 2 * round_up(n * ((n + 63) / 64 * 64) * 2) +
             round_up((size_t)tile * tile * 8) + 12 * n * 8 * r.nrhs +
             // panel solve on tensor cores: L_jj^-T, its 16-bit copies, the panel's
             3 * round_up((size_t)tile * tile * 4) + 2 * round_up(n * (size_t)tile * 2) +
             // pieces of ||A||_inf: a row sum per 64-column strip, a column sum
             // per 1024-row chunk
             round_up(((n + 63) / 64 + (n + 1023) / 1024) * n * 4);
    // with one or two right-hand sides: the products' packed copy of A's
    // lower triangle and their partial sums
    // (strips of 256 columns from their diagonal down, columns of n rounded
    // up to even, 8 bytes per entry)
    if (solo_mixed && r.nrhs <= 2) {
        const size_t n2 = (n + 1) & ~size_t(1), strips = (n + 255) / 256;
        b += round_up(256 * (strips * n2 - 128 * strips * (strips - 1)) * 8) +
             round_up(2 * strips * n * 8 * (size_t)r.nrhs);
    }
    return b;
}

bool is_small(const gpch_server *s, const gpch_request &r) { return r.n <= s->o.batch_max_n; }

gpch_status ensure(Lane *L, size_t bytes)
{
    if (bytes <= L->cap) return GPCH_OK;
    if (L->buf) {
        cudaStreamSynchronize(L->stream);
        cudaFree(L->buf);
        L->buf = nullptr;
        L->cap = 0;
    }
    if (cudaMalloc(&L->buf, bytes) != cudaSuccess) {
        cudaGetLastError();
        return GPCH_OOM_BUDGET;
    }
    L->cap = bytes;
    return GPCH_OK;
}

// The tile of a solo request: the autotuned refined-solve tile of its size
// bucket (the defaults until the device is tuned).
int pick_tile_dev(int device, int64_t n) { return gpch::tune_table(device).refined_tile[gpch::tune_bucket(n)]; }

// Solve one request alone on the lane.
void run_solo(Lane *L, Req *q)
{
    gpch_server *S = L->srv;
    const gpch_request &r = q->r;
    const bool mixed = S->o.solo_prec != GPCH_PREC_FP64;
    const size_t n = (size_t)r.n;
    const size_t oA = 0, oX = oA + round_up(n * n * 8), oB = oX + round_up(n * r.d * 8),
                 oO = oB + round_up(n * r.nrhs * 8), end = oO + round_up(n * r.nrhs * 8);
    gpch_status st = ensure(L, end);
    if (st != GPCH_OK) {
        q->status = st;
        return;
    }
    char *b = static_cast<char *>(L->buf);
    double *dA = reinterpret_cast<double *>(b + oA), *dX = reinterpret_cast<double *>(b + oX);
    double *dB = reinterpret_cast<double *>(b + oB), *dO = reinterpret_cast<double *>(b + oO);
    cudaMemcpyAsync(dX, r.X, n * r.d * 8, cudaMemcpyHostToDevice, L->stream);
    cudaMemcpyAsync(dB, r.B, n * r.nrhs * 8, cudaMemcpyHostToDevice, L->stream);
    st = gpch_se_matrix(L->ctx, r.n, r.d, dX, r.sf2, r.ell, r.sn2, dA, r.n, L->stream);
    if (st == GPCH_OK) {
        if (mixed) {
            q->path = 2;
            gpch_refine_stats rs;
            st = gpch_solve_refined(L->ctx, r.n, dA, r.n, dB, r.n, dO, r.n, r.nrhs, S->o.solo_prec, pick_tile_dev(S->device, r.n),
                                    S->o.bwd_tol, 500, L->stream, &rs);
            q->iterations = rs.iterations;
            q->backward_error = rs.backward_error_max;
        } else {
            q->path = 3;
            int64_t info = 0;
            st = gpch_chol_factor(L->ctx, r.n, pick_tile_dev(S->device, r.n), dA, r.n, L->stream, &info);
            if (st == GPCH_OK) {
                cudaMemcpyAsync(dO, dB, n * r.nrhs * 8, cudaMemcpyDeviceToDevice, L->stream);
                st = gpch_chol_solve(L->ctx, r.n, dA, r.n, dO, r.n, r.nrhs, L->stream);
            }
        }
    }
    if (st == GPCH_OK) {
        cudaMemcpyAsync(r.Xout, dO, n * r.nrhs * 8, cudaMemcpyDeviceToHost, L->stream);
        if (cudaStreamSynchronize(L->stream) != cudaSuccess) {
            cudaGetLastError();
            st = GPCH_CUDA_ERROR;
        }
    }
    q->status = st;
}

// Solve a group of small requests with one batched launch sequence.
void run_batch(Lane *L, std::vector<Req *> &qs)
{
    size_t end = 0;
    std::vector<size_t> oA(qs.size()), oX(qs.size()), oB(qs.size());
    for (size_t i = 0; i < qs.size(); ++i) {
        const gpch_request &r = qs[i]->r;
        const size_t n = (size_t)r.n;
        oA[i] = end;
        end += round_up(n * n * 8);
        oX[i] = end;
        end += round_up(n * r.d * 8);
        oB[i] = end;
        end += round_up(n * r.nrhs * 8);
    }
    gpch_status st = ensure(L, end);
    std::vector<gpch_system> sys(qs.size());
    char *b = static_cast<char *>(L->buf);
    for (size_t i = 0; i < qs.size() && st == GPCH_OK; ++i) {
        const gpch_request &r = qs[i]->r;
        const size_t n = (size_t)r.n;
        double *dA = reinterpret_cast<double *>(b + oA[i]), *dX = reinterpret_cast<double *>(b + oX[i]);
        double *dB = reinterpret_cast<double *>(b + oB[i]);
        cudaMemcpyAsync(dX, r.X, n * r.d * 8, cudaMemcpyHostToDevice, L->stream);
        cudaMemcpyAsync(dB, r.B, n * r.nrhs * 8, cudaMemcpyHostToDevice, L->stream);
        st = gpch_se_matrix(L->ctx, r.n, r.d, dX, r.sf2, r.ell, r.sn2, dA, r.n, L->stream);
        sys[i] = gpch_system{r.n, dA, r.n, dB, r.n, r.nrhs};
    }
    std::vector<int64_t> info(qs.size(), 0);
    if (st == GPCH_OK) st = gpch::batched_solve_direct(L->ctx, (int)qs.size(), sys.data(), L->stream, info.data());
    for (size_t i = 0; i < qs.size(); ++i) {
        qs[i]->path = 1;
        qs[i]->status = st != GPCH_OK ? st : (info[i] != 0 ? GPCH_NOT_SPD : GPCH_OK);
        if (qs[i]->status == GPCH_OK)
            cudaMemcpyAsync(qs[i]->r.Xout, sys[i].B, (size_t)qs[i]->r.n * qs[i]->r.nrhs * 8, cudaMemcpyDeviceToHost,
                            L->stream);
    }
    if (cudaStreamSynchronize(L->stream) != cudaSuccess) {
        cudaGetLastError();
        for (auto *q : qs) q->status = GPCH_CUDA_ERROR;
    }
}

void lane_main(Lane *L)
{
    gpch_server *S = L->srv;
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        S->cv_dispatch.wait(lk, [&] { return S->stop || !L->job.empty(); });
        if (L->job.empty() && S->stop) break;
        std::vector<Req *> job = L->job;
        lk.unlock();
        const auto t0 = clk::now();
        for (auto *q : job) q->t_start = t0;
        if (job.size() == 1 && !is_small(S, job[0]->r)) run_solo(L, job[0]);
        else run_batch(L, job);
        const auto t1 = clk::now();
        lk.lock();
        for (auto *q : job) {
            q->t_end = t1;
            q->done = true;
            S->mem_reserved -= q->mem;
            if (q->status == GPCH_OK) {
                ++S->completed;
                S->latencies_ms.push_back(std::chrono::duration<double, std::milli>(t1 - q->t_submit).count());
            } else {
                ++S->failed;
            }
        }
        if (job.size() > 1 || is_small(S, job[0]->r)) {
            ++S->batches;
            S->batched_requests += (int64_t)job.size();
        }
        S->t_last_done = t1;
        L->job.clear();
        L->busy = false;
        S->cv_done.notify_all();
        S->cv_dispatch.notify_all();
    }
}

// Admit what fits, first fit in arrival order.  Called with the lock held.
void admit(gpch_server *S)
{
    for (Lane *L : S->lanes) {
        if (L->busy || S->queue.empty()) continue;
        std::vector<Req *> take;
        size_t mem = 0;
        for (auto it = S->queue.begin(); it != S->queue.end();) {
            Req *q = *it;
            const bool small = is_small(S, q->r);
            if (!take.empty() && (!small || (int)take.size() >= S->o.batch_max_count)) {
                ++it;
                continue;
            }
            const size_t need = request_bytes(q->r, !small && S->o.solo_prec != GPCH_PREC_FP64, pick_tile_dev(S->device, q->r.n));
            if (S->o.hbm_budget && S->mem_reserved + mem + need > S->o.hbm_budget) {
                ++it;
                continue;
            }
            q->mem = need;
            mem += need;
            take.push_back(q);
            it = S->queue.erase(it);
            if (!small) break;   // a large request runs alone
        }
        if (take.empty()) break;
        S->mem_reserved += mem;
        if (S->mem_reserved > S->mem_peak) S->mem_peak = S->mem_reserved;
        L->job = take;
        L->busy = true;
    }
}

void dispatcher_main(gpch_server *S)
{
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop) {
        admit(S);
        S->cv_dispatch.notify_all();
        S->cv_dispatch.wait_for(lk, std::chrono::microseconds(200));
    }
}

}  // namespace

extern "C" {

gpch_status gpch_server_create(int device, const gpch_server_opts *opts, gpch_server **out)
{
    if (!out || !opts) return GPCH_INVALID_ARG;
    *out = nullptr;
    if (opts->lanes < 1 || opts->lanes > 32 || opts->batch_max_count < 1 || opts->batch_max_n < 0 ||
        opts->bwd_tol <= 0.0)
        return GPCH_INVALID_ARG;
    if (opts->solo_prec != GPCH_PREC_FP64 && opts->solo_prec != GPCH_PREC_BF16 &&
        opts->solo_prec != GPCH_PREC_SPLIT_BF16 && opts->solo_prec != GPCH_PREC_SPLIT_F16)
        return GPCH_INVALID_ARG;
    gpch_server *S = new gpch_server();
    S->device = device;
    S->o = *opts;
    for (int i = 0; i < opts->lanes; ++i) {
        Lane *L = new Lane();
        L->srv = S;
        gpch_status st = gpch_create(&L->ctx, device, 0);
        if (st == GPCH_OK && cudaStreamCreateWithFlags(&L->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            st = GPCH_CUDA_ERROR;
        }
        if (st != GPCH_OK) {
            if (L->ctx) gpch_destroy(L->ctx);
            delete L;
            for (Lane *M : S->lanes) {
                cudaStreamDestroy(M->stream);
                gpch_destroy(M->ctx);
                delete M;
            }
            delete S;
            return st;
        }
        S->lanes.push_back(L);
    }
    for (Lane *L : S->lanes) L->th = std::thread(lane_main, L);
    S->dispatcher = std::thread(dispatcher_main, S);
    *out = S;
    return GPCH_OK;
}

gpch_status gpch_server_submit(gpch_server *S, const gpch_request *r, uint64_t *ticket)
{
    if (!S || !r || !ticket) return GPCH_INVALID_ARG;
    if (r->n < 1 || r->d < 1 || r->d > 64 || r->nrhs < 1 || r->ell <= 0.0 || !r->X || !r->B || !r->Xout)
        return GPCH_INVALID_ARG;
    const bool small = r->n <= S->o.batch_max_n;
    const size_t need = request_bytes(*r, !small && S->o.solo_prec != GPCH_PREC_FP64, pick_tile_dev(S->device, r->n));
    if (S->o.hbm_budget && need > S->o.hbm_budget) return GPCH_OOM_BUDGET;
    Req *q = new Req();
    q->r = *r;
    q->t_submit = clk::now();
    std::lock_guard<std::mutex> lk(S->mu);
    q->ticket = S->next_ticket++;
    if (!S->any_submit) {
        S->any_submit = true;
        S->t_first_submit = q->t_submit;
    }
    S->reqs[q->ticket] = q;
    S->queue.push_back(q);
    admit(S);
    S->cv_dispatch.notify_all();
    *ticket = q->ticket;
    return GPCH_OK;
}

static void fill_result(const Req *q, gpch_result *res)
{
    if (!res) return;
    res->status = q->status;
    res->path = q->path;
    res->iterations = q->iterations;
    res->backward_error = q->backward_error;
    res->latency_ms = std::chrono::duration<double, std::milli>(q->t_end - q->t_submit).count();
    res->queue_ms = std::chrono::duration<double, std::milli>(q->t_start - q->t_submit).count();
}

gpch_status gpch_server_wait(gpch_server *S, uint64_t ticket, double timeout_s, gpch_result *res)
{
    if (!S) return GPCH_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return GPCH_INVALID_ARG;
    Req *q = it->second;
    const auto deadline = clk::now() + std::chrono::duration_cast<clk::duration>(std::chrono::duration<double>(timeout_s));
    while (!q->done) {
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !q->done) return GPCH_TIMEOUT;
    }
    fill_result(q, res);
    S->reqs.erase(it);
    const gpch_status st = q->status;
    delete q;
    return st;
}

gpch_status gpch_server_poll(gpch_server *S, uint64_t ticket, int *done, gpch_result *res)
{
    if (!S || !done) return GPCH_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return GPCH_INVALID_ARG;
    *done = it->second->done ? 1 : 0;
    if (*done) fill_result(it->second, res);
    return GPCH_OK;
}

gpch_status gpch_server_get_stats(gpch_server *S, gpch_server_stats *out)
{
    if (!S || !out) return GPCH_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    *out = gpch_server_stats{};
    out->completed = S->completed;
    out->failed = S->failed;
    out->batches = S->batches;
    out->batched_requests = S->batched_requests;
    out->peak_reserved_bytes = S->mem_peak;
    std::vector<double> v = S->latencies_ms;
    if (!v.empty()) {
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) {
            const double pos = p * (double)(v.size() - 1);
            const size_t i = (size_t)pos;
            const double f = pos - (double)i;
            return i + 1 < v.size() ? v[i] * (1.0 - f) + v[i + 1] * f : v[i];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        out->max_ms = v.back();
        const double span = std::chrono::duration<double>(S->t_last_done - S->t_first_submit).count();
        out->solves_per_s = span > 0 ? (double)S->completed / span : 0.0;
    }
    return GPCH_OK;
}

gpch_status gpch_server_destroy(gpch_server *S)
{
    if (!S) return GPCH_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_dispatch.notify_all();
    if (S->dispatcher.joinable()) S->dispatcher.join();
    for (Lane *L : S->lanes) {
        if (L->th.joinable()) L->th.join();
        if (L->buf) cudaFree(L->buf);
        cudaStreamDestroy(L->stream);
        gpch_destroy(L->ctx);
        delete L;
    }
    for (auto &kv : S->reqs) delete kv.second;
    for (Req *q : S->queue) (void)q;   // queued requests are owned by reqs
    delete S;
    return GPCH_OK;
}

}  // extern "C"
