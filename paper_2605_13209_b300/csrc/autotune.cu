// autotune.cu -- tile choices measured on the GPU at hand.
//
// Two kinds of tile are tuned, per problem-size bucket (n <= 512, 1024,
// ..., 65536, larger):
//   * the refined solve's tile (the block size of the mixed factor's
//     Algorithm 1, candidates 256, 384, 512): it sets the length of the
//     FP64 diagonal chain against the size of the tensor-core update passes;
//   * the batched factors' trailing-update tile (32 or 64 rows and columns
//     per CTA), for the FP64 and the mixed batch: small systems give few
//     64 x 64 tiles per step, so smaller tiles can fill the GPU better.  The
//     result of a batched solve does not depend on this tile.
// The tuner times every candidate with CUDA events on synthetic
// squared-exponential systems generated on the device (points from a
// counter-based generator, splitmix64), keeps the fastest, and stores the
// table in a JSON file keyed by the GPU's name, from which later processes
// load it instead of measuring.  Until a table is measured or loaded the
// defaults below hold.
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.cuh"

namespace gpch {

namespace {

std::mutex g_tune_mu;
std::map<int, TuneTable> g_tune;

TuneTable default_table()
{
    TuneTable t{};
    for (int b = 0; b < TUNE_BUCKETS; ++b) {
        t.refined_tile[b] = b <= 3 ? 256 : 512;   // n <= 4096: 256
        t.batch_bt[0][b] = 64;
        t.batch_bt[1][b] = 64;
    }
    t.tuned = 0;
    return t;
}

}  // namespace

int tune_bucket(int64_t n)
{
    int b = 0;
    int64_t lim = 512;
    while (b < TUNE_BUCKETS - 1 && n > lim) {
        lim *= 2;
        ++b;
    }
    return b;
}

TuneTable tune_table(int device)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(device);
    return it == g_tune.end() ? default_table() : it->second;
}

void tune_set(int device, const TuneTable &t)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[device] = t;
}

}  // namespace gpch

namespace {

using gpch::TUNE_BUCKETS;
using gpch::TuneTable;

// ------------------------------------------------------------ JSON cache
//
// {"<gpu name>": {"refined_tile": [9 ints], "batch_tile_fp64": [9 ints],
//                 "batch_tile_mixed": [9 ints]}, ...}

std::string read_file(const char *path)
{
    std::string s;
    FILE *f = std::fopen(path, "rb");
    if (!f) return s;
    char buf[4096];
    size_t k;
    while ((k = std::fread(buf, 1, sizeof(buf), f)) > 0) s.append(buf, k);
    std::fclose(f);
    return s;
}

// Top-level "name": {object} pairs of the cache file, object text kept raw.
std::vector<std::pair<std::string, std::string>> split_entries(const std::string &s)
{
    std::vector<std::pair<std::string, std::string>> out;
    size_t i = s.find('{');
    if (i == std::string::npos) return out;
    ++i;
    while (true) {
        const size_t q0 = s.find('"', i);
        if (q0 == std::string::npos) break;
        const size_t q1 = s.find('"', q0 + 1);
        if (q1 == std::string::npos) break;
        const size_t b0 = s.find('{', q1);
        if (b0 == std::string::npos) break;
        int depth = 0;
        size_t j = b0;
        for (; j < s.size(); ++j) {
            if (s[j] == '{') ++depth;
            if (s[j] == '}' && --depth == 0) break;
        }
        if (j >= s.size()) break;
        out.emplace_back(s.substr(q0 + 1, q1 - q0 - 1), s.substr(b0, j - b0 + 1));
        i = j + 1;
    }
    return out;
}

bool parse_array(const std::string &obj, const char *key, int *vals)
{
    const std::string k = std::string("\"") + key + "\"";
    size_t p = obj.find(k);
    if (p == std::string::npos) return false;
    p = obj.find('[', p);
    if (p == std::string::npos) return false;
    ++p;
    for (int b = 0; b < TUNE_BUCKETS; ++b) {
        char *end = nullptr;
        const long v = std::strtol(obj.c_str() + p, &end, 10);
        if (end == obj.c_str() + p) return false;
        vals[b] = (int)v;
        p = (size_t)(end - obj.c_str());
        while (p < obj.size() && (obj[p] == ',' || obj[p] == ' ')) ++p;
    }
    return true;
}

bool valid_table(const TuneTable &t)
{
    for (int b = 0; b < TUNE_BUCKETS; ++b) {
        if (t.refined_tile[b] < 64 || t.refined_tile[b] > 1024 || t.refined_tile[b] % 64) return false;
        for (int p = 0; p < 2; ++p)
            if (t.batch_bt[p][b] != 32 && t.batch_bt[p][b] != 64) return false;
    }
    return true;
}

bool load_entry(const char *path, const std::string &gpu, TuneTable &t)
{
    if (!path) return false;
    const std::string s = read_file(path);
    for (auto &e : split_entries(s)) {
        if (e.first != gpu) continue;
        TuneTable x{};
        if (parse_array(e.second, "refined_tile", x.refined_tile) &&
            parse_array(e.second, "batch_tile_fp64", x.batch_bt[0]) &&
            parse_array(e.second, "batch_tile_mixed", x.batch_bt[1]) && valid_table(x)) {
            x.tuned = 2;
            t = x;
            return true;
        }
    }
    return false;
}

std::string array_text(const int *v)
{
    std::string s = "[";
    for (int b = 0; b < TUNE_BUCKETS; ++b) {
        s += std::to_string(v[b]);
        if (b + 1 < TUNE_BUCKETS) s += ", ";
    }
    return s + "]";
}

// Writes the cache with this GPU's entry replaced or added; other GPUs'
// entries are kept as they were.  Returns false if the file cannot be
// written (the measured table still applies to this process).
bool save_entry(const char *path, const std::string &gpu, const TuneTable &t)
{
    if (!path) return false;
    auto entries = split_entries(read_file(path));
    const std::string mine = std::string("{\"refined_tile\": ") + array_text(t.refined_tile) +
                             ", \"batch_tile_fp64\": " + array_text(t.batch_bt[0]) +
                             ", \"batch_tile_mixed\": " + array_text(t.batch_bt[1]) + "}";
    bool found = false;
    for (auto &e : entries)
        if (e.first == gpu) {
            e.second = mine;
            found = true;
        }
    if (!found) entries.emplace_back(gpu, mine);
    FILE *f = std::fopen(path, "wb");
    if (!f) return false;
    std::fputs("{\n", f);
    for (size_t i = 0; i < entries.size(); ++i)
        std::fprintf(f, "  \"%s\": %s%s\n", entries[i].first.c_str(), entries[i].second.c_str(),
                     i + 1 < entries.size() ? "," : "");
    std::fputs("}\n", f);
    return std::fclose(f) == 0;
}

}  // namespace

// ------------------------------------------------------------ measurement

namespace {

// Points uniform on [0,1)^d from splitmix64 of (seed, index): the 53 top
// bits of the mixed counter, as a double.
__global__ void tune_points_kernel(int64_t count, uint64_t seed, double *X)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    uint64_t z = seed + 0x9e3779b97f4a7c15ull * (uint64_t)(i + 1);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z ^= z >> 31;
    X[i] = (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

struct DevBuf {
    void *p = nullptr;
    ~DevBuf()
    {
        if (p) cudaFree(p);
    }
};

gpch_status dev_alloc(gpch_ctx *ctx, DevBuf &b, size_t bytes)
{
    if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return gpch::fail(ctx, GPCH_OOM_BUDGET, "autotune: cudaMalloc(%zu) failed", bytes);
    }
    return GPCH_OK;
}

// One SE system of size n (d = 8, ell = 0.5, sn2 = 1e-3) into A (ld n);
// points at X (8 n doubles); right-hand side of ones at B (n doubles).
gpch_status tune_system(gpch_ctx *ctx, int64_t n, uint64_t seed, double *X, double *A, double *B, cudaStream_t s)
{
    tune_points_kernel<<<(unsigned)((8 * n + 255) / 256), 256, 0, s>>>(8 * n, seed, X);
    GPCH_LAUNCH_CHECK(ctx);
    GPCH_CHECK(gpch_se_matrix(ctx, n, 8, X, 1.0, 0.5, 1e-3, A, n, s));
    if (B) {
        std::vector<double> ones((size_t)n, 1.0);
        GPCH_CUDA(ctx, cudaMemcpyAsync(B, ones.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
        GPCH_CUDA(ctx, cudaStreamSynchronize(s));
    }
    return GPCH_OK;
}

// Milliseconds of `run` (the fastest of `reps` after one warm-up),
// measured with CUDA events on s; `prep` runs untimed before each.
template <typename P, typename R>
gpch_status time_best(gpch_ctx *ctx, cudaStream_t s, int reps, P &&prep, R &&run, float *best)
{
    cudaEvent_t e0, e1;
    GPCH_CUDA(ctx, cudaEventCreate(&e0));
    GPCH_CUDA(ctx, cudaEventCreate(&e1));
    *best = 1e30f;
    gpch_status st = GPCH_OK;
    for (int r = 0; r <= reps && st == GPCH_OK; ++r) {
        st = prep();
        if (st != GPCH_OK) break;
        cudaEventRecord(e0, s);
        st = run();
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            cudaGetLastError();
            st = gpch::fail(ctx, GPCH_CUDA_ERROR, "autotune: event synchronize failed");
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0 && st == GPCH_OK && ms < *best) *best = ms;   // r = 0 is the warm-up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

// Fill unmeasured buckets from the nearest measured one.
void fill_nearest(int *v, const bool *have)
{
    for (int b = 0; b < TUNE_BUCKETS; ++b) {
        if (have[b]) continue;
        for (int d = 1; d < TUNE_BUCKETS; ++d) {
            if (b - d >= 0 && have[b - d]) {
                v[b] = v[b - d];
                break;
            }
            if (b + d < TUNE_BUCKETS && have[b + d]) {
                v[b] = v[b + d];
                break;
            }
        }
    }
}

gpch_status measure(gpch_ctx *ctx, int64_t nmax, TuneTable &t)
{
    cudaStream_t s;
    GPCH_CUDA(ctx, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    gpch_ctx *tc = nullptr;   // a private context: its workspace and plans go away with it
    gpch_status st = gpch_create(&tc, ctx->device, 0);
    if (st != GPCH_OK) {
        cudaStreamDestroy(s);
        return gpch::fail(ctx, st, "autotune: context creation failed");
    }
    bool have_r[TUNE_BUCKETS] = {}, have_b[2][TUNE_BUCKETS] = {};
    // refined solve: tile per n
    for (int64_t n = 1024; n <= nmax && st == GPCH_OK; n *= 2) {
        DevBuf X, A, B, Xs;
        if ((st = dev_alloc(ctx, X, 8 * n * sizeof(double))) != GPCH_OK) break;
        if ((st = dev_alloc(ctx, A, (size_t)n * n * sizeof(double))) != GPCH_OK) break;
        if ((st = dev_alloc(ctx, B, n * sizeof(double))) != GPCH_OK) break;
        if ((st = dev_alloc(ctx, Xs, n * sizeof(double))) != GPCH_OK) break;
        double *dA = static_cast<double *>(A.p), *dB = static_cast<double *>(B.p), *dX = static_cast<double *>(Xs.p);
        if ((st = tune_system(ctx, n, 0x7e57ull + n, static_cast<double *>(X.p), dA, dB, s)) != GPCH_OK) break;
        float best = 1e30f;
        int pick = 0;
        for (int tile : {256, 384, 512}) {
            if (tile > n) continue;
            float ms = 0.f;
            gpch_status rs = time_best(
                ctx, s, 2, [] { return GPCH_OK; },
                [&] {
                    return gpch_solve_refined(tc, n, dA, n, dB, n, dX, n, 1, GPCH_PREC_SPLIT_F16, tile, 1e-12, 500, s,
                                              nullptr);
                },
                &ms);
            if (rs != GPCH_OK) continue;   // a tile that fails here is not chosen
            if (ms < best) {
                best = ms;
                pick = tile;
            }
        }
        if (pick) {
            const int b = gpch::tune_bucket(n);
            t.refined_tile[b] = pick;
            have_r[b] = true;
        }
    }
    // batched solves: trailing-update tile per n
    for (int64_t n = 256; n <= 4096 && st == GPCH_OK; n *= 2) {
        const int count = (int)(65536 / n < 8 ? 8 : 65536 / n);
        DevBuf X, A, B, Xs;
        if ((st = dev_alloc(ctx, X, 8 * n * sizeof(double))) != GPCH_OK) break;
        if ((st = dev_alloc(ctx, A, (size_t)count * n * n * sizeof(double))) != GPCH_OK) break;
        if ((st = dev_alloc(ctx, B, (size_t)count * n * sizeof(double))) != GPCH_OK) break;
        if ((st = dev_alloc(ctx, Xs, (size_t)count * n * sizeof(double))) != GPCH_OK) break;
        double *dA = static_cast<double *>(A.p), *dB = static_cast<double *>(B.p), *dX = static_cast<double *>(Xs.p);
        auto regen = [&]() -> gpch_status {
            for (int i = 0; i < count; ++i)
                GPCH_CHECK(tune_system(ctx, n, 0xba7cull + 131 * i + n, static_cast<double *>(X.p),
                                       dA + (size_t)i * n * n, dB + (size_t)i * n, s));
            return GPCH_OK;
        };
        std::vector<gpch_system> fs(count);
        std::vector<gpch_msystem> ms(count);
        for (int i = 0; i < count; ++i) {
            fs[i] = gpch_system{n, dA + (size_t)i * n * n, n, dB + (size_t)i * n, n, 1};
            ms[i] = gpch_msystem{n, dA + (size_t)i * n * n, n, dB + (size_t)i * n, n, dX + (size_t)i * n, n, 1};
        }
        std::vector<int64_t> info(count);
        const int b = gpch::tune_bucket(n);
        for (int p = 0; p < 2 && st == GPCH_OK; ++p) {
            // the FP64 batch factors A in place (regenerated before each of
            // its runs); the mixed batch reads it, so one fresh copy serves
            if (p == 1 && (st = regen()) != GPCH_OK) break;
            float best = 1e30f;
            int pick = 0;
            for (int bt : {64, 32}) {
                TuneTable trial = gpch::tune_table(ctx->device);
                for (int q = 0; q < TUNE_BUCKETS; ++q) trial.batch_bt[p][q] = bt;
                gpch::tune_set(ctx->device, trial);
                float msec = 0.f;
                gpch_status rs;
                if (p == 0)
                    rs = time_best(ctx, s, 2, regen,
                                   [&] { return gpch_batched_solve(tc, count, fs.data(), s, info.data()); }, &msec);
                else
                    rs = time_best(ctx, s, 2, [] { return GPCH_OK; },
                                   [&] {
                                       return gpch_batched_solve_mixed(tc, count, ms.data(), 1e-12, 30, s, info.data(),
                                                                       nullptr);
                                   },
                                   &msec);
                if (rs == GPCH_OK && msec < best) {
                    best = msec;
                    pick = bt;
                }
            }
            if (pick) {
                t.batch_bt[p][b] = pick;
                have_b[p][b] = true;
            }
        }
    }
    gpch_destroy(tc);
    cudaStreamDestroy(s);
    if (st != GPCH_OK) return st;
    fill_nearest(t.refined_tile, have_r);
    fill_nearest(t.batch_bt[0], have_b[0]);
    fill_nearest(t.batch_bt[1], have_b[1]);
    t.tuned = 1;
    return GPCH_OK;
}

void to_info(const TuneTable &t, const char *gpu, gpch_tune_info *out)
{
    if (!out) return;
    std::memset(out, 0, sizeof(*out));
    out->source = t.tuned;
    for (int b = 0; b < TUNE_BUCKETS; ++b) {
        out->refined_tile[b] = t.refined_tile[b];
        out->batch_tile_fp64[b] = t.batch_bt[0][b];
        out->batch_tile_mixed[b] = t.batch_bt[1][b];
    }
    std::snprintf(out->gpu, sizeof(out->gpu), "%s", gpu);
}

gpch_status gpu_name(gpch_ctx *ctx, std::string &name)
{
    cudaDeviceProp prop;
    GPCH_CUDA(ctx, cudaGetDeviceProperties(&prop, ctx->device));
    name = prop.name;
    for (char &c : name)
        if (c == '"' || c == '\\') c = '_';
    return GPCH_OK;
}

}  // namespace

extern "C" gpch_status gpch_autotune(gpch_ctx *ctx, const char *cache_path, int force, int64_t nmax,
                                     gpch_tune_info *out)
{
    GPCH_ARG(ctx, ctx != nullptr, "null context");
    if (nmax == 0) nmax = 32768;
    GPCH_ARG(ctx, nmax >= 1024 && nmax <= 65536, "nmax must be in [1024, 65536] (or 0)");
    GPCH_CUDA(ctx, cudaSetDevice(ctx->device));
    std::string gpu;
    GPCH_CHECK(gpu_name(ctx, gpu));
    TuneTable t = gpch::tune_table(ctx->device);
    if (!force && load_entry(cache_path, gpu, t)) {
        gpch::tune_set(ctx->device, t);
        to_info(t, gpu.c_str(), out);
        return GPCH_OK;
    }
    const TuneTable before = gpch::tune_table(ctx->device);
    TuneTable m = before;
    gpch_status st = measure(ctx, nmax, m);
    if (st != GPCH_OK) {
        gpch::tune_set(ctx->device, before);   // the trial tables of the batch timing are not kept
        return st;
    }
    gpch::tune_set(ctx->device, m);
    save_entry(cache_path, gpu, m);
    to_info(m, gpu.c_str(), out);
    return GPCH_OK;
}

extern "C" gpch_status gpch_tune_get(gpch_ctx *ctx, gpch_tune_info *out)
{
    GPCH_ARG(ctx, ctx != nullptr, "null context");
    GPCH_ARG(ctx, out != nullptr, "null output");
    std::string gpu;
    GPCH_CHECK(gpu_name(ctx, gpu));
    to_info(gpch::tune_table(ctx->device), gpu.c_str(), out);
    return GPCH_OK;
}
