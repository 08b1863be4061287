// sigk_tune.cu -- autotuner of the launch configuration (host code).
//
// The solver's arithmetic is fixed by the truncation (order, rings,
// refinement, ring tolerance: sigk_plan); what remains free is how the work
// is laid out on the GPU:
//   * the persistent grid (the wavefront's width: how many strips are in
//     flight at once) -- the occupancy-derived full grid, three quarters or
//     one half of it;
//   * the schedule -- strip-major (strip l of every pair before strip l + 1 of
//     any) or pair-major (a pair's strips consecutive);
//   * for 16 < d <= 1024, the increment Gram -- tensor cores (float-float
//     coefficients) or the FP32 FMA micro-GEMM.
// sigk_autotune times every candidate on the caller's own inputs (CUDA events
// on the caller's stream, one warm-up and two timed calls each) and keeps the
// fastest per shape class in an in-process cache; sigk_plan consults that
// cache, so a planned call of a tuned class gets the tuned layout.  The cache
// can be saved to and loaded from a text file (one line per class:
// key, grid_ctas, flags, milliseconds).  The results of every candidate are
// identical up to rounding (the schedules and grids bitwise), so tuning never
// trades accuracy; the FP32 FMA Gram rounds the coefficients to FP32 and is a
// candidate only when the caller allows it (allow_fma_gram).
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/sigk.h"

namespace {

struct Tuned {
    int grid_ctas;
    int flags;
    double ms;
};

std::mutex g_mu;
std::map<std::string, Tuned> g_cache;

// Flags that the tuner chooses (the others belong to the caller's problem).
constexpr int kTunedFlags = SIGK_FLAG_PAIR_MAJOR | SIGK_FLAG_NO_TENSOR;

int pow2_ceil(int64_t v) {
    int k = 0;
    while (((int64_t)1 << k) < v && k < 62) ++k;
    return k;
}

}  // namespace

extern "C" {

// The shape class of a call: the op, the batch sizes, d, the swept-length
// bound rounded up to a power of two, the truncation and the problem flags.
sigk_status sigk_tune_key(int op, int64_t n_x, int64_t n_y, int d, const sigk_opts* opts, char* buf,
                          size_t buf_len) {
    if (!opts || !buf || buf_len < 96) return SIGK_ERR_ARG;
    if (op < SIGK_OP_PAIRS || op > SIGK_OP_MMD || n_x < 0 || n_y < 0 || d < 1) return SIGK_ERR_ARG;
    const int pf = opts->flags & ~kTunedFlags & ~SIGK_FLAG_TEST_WITHHOLD_SEAM;
    const int n = snprintf(buf, buf_len, "op%d_nx%lld_ny%lld_d%d_L2^%d_P%d_n%d_f%d_r%d_a%d", op,
                           (long long)n_x, (long long)n_y, d, pow2_ceil(opts->max_len > 0 ? opts->max_len : 8193),
                           opts->order, opts->rings, pf, opts->refine_c > 0.0f ? 1 : 0,
                           opts->ring_tol > 0.0f ? 1 : 0);
    return (n > 0 && (size_t)n < buf_len) ? SIGK_OK : SIGK_ERR_ARG;
}

// Cache access (no GPU needed): put overwrites, get returns SIGK_ERR_ARG when
// the key is absent and otherwise merges the tuned fields into *opts.
sigk_status sigk_tune_cache_put(const char* key, int grid_ctas, int flags, double ms) {
    if (!key || grid_ctas < 0) return SIGK_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    g_cache[key] = Tuned{grid_ctas, flags & kTunedFlags, ms};
    return SIGK_OK;
}

sigk_status sigk_tune_cache_get(const char* key, sigk_opts* opts, double* ms) {
    if (!key || !opts) return SIGK_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(key);
    if (it == g_cache.end()) return SIGK_ERR_ARG;
    opts->grid_ctas = it->second.grid_ctas;
    opts->flags = (opts->flags & ~kTunedFlags) | it->second.flags;
    if (ms) *ms = it->second.ms;
    return SIGK_OK;
}

int64_t sigk_tune_cache_size(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    return (int64_t)g_cache.size();
}

void sigk_tune_cache_clear(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_cache.clear();
}

sigk_status sigk_tune_cache_save(const char* path) {
    if (!path) return SIGK_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    FILE* f = fopen(path, "w");
    if (!f) return SIGK_ERR_ARG;
    for (const auto& kv : g_cache)
        fprintf(f, "%s %d %d %.6f\n", kv.first.c_str(), kv.second.grid_ctas, kv.second.flags, kv.second.ms);
    return fclose(f) == 0 ? SIGK_OK : SIGK_ERR_ARG;
}

// Adds the file's entries to the cache (a malformed line fails the load,
// keeping the entries before it).
sigk_status sigk_tune_cache_load(const char* path) {
    if (!path) return SIGK_ERR_ARG;
    FILE* f = fopen(path, "r");
    if (!f) return SIGK_ERR_ARG;
    char key[256];
    int grid = 0, flags = 0;
    double ms = 0.0;
    sigk_status st = SIGK_OK;
    for (;;) {
        const int r = fscanf(f, "%255s %d %d %lf", key, &grid, &flags, &ms);
        if (r == EOF) break;
        if (r != 4 || grid < 0) {
            st = SIGK_ERR_ARG;
            break;
        }
        std::lock_guard<std::mutex> lk(g_mu);
        g_cache[key] = Tuned{grid, flags & kTunedFlags, ms};
    }
    fclose(f);
    return st;
}

// Times the op under every candidate layout and caches the fastest.
sigk_status sigk_autotune(int op, const float* X, const int64_t* len_x, int64_t n_x, const float* Y,
                          const int64_t* len_y, int64_t n_y, int d, double* out_scratch, void* ws,
                          size_t ws_bytes, void* stream, const sigk_opts* opts_in, int allow_fma_gram,
                          sigk_opts* opts_out, double* ms_out) {
    if (!opts_in || !opts_out || !out_scratch) return SIGK_ERR_ARG;
    if (op == SIGK_OP_GRAM && !Y) n_y = 0;
    if (op == SIGK_OP_PAIRS) n_y = n_x;
    char key[256];
    sigk_status st = sigk_tune_key(op, n_x, n_y, d, opts_in, key, sizeof(key));
    if (st != SIGK_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const bool allow_fma = allow_fma_gram != 0;
    const bool tc_range = d > 16 && d <= 1024 && !(opts_in->flags & SIGK_FLAG_FP64) &&
                          !(opts_in->flags & SIGK_FLAG_NO_TENSOR);
    // candidates: grid (0 = full occupancy, or a fraction of it, as CTAs) x
    // schedule x Gram path
    if (!sigk_workspace_size(op, n_x, n_y, d, opts_in)) return SIGK_ERR_ARG;
    std::vector<sigk_opts> cand;
    for (int g = 0; g < 3; ++g) {
        for (int pm = 0; pm < 2; ++pm) {
            for (int fm = 0; fm < ((tc_range && allow_fma) ? 2 : 1); ++fm) {
                sigk_opts o = *opts_in;
                o.flags &= ~SIGK_FLAG_PAIR_MAJOR;
                if (pm) o.flags |= SIGK_FLAG_PAIR_MAJOR;
                if (fm) o.flags |= SIGK_FLAG_NO_TENSOR;
                o.grid_ctas = 0;
                if (g > 0) {
                    // a fraction of the occupancy-derived grid (up to 4 CTAs per SM)
                    o.grid_ctas = g == 1 ? 3 * sms : 2 * sms;
                }
                cand.push_back(o);
            }
        }
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return SIGK_ERR_CUDA;
    double best = 1e300;
    sigk_opts best_o = *opts_in;
    for (const sigk_opts& o : cand) {
        const size_t need = sigk_workspace_size(op, n_x, n_y, d, &o);
        if (!need || need > ws_bytes) continue;
        auto run = [&]() -> sigk_status {
            if (op == SIGK_OP_PAIRS)
                return sigk_pairs(X, len_x, Y, len_y, n_x, d, out_scratch, ws, ws_bytes, stream, &o);
            if (op == SIGK_OP_GRAM)
                return sigk_gram(X, len_x, n_x, n_y ? Y : nullptr, len_y, n_y, d, out_scratch, ws, ws_bytes,
                                 stream, &o);
            return sigk_mmd(X, len_x, n_x, Y, len_y, n_y, d, out_scratch, nullptr, ws, ws_bytes, stream, &o);
        };
        if ((st = run()) != SIGK_OK) break;  // warm-up
        if ((st = sigk_sync_status(ws, ws_bytes, stream)) != SIGK_OK) break;
        cudaEventRecord(e0, s);
        for (int r = 0; r < 2 && st == SIGK_OK; ++r) st = run();
        cudaEventRecord(e1, s);
        if (st != SIGK_OK) break;
        if ((st = sigk_sync_status(ws, ws_bytes, stream)) != SIGK_OK) break;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms * 0.5 < best) {
            best = ms * 0.5;
            best_o = o;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != SIGK_OK) return st;
    if (best >= 1e300) return SIGK_ERR_WORKSPACE;  // no candidate layout fits the workspace
    sigk_tune_cache_put(key, best_o.grid_ctas, best_o.flags, best);
    *opts_out = best_o;
    if (ms_out) *ms_out = best;
    return SIGK_OK;
}

}  // extern "C"
