// tuner.cu -- tile-width choice for the dense tensor-core GEMM: a per-thread
// override, and a measured autotuner whose results refine the shape planner.
//
// The paper derives its block sizes from the static shapes and types and
// then confirms the best one by measurement (Sec. 3.4: 32x32 doubles best,
// then 64x64).  Here the static rule is the planner in dense_tc_launch; the
// measured step is moa_tune_dense, which times every tile width on the
// caller's buffers and records the fastest for the problem's shape bucket
// (half-octaves of m, n, p, per precision mode).  Later calls in that bucket
// use the recorded width.  The table can be saved to and loaded from a text
// file (also loaded from MOA_TUNE_CACHE on first use).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>

#include "internal.h"

namespace moa {
int gemm_ex(int64_t m, int64_t n, int64_t p, moa_dtype dt, const void* A, const void* B, void* C,
            int slices, void* ws, size_t ws_bytes, cudaStream_t s, moa_stats* st);

namespace {
thread_local int t_override = 0;
thread_local int t_override_m = 0;
std::mutex g_mu;
using Key = std::tuple<int, int, int, int>;
std::map<Key, int> g_table;
bool g_loaded = false;

int bucket(int64_t x) { return x <= 1 ? 0 : static_cast<int>(std::lround(2.0 * std::log2(double(x)))); }
Key key_of(moa_dtype dt, int64_t m, int64_t n, int64_t p) {
    return Key{static_cast<int>(dt), bucket(m), bucket(n), bucket(p)};
}

int load_locked(const char* path) {
    FILE* f = std::fopen(path, "r");
    if (!f) return fail(MOA_ERR_ARG, std::string("cannot open tune cache ") + path);
    int dt, bm, bnn, bp, w, count = 0;
    while (std::fscanf(f, "%d %d %d %d %d", &dt, &bm, &bnn, &bp, &w) == 5) {
        if (w == 64 || w == 128 || w == 256) {
            g_table[Key{dt, bm, bnn, bp}] = w;
            ++count;
        }
    }
    std::fclose(f);
    return MOA_OK;
}
}  // namespace

int tile_override() { return t_override; }
int tile_m_override() { return t_override_m; }

// MOA_RASTER_GROUP if set (1..1024), else 0.
static int raster_env() {
    static int g = -1;
    if (g < 0) {
        const char* env = std::getenv("MOA_RASTER_GROUP");
        const long v = env ? std::strtol(env, nullptr, 10) : 0;
        g = static_cast<int>(v >= 1 && v <= 1024 ? v : 0);
    }
    return g;
}

int raster_group() {
    const int g = raster_env();
    return g ? g : 16;
}

int split_raster_group(int64_t n) {
    const int g = raster_env();
    return g ? g : (n > 12288 ? 8 : 16);
}

int tuned_block_n(moa_dtype dt, int64_t m, int64_t n, int64_t p) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_loaded) {
        g_loaded = true;
        if (const char* env = std::getenv("MOA_TUNE_CACHE")) load_locked(env);
    }
    auto it = g_table.find(key_of(dt, m, n, p));
    return it == g_table.end() ? 0 : it->second;
}

}  // namespace moa

extern "C" {

int moa_set_block_n(int block_n) {
    if (block_n != 0 && block_n != 64 && block_n != 128 && block_n != 192 && block_n != 256)
        return moa::fail(MOA_ERR_ARG, "block_n must be 0, 64, 128, 192 or 256");
    moa::t_override = block_n;
    return MOA_OK;
}

int moa_set_block_m(int block_m) {
    if (block_m != 0 && block_m != 128 && block_m != 256)
        return moa::fail(MOA_ERR_ARG, "block_m must be 0, 128 or 256");
    moa::t_override_m = block_m;
    return MOA_OK;
}

int moa_tune_dense(int64_t m, int64_t n, int64_t p, moa_dtype dt, const void* A, const void* B,
                   void* C, void* ws, size_t ws_bytes, void* stream, int* best_block_n,
                   float* best_ms) {
    if (dt != MOA_BF16 && dt != MOA_F32_TF32)
        return moa::fail(MOA_ERR_DTYPE, "only the dense tensor-core modes have tile widths");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return moa::fail(MOA_ERR_CUDA, "cudaEventCreate");
    const int saved = moa::t_override;
    int best = 0;
    float best_t = 1e30f;
    int rc = MOA_OK;
    for (int w : {256, 128, 64}) {
        moa::t_override = w;
        rc = moa::gemm_ex(m, n, p, dt, A, B, C, 0, ws, ws_bytes, s, nullptr);   // warm-up
        if (rc != MOA_OK) break;
        cudaEventRecord(e0, s);
        for (int r = 0; r < 3; ++r) {
            rc = moa::gemm_ex(m, n, p, dt, A, B, C, 0, ws, ws_bytes, s, nullptr);
            if (rc != MOA_OK) break;
        }
        cudaEventRecord(e1, s);
        if (rc != MOA_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = moa::fail(MOA_ERR_CUDA, "cudaEventSynchronize");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= 3.f;
        if (ms < best_t) {
            best_t = ms;
            best = w;
        }
    }
    moa::t_override = saved;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != MOA_OK) return rc;
    {
        std::lock_guard<std::mutex> lk(moa::g_mu);
        moa::g_table[moa::key_of(dt, m, n, p)] = best;
    }
    if (best_block_n) *best_block_n = best;
    if (best_ms) *best_ms = best_t;
    return MOA_OK;
}

int moa_tune_save(const char* path) {
    if (!path) return moa::fail(MOA_ERR_ARG, "NULL path");
    std::lock_guard<std::mutex> lk(moa::g_mu);
    FILE* f = std::fopen(path, "w");
    if (!f) return moa::fail(MOA_ERR_ARG, std::string("cannot write ") + path);
    for (const auto& kv : moa::g_table)
        std::fprintf(f, "%d %d %d %d %d\n", std::get<0>(kv.first), std::get<1>(kv.first),
                     std::get<2>(kv.first), std::get<3>(kv.first), kv.second);
    std::fclose(f);
    return MOA_OK;
}

int moa_tune_load(const char* path) {
    if (!path) return moa::fail(MOA_ERR_ARG, "NULL path");
    std::lock_guard<std::mutex> lk(moa::g_mu);
    moa::g_loaded = true;
    return moa::load_locked(path);
}

int moa_tune_clear(void) {
    std::lock_guard<std::mutex> lk(moa::g_mu);
    moa::g_table.clear();
    return MOA_OK;
}

}  // extern "C"
