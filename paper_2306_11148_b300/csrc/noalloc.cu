// noalloc.cu -- moa_gemm_f32split_noalloc: the FP32-accuracy split GEMM for
// callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at all: real-time or safety-certified
// hosts whose device memory is fixed at start-up (a run-time allocation can
// block, synchronise the device or fail late), plugins that live inside
// another runtime's memory pool and are handed no allocator, and embedded
// deployments with a static memory plan.  For them this entry point keeps its
// scratch (the three BF16 slice planes of A and of B, and for few-tile
// problems the split-K counters and FP32 partial tiles) in one file-scope
// device array, kNoAllocScratchBytes large, that exists on every GPU which
// loads this library until the process exits.  The caller still passes A, B
// and C.  No cudaMalloc, cudaFree or allocating library routine is called on
// this path.
//
// The array's name is, in host code, only a host-side stand-in for the
// device symbol; a kernel handed that name would fault, or on systems where
// the GPU can reach host memory silently use the wrong memory.  So the first
// call on each device, with that device current, looks up the array's device
// address with cudaGetSymbolAddress (checking the result) and caches it; every
// later call on that device reuses it.  Make that first call before any stream
// capture begins.
//
// Every call shares the one array and leaves its contents behind for the next
// call.  Nothing in it needs to start at zero except the split-K counters,
// which each call clears itself (an asynchronous memset on the call's stream)
// before its GEMM kernel; the slice pre-pass rewrites every slice byte the
// GEMM reads (padding included), and every partial tile is written before it
// is read.  Calls whose work overlaps on the GPU (different streams, or host
// threads that do not order their calls) race on the array: serialise them,
// e.g. on one stream.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <mutex>

#include "internal.h"
#include "split.h"

namespace moa {
int gemm_ex(int64_t m, int64_t n, int64_t p, moa_dtype dt, const void* A, const void* B, void* C,
            int slices, void* ws, size_t ws_bytes, cudaStream_t s, moa_stats* st);
int validate_gemm_args(int64_t m, int64_t n, int64_t p, int dt, const void* A, const void* B,
                       const void* C);

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;   // 32 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_dev[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (set up once).
int scratch_address(void** out) {
    int d = 0;
    cudaError_t e = cudaGetDevice(&d);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (d < 0 || d >= kMaxDevices) return fail(MOA_ERR_CUDA, "device index out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_dev[d]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr)
            return cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol,
                             "cudaGetSymbolAddress(no-alloc scratch)");
        g_scratch_dev[d] = p;
    }
    *out = g_scratch_dev[d];
    return MOA_OK;
}

// need == SIZE_MAX: a count not formed (known only to exceed the array).
int too_big(int64_t m, int64_t n, int64_t p, size_t need) {
    char buf[240];
    char nb[32];
    if (need == SIZE_MAX)
        std::snprintf(nb, sizeof nb, "more than %zu", kNoAllocScratchBytes);
    else
        std::snprintf(nb, sizeof nb, "%zu", need);
    std::snprintf(buf, sizeof buf,
                  "problem %lldx%lldx%lld needs %s bytes of scratch; the static no-alloc "
                  "scratch holds %zu bytes (use moa_gemm_ex with a workspace instead)",
                  static_cast<long long>(m), static_cast<long long>(n), static_cast<long long>(p),
                  nb, kNoAllocScratchBytes);
    return fail(MOA_ERR_WORKSPACE, buf);
}

}  // namespace
}  // namespace moa

extern "C" {

int moa_gemm_f32split_noalloc(int64_t m, int64_t n, int64_t p, const float* A, const float* B,
                              float* C, void* stream) {
    // The checks of moa_gemm_ex first: every dimension is then at most 2^31,
    // so the size products below cannot wrap.
    int rc = moa::validate_gemm_args(m, n, p, MOA_F32_SPLIT, A, B, C);
    if (rc != MOA_OK) return rc;
    // The slice planes alone (three BF16 planes of A and of B at 16-byte row
    // pitches) must fit before the full layout is sized.
    // Each element count is below 2^63 here; the sum is compared with the
    // limit / 6 so that the byte count is only formed once it is small.
    const size_t ea = static_cast<size_t>(m) * static_cast<size_t>(moa::round_up(n, 8));
    const size_t eb = static_cast<size_t>(n) * static_cast<size_t>(moa::round_up(p, 8));
    const size_t lim = moa::kNoAllocScratchBytes / 6;
    if (ea > lim || eb > lim || ea + eb > lim)
        return moa::too_big(m, n, p, (ea > lim || eb > lim) ? SIZE_MAX : 6 * (ea + eb));
    const size_t need = moa::split_workspace_bytes(m, n, p, MOA_F32_SPLIT, 0);
    if (need > moa::kNoAllocScratchBytes) return moa::too_big(m, n, p, need);
    if (m == 0 || p == 0) return MOA_OK;
    void* ws = nullptr;
    if (need > 0) {
        rc = moa::scratch_address(&ws);
        if (rc != MOA_OK) return rc;
    }
    return moa::gemm_ex(m, n, p, MOA_F32_SPLIT, A, B, C, 0, ws, moa::kNoAllocScratchBytes,
                        static_cast<cudaStream_t>(stream), nullptr);
}

}  // extern "C"
