// noalloc.cu -- moa_gemm_f32split_noalloc: the FP32-accuracy split GEMM for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside a CUDA-graph
// capture region that must not allocate, real-time or safety-certified hosts
// whose memory is fixed at start-up, plugins living inside another runtime's
// memory pool, or embedded deployments with a static memory plan.  For them
// this entry point keeps its scratch (the three BF16 slice planes of A and of
// B) in one file-scope device array, kNoAllocScratchBytes large, that exists
// on every GPU which loads this library until the process exits.  The caller
// still passes A, B and C.  No cudaMalloc, cudaFree or allocating library
// routine is called on this path.
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
// call; the split pre-pass rewrites every byte the GEMM reads (padding
// included), so nothing has to start at zero.  Calls whose work overlaps on
// the GPU (different streams, or host threads that do not order their calls)
// race on the array: serialise them, e.g. on one stream.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "internal.h"
#include "split.h"

namespace moa {
int gemm_ex(int64_t m, int64_t n, int64_t p, moa_dtype dt, const void* A, const void* B, void* C,
            int slices, void* ws, size_t ws_bytes, cudaStream_t s, moa_stats* st);

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

}  // namespace
}  // namespace moa

extern "C" {

int moa_gemm_f32split_noalloc(int64_t m, int64_t n, int64_t p, const float* A, const float* B,
                              float* C, void* stream) {
    if (m < 0 || n < 0 || p < 0) return moa::fail(MOA_ERR_ARG, "negative dimension");
    const size_t need = moa::split_workspace_bytes(m, n, p, MOA_F32_SPLIT, 0);
    if (need > moa::kNoAllocScratchBytes) {
        char buf[200];
        std::snprintf(buf, sizeof buf,
                      "problem %lldx%lldx%lld needs %zu bytes of scratch; the static no-alloc "
                      "scratch holds %zu bytes (use moa_gemm_ex with a workspace instead)",
                      static_cast<long long>(m), static_cast<long long>(n),
                      static_cast<long long>(p), need, moa::kNoAllocScratchBytes);
        return moa::fail(MOA_ERR_WORKSPACE, buf);
    }
    if (m == 0 || p == 0) return MOA_OK;
    void* ws = nullptr;
    if (need > 0) {
        const int rc = moa::scratch_address(&ws);
        if (rc != MOA_OK) return rc;
    }
    return moa::gemm_ex(m, n, p, MOA_F32_SPLIT, A, B, C, 0, ws, moa::kNoAllocScratchBytes,
                        static_cast<cudaStream_t>(stream), nullptr);
}

}  // extern "C"
