// runtime.cu -- host runtime shared by every entry point: error reporting,
// the per-device status word, device properties, TMA descriptor encoding
// (driver entry point fetched at run time, so no link against libcuda), and
// the padding copy used when a row pitch is not a multiple of 16 bytes.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <nvtx3/nvToolsExt.h>

#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>

#include "internal.h"
#include "ptx.cuh"

namespace moa {

namespace {
thread_local std::string g_last_error;
std::mutex g_mu;
uint64_t g_wait_limit_ns = 0;
constexpr int kMaxDevices = 64;
int* g_status[kMaxDevices] = {nullptr};
int g_sms[kMaxDevices] = {0};
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
thread_local cudaEvent_t g_prof_start = nullptr;
thread_local int* t_status_override = nullptr;
thread_local cudaEvent_t g_prof_stop = nullptr;

int current_device() {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess) return -1;
    return d;
}
}  // namespace

// Per-device status word: a file-scope device variable; host code only ever
// uses the address cudaGetSymbolAddress gives for the current device.
__device__ int g_moa_device_status;

void set_error(const std::string& msg) { g_last_error = msg; }

void prof_begin(cudaStream_t s) {
    if (g_prof_start) cudaEventRecord(g_prof_start, s);
}
void prof_end(cudaStream_t s) {
    if (g_prof_stop) cudaEventRecord(g_prof_stop, s);
}

int fail(int status, const std::string& msg) {
    g_last_error = msg;
    log_msg(1, "error %d: %s", status, msg.c_str());
    return status;
}

int cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    log_msg(1, "error %d: %s", MOA_ERR_CUDA, g_last_error.c_str());
    return MOA_ERR_CUDA;
}

int log_level() {
    static const int level = [] {
        const char* e = std::getenv("MOA_LOG");
        const long v = e ? std::strtol(e, nullptr, 10) : 0;
        return static_cast<int>(v < 0 ? 0 : (v > 3 ? 3 : v));
    }();
    return level;
}

void log_msg(int level, const char* fmt, ...) {
    if (level > log_level()) return;
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    std::fprintf(stderr, "[moa] %s\n", buf);
}

namespace {
constexpr unsigned char kCanaryByte = 0xA5;
__global__ void canary_check_kernel(const unsigned char* guard, int n, int* status) {
    bool bad = false;
    for (int i = threadIdx.x; i < n; i += blockDim.x) bad |= guard[i] != kCanaryByte;
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicCAS(status, kDevOk, kDevCanary);
}
}  // namespace

bool canary_enabled() {
    static const bool on = [] {
        const char* e = std::getenv("MOA_DEBUG_CANARY");
        return e && std::strtol(e, nullptr, 10) != 0;
    }();
    return on;
}

int canary_arm(void* guard, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(guard, kCanaryByte, kCanaryBytes, s);
    return e == cudaSuccess ? MOA_OK : cuda_fail(e, "cudaMemsetAsync(canary)");
}

int canary_check(const void* guard, cudaStream_t s) {
    int* status = launch_status_ptr();
    if (!status) return MOA_ERR_CUDA;
    canary_check_kernel<<<1, 64, 0, s>>>(static_cast<const unsigned char*>(guard),
                                          static_cast<int>(kCanaryBytes), status);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MOA_OK : cuda_fail(e, "canary_check_kernel launch");
}

void trace_push(const char* name) { nvtxRangePushA(name); }
void trace_pop() { nvtxRangePop(); }

int* device_status_ptr() {
    const int d = current_device();
    if (d < 0 || d >= kMaxDevices) {
        set_error("no current CUDA device");
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_status[d]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_moa_device_status);
        if (e != cudaSuccess) {
            cuda_fail(e, "cudaGetSymbolAddress(status)");
            return nullptr;
        }
        g_status[d] = static_cast<int*>(p);
    }
    return g_status[d];
}

int* launch_status_ptr() {
    return t_status_override ? t_status_override : device_status_ptr();
}

void set_status_override(int* p) { t_status_override = p; }

int num_sms() {
    const int d = current_device();
    if (d < 0 || d >= kMaxDevices) return 1;
    if (g_sms[d] == 0) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d);
        g_sms[d] = v > 0 ? v : 1;
    }
    return g_sms[d];
}

int smem_attr_once(const void* func, int bytes, std::atomic<uint64_t>& done, const char* what) {
    const int d = current_device();
    const uint64_t bit = (d >= 0 && d < 64) ? (1ull << d) : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return MOA_OK;
    cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return cuda_fail(e, what);
    if (bit) done.fetch_or(bit, std::memory_order_acq_rel);
    return MOA_OK;
}

uint64_t wait_limit_ns() {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_wait_limit_ns == 0) {
        const char* env = std::getenv("MOA_WAIT_LIMIT_NS");
        g_wait_limit_ns = env ? std::strtoull(env, nullptr, 10) : 0;
        if (g_wait_limit_ns == 0) g_wait_limit_ns = 2000000000ull;
    }
    return g_wait_limit_ns;
}

static int get_encode() {
    if (g_encode) return MOA_OK;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
        return fail(MOA_ERR_CUDA, "cuTensorMapEncodeTiled entry point unavailable");
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    return MOA_OK;
}

int make_tmap_2d(CUtensorMap* map, CUtensorMapDataType dt, const void* base, uint64_t inner,
                 uint64_t outer, uint64_t pitch_bytes, uint32_t box_inner, uint32_t box_outer) {
    int rc = get_encode();
    if (rc != MOA_OK) return rc;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {pitch_bytes};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        char buf[256];
        std::snprintf(buf, sizeof buf,
                      "cuTensorMapEncodeTiled(2d) failed (%d): inner=%llu outer=%llu pitch=%llu "
                      "box=%ux%u",
                      static_cast<int>(r), static_cast<unsigned long long>(inner),
                      static_cast<unsigned long long>(outer),
                      static_cast<unsigned long long>(pitch_bytes), box_inner, box_outer);
        return fail(MOA_ERR_CUDA, buf);
    }
    return MOA_OK;
}

int make_tmap_3d(CUtensorMap* map, CUtensorMapDataType dt, const void* base, uint64_t inner,
                 uint64_t outer, uint64_t depth, uint64_t pitch_bytes, uint64_t plane_bytes,
                 uint32_t box_inner, uint32_t box_outer, int swizzle_bytes) {
    int rc = get_encode();
    if (rc != MOA_OK) return rc;
    cuuint64_t dims[3] = {inner, outer, depth};
    cuuint64_t strides[2] = {pitch_bytes, plane_bytes};
    cuuint32_t box[3] = {box_inner, box_outer, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = g_encode(map, dt, 3, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE,
                          swizzle_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        char buf[256];
        std::snprintf(buf, sizeof buf, "cuTensorMapEncodeTiled(3d) failed (%d)", static_cast<int>(r));
        return fail(MOA_ERR_CUDA, buf);
    }
    return MOA_OK;
}

// ------------------------------------------------------------------ padding copy
namespace {
template <typename T>
__global__ void pad_copy_kernel(const T* __restrict__ src, T* __restrict__ dst, int64_t rows,
                                int64_t cols, int64_t ld) {
    const int64_t total = rows * ld;
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t r = e / ld, c = e % ld;
        dst[e] = c < cols ? src[r * cols + c] : T(0);
    }
}
}  // namespace

int pad_copy_launch(const void* src, void* dst, int64_t rows, int64_t cols, int64_t ld, int esize,
                    cudaStream_t s) {
    const int64_t total = rows * ld;
    if (total == 0) return MOA_OK;
    const int threads = 256;
    const int64_t want = ceil_div(total, threads);
    const int blocks = static_cast<int>(want < 8L * num_sms() ? want : 8L * num_sms());
    switch (esize) {
        case 2:
            pad_copy_kernel<uint16_t><<<blocks, threads, 0, s>>>(
                static_cast<const uint16_t*>(src), static_cast<uint16_t*>(dst), rows, cols, ld);
            break;
        case 4:
            pad_copy_kernel<uint32_t><<<blocks, threads, 0, s>>>(
                static_cast<const uint32_t*>(src), static_cast<uint32_t*>(dst), rows, cols, ld);
            break;
        case 8:
            pad_copy_kernel<uint64_t><<<blocks, threads, 0, s>>>(
                static_cast<const uint64_t*>(src), static_cast<uint64_t*>(dst), rows, cols, ld);
            break;
        default:
            return fail(MOA_ERR_ARG, "pad_copy: bad element size");
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "pad_copy_kernel launch");
    return MOA_OK;
}

// ------------------------------------------------------------------ transpose
namespace {
// 64 x 64 tiles through shared memory, 256 threads.  Reads rows of X and
// writes rows of Xt, 16 bytes per access when both pitches allow it.
template <bool VEC>
__global__ void __launch_bounds__(256)
    transpose_pad_kernel(const float* __restrict__ X, int64_t rows, int64_t cols,
                         float* __restrict__ Xt, int64_t ld) {
    __shared__ float tile[64][65];
    const int64_t c0 = static_cast<int64_t>(blockIdx.x) * 64;   // column block of X
    const int64_t r0 = static_cast<int64_t>(blockIdx.y) * 64;   // row block of X (< ld)
    const int t = threadIdx.x;
    if (VEC) {
        // 64 rows x 16 float4: thread t loads rows (t / 16) + 16 q, float4 (t % 16)
        const int cv = (t & 15) * 4;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int rr = (t >> 4) + 16 * q;
            const int64_t r = r0 + rr, c = c0 + cv;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (r < rows && c + 3 < cols) {
                v = *reinterpret_cast<const float4*>(X + r * cols + c);
            } else if (r < rows) {
                if (c < cols) v.x = X[r * cols + c];
                if (c + 1 < cols) v.y = X[r * cols + c + 1];
                if (c + 2 < cols) v.z = X[r * cols + c + 2];
            }
            tile[rr][cv] = v.x;
            tile[rr][cv + 1] = v.y;
            tile[rr][cv + 2] = v.z;
            tile[rr][cv + 3] = v.w;
        }
        __syncthreads();
        // Xt rows c0 .. c0+63, each 64 values r0 .. r0+63 as 16 float4
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int cc = (t >> 4) + 16 * q;
            const int rv = (t & 15) * 4;
            const int64_t c = c0 + cc, r = r0 + rv;
            if (c >= cols || r >= ld) continue;
            const float4 v = make_float4(tile[rv][cc], tile[rv + 1][cc], tile[rv + 2][cc],
                                         tile[rv + 3][cc]);
            *reinterpret_cast<float4*>(Xt + c * ld + r) = v;   // ld % 4 == 0, r % 4 == 0
        }
    } else {
        for (int e = t; e < 64 * 64; e += 256) {
            const int rr = e >> 6, cc = e & 63;
            const int64_t r = r0 + rr, c = c0 + cc;
            tile[rr][cc] = (r < rows && c < cols) ? X[r * cols + c] : 0.f;
        }
        __syncthreads();
        for (int e = t; e < 64 * 64; e += 256) {
            const int cc = e >> 6, rr = e & 63;
            const int64_t c = c0 + cc, r = r0 + rr;
            if (c < cols && r < ld) Xt[c * ld + r] = tile[rr][cc];
        }
    }
}
}  // namespace

int transpose_pad_launch(const float* X, int64_t rows, int64_t cols, float* Xt, int64_t ld,
                         cudaStream_t s) {
    const int64_t gx = ceil_div(cols, 64), gy = ceil_div(ld, 64);
    if (gy > 65535) return fail(MOA_ERR_ARG, "transpose: too many rows");
    dim3 grid(static_cast<unsigned>(gx), static_cast<unsigned>(gy));
    const bool vec = (cols % 4 == 0) && (ld % 4 == 0) && (reinterpret_cast<uintptr_t>(X) % 16 == 0) &&
                     (reinterpret_cast<uintptr_t>(Xt) % 16 == 0);
    if (vec)
        transpose_pad_kernel<true><<<grid, 256, 0, s>>>(X, rows, cols, Xt, ld);
    else
        transpose_pad_kernel<false><<<grid, 256, 0, s>>>(X, rows, cols, Xt, ld);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "transpose_pad_kernel launch");
    return MOA_OK;
}

// ------------------------------------------------------------------ self-test
namespace {
// One CTA waits, through the same bounded mbar_wait every pipeline uses, on
// an mbarrier that nothing ever arrives at; after `limit_ns` the wait gives
// up, records kDevTimeout in the status word and the kernel returns.  Holds
// no TMEM and issues no asynchronous copies.
__global__ void wait_timeout_selftest_kernel(uint64_t limit_ns, int* status) {
    __shared__ uint64_t bar;
    __shared__ CtaCtl ctl;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        ctl.abort = 0;
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_wait(&bar, 0, &ctl, limit_ns, status);
    __syncthreads();
}
}  // namespace

}  // namespace moa

// ------------------------------------------------------------------ public housekeeping
extern "C" {

const char* moa_last_error(void) { return moa::g_last_error.c_str(); }

uint64_t moa_set_wait_limit_ns(uint64_t ns) {
    const uint64_t prev = moa::wait_limit_ns();
    std::lock_guard<std::mutex> lk(moa::g_mu);
    moa::g_wait_limit_ns = ns ? ns : 2000000000ull;
    return prev;
}

const char* moa_version(void) { return "moa-b300 0.1.0 (sm_103a)"; }

int moa_selftest_wait_timeout(uint64_t limit_ns, void* stream) {
    if (limit_ns == 0 || limit_ns > 10000000000ull)
        return moa::fail(MOA_ERR_ARG, "limit must be in (0, 10 s]");
    int* status = moa::device_status_ptr();
    if (!status) return MOA_ERR_CUDA;
    moa::wait_timeout_selftest_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(limit_ns,
                                                                                      status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return moa::cuda_fail(e, "wait_timeout_selftest_kernel launch");
    return MOA_OK;
}

int moa_profile_events(void* start_event, void* stop_event) {
    moa::g_prof_start = static_cast<cudaEvent_t>(start_event);
    moa::g_prof_stop = static_cast<cudaEvent_t>(stop_event);
    return MOA_OK;
}

int moa_sync_status(void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return moa::cuda_fail(e, "cudaStreamSynchronize");
    int* dev = moa::device_status_ptr();
    if (!dev) return MOA_ERR_CUDA;
    int v = 0;
    e = cudaMemcpy(&v, dev, sizeof v, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return moa::cuda_fail(e, "read status word");
    if (v != moa::kDevOk) {
        const int zero = 0;
        cudaMemcpy(dev, &zero, sizeof zero, cudaMemcpyHostToDevice);
        if (v == moa::kDevTimeout)
            return moa::fail(MOA_ERR_TIMEOUT, "a device pipeline wait exceeded its time limit");
        if (v == moa::kDevNonFinite)
            return moa::fail(MOA_ERR_NONFINITE, "split pre-pass found a NaN or Inf input");
        if (v == moa::kDevCanary)
            return moa::fail(MOA_ERR_CUDA, "workspace guard bytes past the used workspace were "
                                           "overwritten (MOA_DEBUG_CANARY)");
        return moa::fail(MOA_ERR_CUDA, "unknown device status");
    }
    return MOA_OK;
}

}  // extern "C"
