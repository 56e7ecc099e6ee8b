// peaks.cu -- measured FP64 arithmetic rates of the device (diagnostic).
//
// The native FP64 mode (MOA_F64) is bound by the FP64 pipe, so its roofline
// denominator is this device's own FP64 rate, measured here rather than taken
// from a datasheet: one launch of independent FMA chains on the CUDA cores
// (DFMA), and one of independent warp-level FP64 MMAs (mma.sync m16n8k4,
// the FP64 tensor path), each timed with CUDA events.  Each thread (warp)
// keeps enough independent chains in flight that the latency of one
// operation does not bound the rate.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace moa {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSm = 4;

// Keeps the results live (no allocation: a static device array).
__device__ double g_peak_sink[kPeakThreads];

// kFmaChains independent chains a thread (enough to cover the FMA latency),
// 2 flops per FMA.
constexpr int kFmaChains = 16;
constexpr int kMmaChains = 8;
__global__ void __launch_bounds__(kPeakThreads)
    fp64_fma_rate_kernel(double x, double y, int iters) {
    // every operand in a register, accumulator form (as in a GEMM's inner
    // product): a_i := u_(i%4) * v + a_i
    double a[kFmaChains], u[4];
#pragma unroll
    for (int i = 0; i < kFmaChains; ++i) a[i] = x + 0.001 * (threadIdx.x + i);
#pragma unroll
    for (int i = 0; i < 4; ++i) u[i] = y * (1.0 + 0.25 * i) + 1e-12 * threadIdx.x;
    const double v = x - 1e-12 * threadIdx.x;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
#pragma unroll
            for (int i = 0; i < kFmaChains; ++i) a[i] = fma(u[i & 3], v, a[i]);
        }
    }
    double s = 0;
#pragma unroll
    for (int i = 0; i < kFmaChains; ++i) s += a[i];
    if (s == 12345.678) g_peak_sink[threadIdx.x] = s;   // never true for the inputs used
}

// kMmaChains independent m16n8k4 FP64 MMAs a warp per step: 16 x 8 x 4 x 2
// flops each.
__global__ void __launch_bounds__(kPeakThreads)
    fp64_mma_rate_kernel(double x, int iters) {
    double acc[kMmaChains][4];
#pragma unroll
    for (int j = 0; j < kMmaChains; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[j][i] = 0.0;
    const double a0 = x + 0.001 * threadIdx.x, a1 = x - 0.001 * threadIdx.x, b0 = x * 0.5;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
#pragma unroll
            for (int j = 0; j < kMmaChains; ++j)
                asm volatile(
                    "mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 "
                    "{%0, %1, %2, %3}, {%4, %5}, {%6}, {%0, %1, %2, %3};"
                    : "+d"(acc[j][0]), "+d"(acc[j][1]), "+d"(acc[j][2]), "+d"(acc[j][3])
                    : "d"(a0), "d"(a1), "d"(b0));
        }
    }
    double s = 0;
#pragma unroll
    for (int j = 0; j < kMmaChains; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) s += acc[j][i];
    if (s == 12345.678) g_peak_sink[threadIdx.x] = s;
}

}  // namespace
}  // namespace moa

extern "C" {

int moa_measure_fp64_rate(int kind, void* stream, double* tflops) {
    if ((kind != 0 && kind != 1) || tflops == nullptr)
        return moa::fail(MOA_ERR_ARG, "kind must be 0 (FMA) or 1 (MMA); tflops must not be NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int blocks = moa::num_sms() * moa::kPeakBlocksPerSm;
    const double threads = static_cast<double>(blocks) * moa::kPeakThreads;
    // work per outer iteration of the whole grid
    const double per_iter =
        kind == 0 ? threads * 8 * moa::kFmaChains * 2
                  : threads / 32 * 8 * moa::kMmaChains * (16.0 * 8 * 4 * 2);
    auto launch = [&](int iters) {
        if (kind == 0)
            moa::fp64_fma_rate_kernel<<<blocks, moa::kPeakThreads, 0, s>>>(1.0000001, 1e-9, iters);
        else
            moa::fp64_mma_rate_kernel<<<blocks, moa::kPeakThreads, 0, s>>>(1.0000001, iters);
        return cudaGetLastError();
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return moa::fail(MOA_ERR_CUDA, "cudaEventCreate");
    }
    int rc = MOA_OK;
    // a short warm-up launch, then five launches of about 1.5e10 flops (a
    // kernel's length, not a sustained run: long FP64 runs lower the clock
    // under the power limit); the best of them
    const int iters = static_cast<int>(1.5e10 / per_iter) + 1;
    cudaError_t e = launch(8);
    double best = 0.0;
    for (int r = 0; r < 5 && e == cudaSuccess; ++r) {
        float ms = 0.f;
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) e = launch(iters);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms > 0.f) best = std::max(best, per_iter * iters / (ms * 1e-3) / 1e12);
    }
    if (e != cudaSuccess)
        rc = moa::cuda_fail(e, "moa_measure_fp64_rate");
    else
        *tflops = best;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

}  // extern "C"
