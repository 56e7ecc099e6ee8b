// gemm_simt.cu -- the ONF GEMM on the CUDA cores (no tensor cores):
// native FP64 (DFMA) for MOA_F64 and plain FP32 (FFMA) for MOA_F32_SIMT.
//
// C[(i*p)+j] := sum_k A[(i*n)+k] * B[(k*p)+j]   (Eq. (eq:dnf), Sec. 2)
//
// Blocking follows Sec. 3.1-3.4: each CTA owns a BM x BN block of C (the
// block-block product of Fig. fig:omega), the k loop is cut into BK-deep
// slabs staged in shared memory (A slab stored k-major so that a column of A
// is a contiguous broadcast, B slab kept as contiguous row pieces, the "row
// of B" of Fig. fig:mm), and each thread accumulates a TM x TN register block
// in k order.  Every per-element sum runs k = 0..n-1 in order.
#include <cuda_runtime.h>

#include "internal.h"

namespace moa {
namespace {

template <typename T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    simt_gemm_kernel(const T* __restrict__ A, const T* __restrict__ B, T* __restrict__ C,
                     int64_t m, int64_t n, int64_t p) {
    constexpr int NT = (BM / TM) * (BN / TN);
    __shared__ T As[2][BK][BM];
    __shared__ T Bs[2][BK][BN];

    const int tid = threadIdx.x;
    const int tx = tid % (BN / TN);
    const int ty = tid / (BN / TN);
    const int64_t row0 = static_cast<int64_t>(blockIdx.y) * BM;
    const int64_t col0 = static_cast<int64_t>(blockIdx.x) * BN;

    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

    auto load = [&](int buf, int64_t k0) {
#pragma unroll
        for (int e = tid; e < BM * BK; e += NT) {
            const int r = e / BK, c = e % BK;
            const int64_t gi = row0 + r, gk = k0 + c;
            As[buf][c][r] = (gi < m && gk < n) ? A[gi * n + gk] : T(0);
        }
#pragma unroll
        for (int e = tid; e < BK * BN; e += NT) {
            const int r = e / BN, c = e % BN;
            const int64_t gk = k0 + r, gj = col0 + c;
            Bs[buf][r][c] = (gk < n && gj < p) ? B[gk * p + gj] : T(0);
        }
    };

    const int64_t nk = (n + BK - 1) / BK;
    if (nk > 0) load(0, 0);
    __syncthreads();
    for (int64_t kb = 0; kb < nk; ++kb) {
        const int buf = static_cast<int>(kb & 1);
        if (kb + 1 < nk) load(buf ^ 1, (kb + 1) * BK);
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            T a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = As[buf][k][ty * TM + i];
#pragma unroll
            for (int j = 0; j < TN; ++j) b[j] = Bs[buf][k][tx * TN + j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int64_t gi = row0 + ty * TM + i;
        if (gi >= m) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int64_t gj = col0 + tx * TN + j;
            if (gj < p) C[gi * p + gj] = acc[i][j];
        }
    }
}

template <typename T, int BM, int BN, int BK, int TM, int TN>
int launch_simt(int64_t m, int64_t n, int64_t p, const T* A, const T* B, T* C, cudaStream_t s) {
    const int64_t gx = ceil_div(p, BN), gy = ceil_div(m, BM);
    if (gy > 65535) return fail(MOA_ERR_ARG, "m too large for the SIMT grid");
    dim3 grid(static_cast<unsigned>(gx), static_cast<unsigned>(gy));
    prof_begin(s);
    simt_gemm_kernel<T, BM, BN, BK, TM, TN><<<grid, (BM / TM) * (BN / TN), 0, s>>>(A, B, C, m, n, p);
    cudaError_t e = cudaGetLastError();
    prof_end(s);
    if (e != cudaSuccess) return cuda_fail(e, "simt_gemm_kernel launch");
    return MOA_OK;
}

}  // namespace

int simt_f64_launch(int64_t m, int64_t n, int64_t p, const double* A, const double* B, double* C,
                    cudaStream_t s) {
    return launch_simt<double, 64, 64, 16, 4, 4>(m, n, p, A, B, C, s);
}

int simt_f32_launch(int64_t m, int64_t n, int64_t p, const float* A, const float* B, float* C,
                    cudaStream_t s) {
    return launch_simt<float, 128, 128, 8, 8, 8>(m, n, p, A, B, C, s);
}

}  // namespace moa
