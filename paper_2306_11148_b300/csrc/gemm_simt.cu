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

// Plain FP32 (FFMA) GEMM with register prefetch: 128 x 128 block of C per
// CTA, 256 threads, 16-deep k slabs.  Thread (tx, ty) owns rows
// {4ty..4ty+3, 64+4ty..64+4ty+3} and columns {4tx..4tx+3, 64+4tx..64+4tx+3}
// of the block, so that each of its shared-memory reads is one 16-byte load
// and a warp's reads of a B row cover 256 contiguous bytes.  The next slab is
// read from global memory into registers while the current one is used.
// Every per-element sum still runs k = 0..n-1 in order.
constexpr int kSBM = 128, kSBN = 128, kSBK = 16;

__device__ __forceinline__ float4 ldg4_or_zero(const float* __restrict__ X, int64_t rows,
                                               int64_t cols, int64_t r, int64_t c0, bool vec) {
    if (r >= rows) return make_float4(0.f, 0.f, 0.f, 0.f);
    const float* src = X + r * cols + c0;
    if (vec && c0 + 4 <= cols) return *reinterpret_cast<const float4*>(src);
    float v[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = (c0 + e < cols) ? src[e] : 0.f;
    return make_float4(v[0], v[1], v[2], v[3]);
}

__global__ void __launch_bounds__(256, 2)
    sgemm_kernel(const float* __restrict__ A, const float* __restrict__ B, float* __restrict__ C,
                 int64_t m, int64_t n, int64_t p, int vec_a, int vec_b) {
    __shared__ __align__(16) float As[2][kSBK][kSBM];   // k-major: a column of A is contiguous
    __shared__ __align__(16) float Bs[2][kSBK][kSBN];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t row0 = static_cast<int64_t>(blockIdx.y) * kSBM;
    const int64_t col0 = static_cast<int64_t>(blockIdx.x) * kSBN;
    // global -> register mapping: A rows ar, ar + 64 at k offset ak; B rows
    // bk, bk + 8 at column offset bc
    const int ar = tid >> 2, ak = (tid & 3) * 4;
    const int bk = tid >> 5, bc = (tid & 31) * 4;

    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    float4 ra[2], rb[2];
    auto fetch = [&](int64_t k0) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            ra[h] = ldg4_or_zero(A, m, n, row0 + ar + 64 * h, k0 + ak, vec_a != 0);
            rb[h] = ldg4_or_zero(B, n, p, k0 + bk + 8 * h, col0 + bc, vec_b != 0);
        }
    };
    auto stash = [&](int buf) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            As[buf][ak + 0][ar + 64 * h] = ra[h].x;
            As[buf][ak + 1][ar + 64 * h] = ra[h].y;
            As[buf][ak + 2][ar + 64 * h] = ra[h].z;
            As[buf][ak + 3][ar + 64 * h] = ra[h].w;
            *reinterpret_cast<float4*>(&Bs[buf][bk + 8 * h][bc]) = rb[h];
        }
    };

    const int64_t nk = (n + kSBK - 1) / kSBK;
    if (nk > 0) {
        fetch(0);
        stash(0);
    }
    __syncthreads();
    for (int64_t kb = 0; kb < nk; ++kb) {
        const int buf = static_cast<int>(kb & 1);
        if (kb + 1 < nk) fetch((kb + 1) * kSBK);   // in flight during the slab below
#pragma unroll
        for (int k = 0; k < kSBK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][k][4 * ty]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][k][64 + 4 * ty]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][k][4 * tx]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][k][64 + 4 * tx]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if (kb + 1 < nk) stash(buf ^ 1);   // the other buffer was last read before the
        __syncthreads();                   // previous barrier
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t gi = row0 + (i < 4 ? 4 * ty + i : 64 + 4 * ty + (i - 4));
        if (gi >= m) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t gj = col0 + 64 * h + 4 * tx;
            float* dst = C + gi * p + gj;
            if (vec_b && gj + 4 <= p) {
                *reinterpret_cast<float4*>(dst) = make_float4(acc[i][4 * h], acc[i][4 * h + 1],
                                                              acc[i][4 * h + 2], acc[i][4 * h + 3]);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (gj + e < p) dst[e] = acc[i][4 * h + e];
            }
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
    const int64_t gx = ceil_div(p, kSBN), gy = ceil_div(m, kSBM);
    if (gy > 65535) return fail(MOA_ERR_ARG, "m too large for the SIMT grid");
    // 16-byte loads and stores need 16-byte aligned rows
    const int vec_a = (n % 4 == 0) && (reinterpret_cast<uintptr_t>(A) % 16 == 0);
    const int vec_b = (p % 4 == 0) && (reinterpret_cast<uintptr_t>(B) % 16 == 0) &&
                      (reinterpret_cast<uintptr_t>(C) % 16 == 0);
    dim3 grid(static_cast<unsigned>(gx), static_cast<unsigned>(gy));
    prof_begin(s);
    sgemm_kernel<<<grid, 256, 0, s>>>(A, B, C, m, n, p, vec_a, vec_b);
    cudaError_t e = cudaGetLastError();
    prof_end(s);
    if (e != cudaSuccess) return cuda_fail(e, "sgemm_kernel launch");
    return MOA_OK;
}

}  // namespace moa
