// products.cu -- the other two products of the MoA inner/outer-product
// family (the paper's Appendix: one algorithm covers the matrix, Hadamard and
// Kronecker products).  With the outer product T[i,j,k,l] = A[i,j] * B[k,l]:
//   Kronecker  C[(i*p)+k, (j*q)+l] := T[i,j,k,l]            (no reduction)
//   Hadamard   C[i, j]             := T[i,j,i,j]            (diagonal, m=p, n=q)
//   matrix     C[i, l]             := sum_j T[i,j,j,l]      (Eq. eq:dnf; the GEMM kernels)
// Every output element is one product, rounded once.  Both kernels are HBM
// bound: 16-byte stores (and loads for Hadamard) where the row pitch allows.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "internal.h"

namespace moa {
namespace {

template <typename TI, typename TO>
__device__ __forceinline__ TO prod(TI a, TI b) {
    return static_cast<TO>(a) * static_cast<TO>(b);
}
template <>
__device__ __forceinline__ float prod<__nv_bfloat16, float>(__nv_bfloat16 a, __nv_bfloat16 b) {
    return __bfloat162float(a) * __bfloat162float(b);   // exact: 8-bit x 8-bit significands
}

// One block row of C per blockIdx.y (r = i*p + k); threads sweep the nq
// columns of that row, four consecutive outputs each.
template <typename TI, typename TO>
__global__ void kronecker_kernel(const TI* __restrict__ A, const TI* __restrict__ B,
                                 TO* __restrict__ C, int64_t m, int64_t n, int64_t p, int64_t q,
                                 int vec) {
    const int64_t r = blockIdx.y + static_cast<int64_t>(blockIdx.z) * gridDim.y;
    if (r >= m * p) return;
    const int64_t i = r / p, k = r - i * p;
    const int64_t ncols = n * q;
    const TI* arow = A + i * n;
    const TI* brow = B + k * q;
    TO* crow = C + r * ncols;
    for (int64_t c0 = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) * 4;
         c0 < ncols; c0 += static_cast<int64_t>(gridDim.x) * blockDim.x * 4) {
        TO v[4];
        int64_t j = c0 / q, l = c0 - j * q;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            v[e] = (c0 + e < ncols) ? prod<TI, TO>(arow[j], brow[l]) : TO(0);
            if (++l == q) {
                l = 0;
                ++j;
            }
        }
        if (vec && c0 + 3 < ncols) {
            if constexpr (sizeof(TO) == 4) {
                *reinterpret_cast<float4*>(crow + c0) = make_float4(v[0], v[1], v[2], v[3]);
            } else {
                reinterpret_cast<double2*>(crow + c0)[0] = make_double2(v[0], v[1]);
                reinterpret_cast<double2*>(crow + c0)[1] = make_double2(v[2], v[3]);
            }
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (c0 + e < ncols) crow[c0 + e] = v[e];
        }
    }
}

template <typename TI, typename TO>
__global__ void hadamard_kernel(const TI* __restrict__ A, const TI* __restrict__ B,
                                TO* __restrict__ C, int64_t total) {
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x)
        C[e] = prod<TI, TO>(A[e], B[e]);
}

int elem_sizes(moa_dtype dt, int* in, int* out) {
    switch (dt) {
        case MOA_F64: *in = 8; *out = 8; return MOA_OK;
        case MOA_F32_SIMT:
        case MOA_F32_TF32: *in = 4; *out = 4; return MOA_OK;
        case MOA_BF16: *in = 2; *out = 4; return MOA_OK;
        default: return fail(MOA_ERR_DTYPE, "products take MOA_F64, FP32 (MOA_F32_*) or MOA_BF16");
    }
}

}  // namespace
}  // namespace moa

extern "C" {

int moa_kronecker(int64_t m, int64_t n, int64_t p, int64_t q, moa_dtype dt, const void* A,
                  const void* B, void* C, void* stream) {
    moa::TraceRange tr("moa_kronecker");
    int ie, oe;
    int rc = moa::elem_sizes(dt, &ie, &oe);
    if (rc != MOA_OK) return rc;
    if (m < 0 || n < 0 || p < 0 || q < 0) return moa::fail(MOA_ERR_ARG, "negative dimension");
    const int64_t rows = m * p, cols = n * q;
    if (rows == 0 || cols == 0) return MOA_OK;
    if (!A || !B || !C) return moa::fail(MOA_ERR_ARG, "NULL operand");
    if (reinterpret_cast<uintptr_t>(A) % ie || reinterpret_cast<uintptr_t>(B) % ie ||
        reinterpret_cast<uintptr_t>(C) % oe)
        return moa::fail(MOA_ERR_ALIGN, "pointer not aligned to its element size");
    const int vec = (cols % 4 == 0) && (reinterpret_cast<uintptr_t>(C) % 16 == 0);
    const int threads = 256;
    const int64_t gx = moa::ceil_div(moa::ceil_div(cols, 4), threads);
    dim3 grid(static_cast<unsigned>(gx < 64 ? gx : 64), static_cast<unsigned>(rows < 65535 ? rows : 65535),
              static_cast<unsigned>(moa::ceil_div(rows, 65535)));
    if (grid.z > 65535) return moa::fail(MOA_ERR_ARG, "Kronecker product too tall");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dt == MOA_F64)
        moa::kronecker_kernel<double, double><<<grid, threads, 0, s>>>(
            static_cast<const double*>(A), static_cast<const double*>(B), static_cast<double*>(C), m,
            n, p, q, vec);
    else if (dt == MOA_BF16)
        moa::kronecker_kernel<__nv_bfloat16, float><<<grid, threads, 0, s>>>(
            static_cast<const __nv_bfloat16*>(A), static_cast<const __nv_bfloat16*>(B),
            static_cast<float*>(C), m, n, p, q, vec);
    else
        moa::kronecker_kernel<float, float><<<grid, threads, 0, s>>>(
            static_cast<const float*>(A), static_cast<const float*>(B), static_cast<float*>(C), m, n,
            p, q, vec);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return moa::cuda_fail(e, "kronecker_kernel launch");
    return MOA_OK;
}

int moa_hadamard(int64_t m, int64_t n, moa_dtype dt, const void* A, const void* B, void* C,
                 void* stream) {
    moa::TraceRange tr("moa_hadamard");
    int ie, oe;
    int rc = moa::elem_sizes(dt, &ie, &oe);
    if (rc != MOA_OK) return rc;
    if (m < 0 || n < 0) return moa::fail(MOA_ERR_ARG, "negative dimension");
    const int64_t total = m * n;
    if (total == 0) return MOA_OK;
    if (!A || !B || !C) return moa::fail(MOA_ERR_ARG, "NULL operand");
    if (reinterpret_cast<uintptr_t>(A) % ie || reinterpret_cast<uintptr_t>(B) % ie ||
        reinterpret_cast<uintptr_t>(C) % oe)
        return moa::fail(MOA_ERR_ALIGN, "pointer not aligned to its element size");
    const int threads = 256;
    const int64_t want = moa::ceil_div(total, threads);
    const int blocks = static_cast<int>(want < 32L * moa::num_sms() ? want : 32L * moa::num_sms());
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dt == MOA_F64)
        moa::hadamard_kernel<double, double><<<blocks, threads, 0, s>>>(
            static_cast<const double*>(A), static_cast<const double*>(B), static_cast<double*>(C),
            total);
    else if (dt == MOA_BF16)
        moa::hadamard_kernel<__nv_bfloat16, float><<<blocks, threads, 0, s>>>(
            static_cast<const __nv_bfloat16*>(A), static_cast<const __nv_bfloat16*>(B),
            static_cast<float*>(C), total);
    else
        moa::hadamard_kernel<float, float><<<blocks, threads, 0, s>>>(
            static_cast<const float*>(A), static_cast<const float*>(B), static_cast<float*>(C), total);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return moa::cuda_fail(e, "hadamard_kernel launch");
    return MOA_OK;
}

}  // extern "C"
