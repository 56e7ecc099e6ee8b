// products.cu -- the MoA inner/outer-product family as ONE kernel (the
// paper's Appendix: a single algorithm, "ipophp", covers the Hadamard,
// Kronecker and matrix products).  With the outer product
// T[i,j,k,l] = A[i,j] * B[k,l] (A is m x n, B is p x q):
//   Kronecker  C[(i*p)+k, (j*q)+l] := T[i,j,k,l]            (no reduction)
//   Hadamard   C[i, j]             := T[i,j,i,j]            (diagonal, m=p, n=q)
//   matrix     C[i, l]             := sum_j T[i,j,j,l]      (contraction, n=p; Eq. eq:dnf)
// All three are one index map over the output C (R rows x Q columns):
//   C[r, c] = sum_{s < S} A[r / ra, c / ca + s] * B[r % rb + s, c % cb]
//   Kronecker (ra, ca, rb, cb, S) = (p, q, p, q, 1)
//   Hadamard                      = (1, 1, R, Q, 1)
//   matrix                        = (1, Q, 1, Q, n)
// ipophp_kernel evaluates that map directly: every output element is its own
// sum of S products, each product rounded, then added in s order (no fused
// multiply-add), so with S = 1 an element is one rounded product and with
// S = n the contraction follows Fig. ip.c's order for each element.  The
// Kronecker and Hadamard products are HBM bound: four consecutive outputs per
// thread with 16-byte stores (and 16-byte loads where the map reads A or B
// contiguously).  The contraction through this SIMT kernel is the algebra's
// reference form; the tensor-core GEMMs are its fast specialisation.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "fastdiv.cuh"
#include "internal.h"

namespace moa {
namespace {

template <typename TI, typename TO>
__device__ __forceinline__ TO widen(TI a) {
    return static_cast<TO>(a);
}
template <>
__device__ __forceinline__ float widen<__nv_bfloat16, float>(__nv_bfloat16 a) {
    return __bfloat162float(a);
}
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }

// The index map of one product kind (see the file comment).
struct ProductMap {
    int64_t R, Q;            // output rows, columns
    int64_t ra, ca, rb, cb;  // divisors / moduli of the map
    int64_t S;               // contraction length (1: no reduction)
    int64_t lda, ldb;        // row pitches of A and B (elements)
    int vec_c;               // C rows start 16-byte aligned and Q % 4 == 0
    int vec_a, vec_b;        // A / B read 4 contiguous elements at 16-byte boundaries
};

// One block row of C per (blockIdx.y, blockIdx.z); threads sweep the row's Q
// columns, four consecutive outputs each.
template <typename TI, typename TO>
__global__ void __launch_bounds__(256)
    ipophp_kernel(const TI* __restrict__ A, const TI* __restrict__ B, TO* __restrict__ C,
                  const ProductMap mp) {
    const int64_t r = blockIdx.y + static_cast<int64_t>(blockIdx.z) * gridDim.y;
    if (r >= mp.R) return;
    const TI* arow = A + (r / mp.ra) * mp.lda;
    const int64_t br = r % mp.rb;
    TO* crow = C + r * mp.Q;
    for (int64_t c0 = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) * 4;
         c0 < mp.Q; c0 += static_cast<int64_t>(gridDim.x) * blockDim.x * 4) {
        // column indices of the 4 outputs: A column c / ca, B column c % cb,
        // stepped instead of divided
        int64_t ac = c0 / mp.ca, ak = c0 - ac * mp.ca;
        int64_t bc = c0 % mp.cb;
        int64_t acol[4], bcol[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            acol[e] = ac;
            bcol[e] = bc;
            if (++ak == mp.ca) {
                ak = 0;
                ++ac;
            }
            if (++bc == mp.cb) bc = 0;
        }
        const int n_out = static_cast<int>(mp.Q - c0 < 4 ? mp.Q - c0 : 4);
        TO v[4];
        if (mp.S == 1) {
            TO a[4], b[4];
            if (mp.vec_a && n_out == 4 && acol[3] == acol[0] + 3) {
                if constexpr (sizeof(TI) == 8) {
                    const double2 x0 = *reinterpret_cast<const double2*>(arow + acol[0]);
                    const double2 x1 = *reinterpret_cast<const double2*>(arow + acol[0] + 2);
                    a[0] = x0.x; a[1] = x0.y; a[2] = x1.x; a[3] = x1.y;
                } else if constexpr (sizeof(TI) == 4) {
                    const float4 x = *reinterpret_cast<const float4*>(arow + acol[0]);
                    a[0] = x.x; a[1] = x.y; a[2] = x.z; a[3] = x.w;
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e) a[e] = widen<TI, TO>(arow[acol[e]]);
                }
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) a[e] = e < n_out ? widen<TI, TO>(arow[acol[e]]) : TO(0);
            }
            const TI* brow = B + br * mp.ldb;
            if (mp.vec_b && n_out == 4 && bcol[3] == bcol[0] + 3) {
                if constexpr (sizeof(TI) == 8) {
                    const double2 x0 = *reinterpret_cast<const double2*>(brow + bcol[0]);
                    const double2 x1 = *reinterpret_cast<const double2*>(brow + bcol[0] + 2);
                    b[0] = x0.x; b[1] = x0.y; b[2] = x1.x; b[3] = x1.y;
                } else if constexpr (sizeof(TI) == 4) {
                    const float4 x = *reinterpret_cast<const float4*>(brow + bcol[0]);
                    b[0] = x.x; b[1] = x.y; b[2] = x.z; b[3] = x.w;
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e) b[e] = widen<TI, TO>(brow[bcol[e]]);
                }
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) b[e] = e < n_out ? widen<TI, TO>(brow[bcol[e]]) : TO(0);
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) v[e] = mul_rn(a[e], b[e]);
        } else {
            // the contraction: products rounded, added in s order from 0
#pragma unroll
            for (int e = 0; e < 4; ++e) v[e] = TO(0);
            for (int64_t s = 0; s < mp.S; ++s) {
                const TI* brow = B + (br + s) * mp.ldb;
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (e < n_out)
                        v[e] = add_rn(v[e], mul_rn(widen<TI, TO>(arow[acol[e] + s]),
                                                   widen<TI, TO>(brow[bcol[e]])));
            }
        }
        if (mp.vec_c && n_out == 4) {
            if constexpr (sizeof(TO) == 4) {
                *reinterpret_cast<float4*>(crow + c0) = make_float4(v[0], v[1], v[2], v[3]);
            } else {
                reinterpret_cast<double2*>(crow + c0)[0] = make_double2(v[0], v[1]);
                reinterpret_cast<double2*>(crow + c0)[1] = make_double2(v[2], v[3]);
            }
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (e < n_out) crow[c0 + e] = v[e];
        }
    }
}

// Loads 4 consecutive elements row[c .. c+3] (16-byte aligned when vec).
template <typename TI, typename TO>
__device__ __forceinline__ void load4_at(const TI* __restrict__ row, uint32_t c, bool vec,
                                         TO (&x)[4]) {
    if constexpr (sizeof(TI) == 8) {
        if (vec) {
            const double2 x0 = *reinterpret_cast<const double2*>(row + c);
            const double2 x1 = *reinterpret_cast<const double2*>(row + c + 2);
            x[0] = x0.x; x[1] = x0.y; x[2] = x1.x; x[3] = x1.y;
            return;
        }
    } else if constexpr (sizeof(TI) == 4) {
        if (vec) {
            const float4 v = *reinterpret_cast<const float4*>(row + c);
            x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
            return;
        }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) x[e] = widen<TI, TO>(row[c + e]);
}

struct OuterMap {
    FastDiv gpr, ra, rb, ca, cb;   // groups per row; the map's divisors
    uint32_t R, Q, total;          // rows, columns; (row block, column group) pairs
    int64_t lda, ldb;
    int vec_a, vec_b, vec_c;
};

// The no-reduction members (S = 1) of the same map with 32-bit index
// arithmetic: each thread takes 4 consecutive outputs in each of ROWS
// consecutive rows per step (the column indices computed once, the row
// indices stepped), consecutive threads take consecutive column groups, so
// every warp store covers 512 contiguous bytes; A and B are read 16 bytes at
// a time where the map reads them contiguously.  ROWS = 8 for the Kronecker
// product (index arithmetic amortised over 8 rows; 0.76-0.78 of HBM against
// 0.59 with one row), 1 for the Hadamard product (pure streaming; 0.98 of
// HBM against 0.89 with 8 rows).
template <typename TI, typename TO, int ROWS>
__global__ void __launch_bounds__(256)
    ipophp_outer_kernel(const TI* __restrict__ A, const TI* __restrict__ B, TO* __restrict__ C,
                        const OuterMap mp) {
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < mp.total;
         g += gridDim.x * blockDim.x) {
        uint32_t cg, ak, bc, ark, br;
        const uint32_t r0 = fdiv(g, mp.gpr, cg) * ROWS;
        uint32_t ar = fdiv(r0, mp.ra, ark);
        fdiv(r0, mp.rb, br);
        const uint32_t c0 = cg * 4;
        uint32_t ac = fdiv(c0, mp.ca, ak);
        fdiv(c0, mp.cb, bc);
        const int n_out = mp.Q - c0 < 4 ? static_cast<int>(mp.Q - c0) : 4;
        uint32_t acol[4], bcol[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            acol[e] = ac;
            bcol[e] = bc;
            if (++ak == mp.ca.d) {
                ak = 0;
                ++ac;
            }
            if (++bc == mp.cb.d) bc = 0;
        }
        const bool a_run = n_out == 4 && acol[3] == acol[0] + 3;   // 4 contiguous A columns
        const bool a_one = n_out == 4 && acol[3] == acol[0];       // one A column
        const bool b_run = n_out == 4 && bcol[3] == bcol[0] + 3;
#pragma unroll
        for (int i = 0; i < ROWS; ++i) {
            const uint32_t r = r0 + i;
            if (r >= mp.R) break;
            const TI* arow = A + static_cast<int64_t>(ar) * mp.lda;
            const TI* brow = B + static_cast<int64_t>(br) * mp.ldb;
            TO a[4], b[4];
            if (a_run) {
                load4_at<TI, TO>(arow, acol[0], mp.vec_a != 0, a);
            } else if (a_one) {
                a[0] = a[1] = a[2] = a[3] = widen<TI, TO>(arow[acol[0]]);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) a[e] = e < n_out ? widen<TI, TO>(arow[acol[e]]) : TO(0);
            }
            if (b_run) {
                load4_at<TI, TO>(brow, bcol[0], mp.vec_b != 0, b);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) b[e] = e < n_out ? widen<TI, TO>(brow[bcol[e]]) : TO(0);
            }
            TO o[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) o[e] = mul_rn(a[e], b[e]);
            TO* crow = C + static_cast<int64_t>(r) * mp.Q;
            if (mp.vec_c && n_out == 4) {
                if constexpr (sizeof(TO) == 4) {
                    *reinterpret_cast<float4*>(crow + c0) = make_float4(o[0], o[1], o[2], o[3]);
                } else {
                    reinterpret_cast<double2*>(crow + c0)[0] = make_double2(o[0], o[1]);
                    reinterpret_cast<double2*>(crow + c0)[1] = make_double2(o[2], o[3]);
                }
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (e < n_out) crow[c0 + e] = o[e];
            }
            // the next row: A row r / ra and B row r % rb, stepped
            if (++ark == mp.ra.d) {
                ark = 0;
                ++ar;
            }
            if (++br == mp.rb.d) br = 0;
        }
    }
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

bool aligned16(const void* p, int64_t pitch_elems, int esize) {
    return reinterpret_cast<uintptr_t>(p) % 16 == 0 && (pitch_elems * esize) % 16 == 0;
}

int launch_product(moa_product_kind kind, int64_t m, int64_t n, int64_t p, int64_t q, moa_dtype dt,
                   const void* A, const void* B, void* C, cudaStream_t s) {
    int ie, oe;
    int rc = elem_sizes(dt, &ie, &oe);
    if (rc != MOA_OK) return rc;
    if (m < 0 || n < 0 || p < 0 || q < 0) return fail(MOA_ERR_ARG, "negative dimension");
    ProductMap mp{};
    mp.lda = n;
    mp.ldb = q;
    switch (kind) {
        case MOA_PRODUCT_KRONECKER:
            mp.R = m * p;
            mp.Q = n * q;
            mp.ra = p; mp.ca = q; mp.rb = p; mp.cb = q;
            mp.S = 1;
            break;
        case MOA_PRODUCT_HADAMARD:
            if (p != m || q != n) return fail(MOA_ERR_ARG, "Hadamard product needs equal shapes");
            mp.R = m;
            mp.Q = n;
            mp.ra = 1; mp.ca = 1; mp.rb = m > 0 ? m : 1; mp.cb = n > 0 ? n : 1;
            mp.S = 1;
            break;
        case MOA_PRODUCT_MATMUL:
            if (n != p) return fail(MOA_ERR_ARG, "matrix product needs n == p");
            mp.R = m;
            mp.Q = q;
            mp.ra = 1; mp.ca = q > 0 ? q : 1; mp.rb = 1; mp.cb = q > 0 ? q : 1;
            mp.S = n;
            break;
        default:
            return fail(MOA_ERR_ARG, "unknown product kind");
    }
    if (mp.R == 0 || mp.Q == 0) return MOA_OK;
    if (!C) return fail(MOA_ERR_ARG, "NULL operand");
    if (mp.S > 0 && (!A || !B)) return fail(MOA_ERR_ARG, "NULL operand");
    if (reinterpret_cast<uintptr_t>(A) % ie || reinterpret_cast<uintptr_t>(B) % ie ||
        reinterpret_cast<uintptr_t>(C) % oe)
        return fail(MOA_ERR_ALIGN, "pointer not aligned to its element size");
    mp.vec_c = (mp.Q % 4 == 0) && (reinterpret_cast<uintptr_t>(C) % 16 == 0);
    // contiguous 4-element reads: the column index steps by 1 (ca == 1 for A,
    // cb >= 4 for B within a group), 16-byte aligned rows, groups of 4 aligned
    mp.vec_a = kind == MOA_PRODUCT_HADAMARD && aligned16(A, mp.lda, ie);
    mp.vec_b = (kind == MOA_PRODUCT_HADAMARD || (kind == MOA_PRODUCT_KRONECKER && q % 4 == 0)) &&
               aligned16(B, mp.ldb, ie);
    const int threads = 256;
    const int rows_step = kind == MOA_PRODUCT_KRONECKER ? 8 : 1;
    const int64_t groups = ceil_div(mp.R, rows_step) * ceil_div(mp.Q, 4);
    if (mp.S == 1 && groups < (int64_t(1) << 31) - 65536L * threads &&
        mp.R < (int64_t(1) << 31) - 8 && mp.Q < (int64_t(1) << 31) - 4) {
        OuterMap om{};
        om.gpr = make_fastdiv(static_cast<uint32_t>(ceil_div(mp.Q, 4)));
        om.ra = make_fastdiv(static_cast<uint32_t>(mp.ra));
        om.rb = make_fastdiv(static_cast<uint32_t>(mp.rb));
        om.ca = make_fastdiv(static_cast<uint32_t>(mp.ca));
        om.cb = make_fastdiv(static_cast<uint32_t>(mp.cb));
        om.R = static_cast<uint32_t>(mp.R);
        om.Q = static_cast<uint32_t>(mp.Q);
        om.total = static_cast<uint32_t>(groups);
        om.lda = mp.lda;
        om.ldb = mp.ldb;
        om.vec_a = mp.vec_a;
        om.vec_b = mp.vec_b;
        om.vec_c = mp.vec_c;
        const int64_t want = ceil_div(groups, threads);
        const int blocks = static_cast<int>(std::min<int64_t>(want, 32L * num_sms()));
        auto run = [&](auto rows_tag) {
            constexpr int ROWS = decltype(rows_tag)::value;
            if (dt == MOA_F64)
                ipophp_outer_kernel<double, double, ROWS><<<blocks, threads, 0, s>>>(
                    static_cast<const double*>(A), static_cast<const double*>(B),
                    static_cast<double*>(C), om);
            else if (dt == MOA_BF16)
                ipophp_outer_kernel<__nv_bfloat16, float, ROWS><<<blocks, threads, 0, s>>>(
                    static_cast<const __nv_bfloat16*>(A), static_cast<const __nv_bfloat16*>(B),
                    static_cast<float*>(C), om);
            else
                ipophp_outer_kernel<float, float, ROWS><<<blocks, threads, 0, s>>>(
                    static_cast<const float*>(A), static_cast<const float*>(B),
                    static_cast<float*>(C), om);
        };
        if (rows_step == 8)
            run(std::integral_constant<int, 8>{});
        else
            run(std::integral_constant<int, 1>{});
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "ipophp_outer_kernel launch");
        return MOA_OK;
    }
    const int64_t gx = ceil_div(ceil_div(mp.Q, 4), threads);
    dim3 grid(static_cast<unsigned>(gx < 64 ? gx : 64),
              static_cast<unsigned>(mp.R < 65535 ? mp.R : 65535),
              static_cast<unsigned>(ceil_div(mp.R, 65535)));
    if (grid.z > 65535) return fail(MOA_ERR_ARG, "product output too tall");
    if (dt == MOA_F64)
        ipophp_kernel<double, double><<<grid, threads, 0, s>>>(
            static_cast<const double*>(A), static_cast<const double*>(B), static_cast<double*>(C), mp);
    else if (dt == MOA_BF16)
        ipophp_kernel<__nv_bfloat16, float><<<grid, threads, 0, s>>>(
            static_cast<const __nv_bfloat16*>(A), static_cast<const __nv_bfloat16*>(B),
            static_cast<float*>(C), mp);
    else
        ipophp_kernel<float, float><<<grid, threads, 0, s>>>(
            static_cast<const float*>(A), static_cast<const float*>(B), static_cast<float*>(C), mp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "ipophp_kernel launch");
    return MOA_OK;
}

}  // namespace
}  // namespace moa

extern "C" {

int moa_product(moa_product_kind kind, int64_t m, int64_t n, int64_t p, int64_t q, moa_dtype dt,
                const void* A, const void* B, void* C, void* stream) {
    moa::TraceRange tr("moa_product");
    return moa::launch_product(kind, m, n, p, q, dt, A, B, C, static_cast<cudaStream_t>(stream));
}

int moa_kronecker(int64_t m, int64_t n, int64_t p, int64_t q, moa_dtype dt, const void* A,
                  const void* B, void* C, void* stream) {
    moa::TraceRange tr("moa_kronecker");
    return moa::launch_product(MOA_PRODUCT_KRONECKER, m, n, p, q, dt, A, B, C,
                               static_cast<cudaStream_t>(stream));
}

int moa_hadamard(int64_t m, int64_t n, moa_dtype dt, const void* A, const void* B, void* C,
                 void* stream) {
    moa::TraceRange tr("moa_hadamard");
    return moa::launch_product(MOA_PRODUCT_HADAMARD, m, n, m, n, dt, A, B, C,
                               static_cast<cudaStream_t>(stream));
}

}  // extern "C"
