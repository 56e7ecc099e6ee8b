// split.cu -- split-precision ONF GEMM: the bulk of the products run as BF16
// slice products on the tcgen05 tensor cores, accumulated in FP32 TMEM, and are
// recombined to FP32 accuracy (MOA_F32_SPLIT) or FP64 accuracy (MOA_F64_SPLIT_*).
//
// The result is still Eq. (eq:dnf) of Sec. 2, C[(i*p)+j] := sum_k A[(i*n)+k] *
// B[(k*p)+j]; the slicing is not in the paper (it is the "Precision" pattern of
// this library):
//
// * FP32 accuracy (Henry, Tang & Heinecke 2019): every FP32 x is split as
//   x = s0 + s1 + s2, s_t = RN_bf16(x - s0 - ... - s_{t-1}); the six slice
//   products with t + u <= 2 are summed into one FP32 accumulator.
// * FP64 accuracy (error-free digit slicing in the manner of Ozaki, Ogita,
//   Oishi & Rump 2012): each row i of A gets the exponent eA_i with
//   max_k |A[i,k]| in [2^(eA_i - 1 - h), 2^(eA_i - h)) (h = 1 headroom bit),
//   each column j of B likewise eB_j; x * 2^(7S - e) is rounded once to an
//   integer D and written as S balanced base-128 digits (|d_0| <= 64 with the
//   headroom bit, d_s in [-64, 64) for s >= 1), each exactly a BF16 value.  Level L = s + t of the triangular product (s + t <= S - 1)
//   is summed over chunks of K short enough that every FP32 partial sum is an
//   integer below 2^24, hence exact; each chunk is flushed into an int32
//   running sum, folded at the level's end into an int64 fixed-point total
//   kept in C, which the epilogue converts to FP64 once and scales by
//   2^(eA_i + eB_j - 7(S+1) + drop).
//
// Kernel layout (one persistent CTA per SM): warp 0 issues TMA loads of
// (A slice, B slice) K blocks; warp 1 issues tcgen05.mma into one of one or
// two TMEM chunk accumulators; the epilogue warps (one per TMEM lane
// quadrant and column group) flush chunks and write C.  The CTAs walk work
// units: whole output tiles, or, in the FP64 modes when the tiles fill at
// most half of the SMs, (tile, K slice) pairs whose int64 totals meet in C by
// exact atomic adds (split K).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "fpbits.cuh"
#include "internal.h"
#include "ptx.cuh"
#include "split.h"

namespace moa {

// ====================================================================== pre-passes
namespace {

__device__ __forceinline__ uint32_t bf16x2_bits(__nv_bfloat162 v) {
    return static_cast<uint32_t>(__bfloat16_as_ushort(v.x)) |
           (static_cast<uint32_t>(__bfloat16_as_ushort(v.y)) << 16);
}

// BF16 bit patterns of two small integers (|lo|, |hi| < 2^8, exact in BF16),
// packed low half first.  The integer is placed in the significand of
// 1.5 * 2^23 (magic-number conversion: for |k| < 2^22 the float with bits
// 0x4B400000 + k equals 1.5 * 2^23 + k) and the offset subtracted, both
// exact; the result has at most 8 significant bits, so its upper 16 bits are
// its BF16 pattern.  Plain ALU work instead of integer-to-float conversions.
__device__ __forceinline__ uint32_t small_ints_bf16x2(int lo, int hi) {
    const uint32_t flo =
        __float_as_uint(__fsub_rn(__uint_as_float(0x4B400000u + static_cast<uint32_t>(lo)), 12582912.0f));
    const uint32_t fhi =
        __float_as_uint(__fsub_rn(__uint_as_float(0x4B400000u + static_cast<uint32_t>(hi)), 12582912.0f));
    return (flo >> 16) | (fhi & 0xFFFF0000u);
}

// Loads X[r, c0 .. c0+7] (zero past `cols`); 16-byte loads when allowed.
__device__ __forceinline__ void load8(const float* __restrict__ X, int64_t r, int64_t cols,
                                      int64_t c0, bool vec, float (&x)[8]) {
    const float* src = X + r * cols + c0;
    if (vec && c0 + 8 <= cols) {
        const float4 a = reinterpret_cast<const float4*>(src)[0];
        const float4 b = reinterpret_cast<const float4*>(src)[1];
        x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
        x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = (c0 + i < cols) ? src[i] : 0.f;
    }
}

// FP32 -> three BF16 slices, zero-padded to row pitch ld (a multiple of 8);
// 8 consecutive elements per thread, one 16-byte store per slice plane.
// Flags NaN/Inf (and values whose leading slice overflows BF16) in the
// status word.
// The pre-pass kernels below are written as "parts" over a range of blocks
// (bid of nblk), so that one launch can run the part for A and the part for
// B side by side: fewer launches per GEMM, which matters for small problems.
__device__ void split3_part(const float* __restrict__ X, int64_t rows, int64_t cols, int64_t ld,
                            __nv_bfloat16* __restrict__ out, int64_t plane, int vec, int* status,
                            int64_t bid, int64_t nblk) {
    const int64_t gpr = ld / 8;                 // 8-element groups per row
    const int64_t total = rows * gpr;
    bool bad = false;
    for (int64_t g = bid * blockDim.x + threadIdx.x; g < total; g += nblk * blockDim.x) {
        const int64_t r = g / gpr, c0 = (g - r * gpr) * 8;
        float x[8];
        load8(X, r, cols, c0, vec != 0, x);
        uint32_t w0[4], w1[4], w2[4];
#pragma unroll
        for (int i = 0; i < 8; i += 2) {
            // two elements per conversion instruction; BF16 -> FP32 is exact
            const __nv_bfloat162 a = __floats2bfloat162_rn(x[i], x[i + 1]);
            const float2 af = __bfloat1622float2(a);
            const float r0 = __fsub_rn(x[i], af.x), r1 = __fsub_rn(x[i + 1], af.y);
            const __nv_bfloat162 b = __floats2bfloat162_rn(r0, r1);
            const float2 bf = __bfloat1622float2(b);
            const __nv_bfloat162 c =
                __floats2bfloat162_rn(__fsub_rn(r0, bf.x), __fsub_rn(r1, bf.y));
            bad |= !isfinite(x[i]) || !isfinite(x[i + 1]) || !isfinite(af.x) || !isfinite(af.y);
            w0[i / 2] = bf16x2_bits(a);
            w1[i / 2] = bf16x2_bits(b);
            w2[i / 2] = bf16x2_bits(c);
        }
        const int64_t o = r * ld + c0;
        *reinterpret_cast<uint4*>(out + o) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
        *reinterpret_cast<uint4*>(out + plane + o) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
        *reinterpret_cast<uint4*>(out + 2 * plane + o) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
    }
    if (bad) atomicCAS(status, kDevOk, kDevNonFinite);
}

// Blocks [0, ga) split A, the rest split B.
__global__ void split3_pair_kernel(const float* __restrict__ A, int64_t m, int64_t n, int64_t lda,
                                   __nv_bfloat16* __restrict__ a_out, int64_t a_plane, int va,
                                   const float* __restrict__ B, int64_t p, int64_t ldb,
                                   __nv_bfloat16* __restrict__ b_out, int64_t b_plane, int vb,
                                   int* status, int ga) {
    if (static_cast<int>(blockIdx.x) < ga)
        split3_part(A, m, n, lda, a_out, a_plane, va, status, blockIdx.x, ga);
    else
        split3_part(B, n, p, ldb, b_out, b_plane, vb, status, blockIdx.x - ga, gridDim.x - ga);
}

// One problem of a grouped FP32-accuracy split call, as the pre-pass sees it:
// its operands, slice planes and the blocks [begin, begin + ga + gb) of the
// launch (the first ga split A, the rest B).
struct SplitGPass {
    const float* A;
    const float* B;
    __nv_bfloat16* a_sl;
    __nv_bfloat16* b_sl;
    int64_t m, n, p, lda, ldb, a_plane, b_plane;
    int* status;   // where this problem's non-finite inputs are recorded
    int va, vb, ga, gb, begin, pad;
};

// The slice pre-pass of every problem of a grouped call in one launch (the
// problem of block b by binary search over the problems' first blocks).
__global__ void __launch_bounds__(256)
    split3_g_kernel(const SplitGPass* __restrict__ pr, int count) {
    const int b = static_cast<int>(blockIdx.x);
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pr[mid].begin <= b) lo = mid; else hi = mid - 1;
    }
    const SplitGPass& x = pr[lo];
    const int local = b - x.begin;
    if (local < x.ga)
        split3_part(x.A, x.m, x.n, x.lda, x.a_sl, x.a_plane, x.va, x.status, local, x.ga);
    else if (local < x.ga + x.gb)
        split3_part(x.B, x.n, x.p, x.ldb, x.b_sl, x.b_plane, x.vb, x.status, local - x.ga, x.gb);
}

// Digit generator of one element: D = round_half_even(x * 2^k) written as
// balanced radix-2^beta digits from the bottom, d_s for s = S-1 .. 1 in
// [-2^(beta-1), 2^(beta-1)), then d_0 = what is left.  next(s) must be called
// for s = S-1, S-2, ..., 0 in that order.
template <typename T>
struct DigitGen;

// FP64 input: D needs up to 62 bits; 64-bit integer steps.
template <>
struct DigitGen<double> {
    long long D;
    __device__ void start(double x, int k, int) { D = Bits<double>::round_scaled(x, k); }
    __device__ int next(int s, int beta, int) {
        if (s == 0) return static_cast<int>(D);
        const int radix = 1 << beta;
        int low = static_cast<int>(D) & (radix - 1);
        low -= (low & (radix >> 1)) << 1;
        D = (D - low) >> beta;
        return low;
    }
    // next(s) + 2^(beta-1): with t = D + 2^(beta-1), the balanced digit plus
    // its bias is t mod 2^beta and the remainder is floor(t / 2^beta).
    __device__ int next_biased(int s, int beta, int) {
        const long long t = D + (1ll << (beta - 1));
        if (s == 0) return static_cast<int>(t);
        D = t >> beta;
        return static_cast<int>(t) & ((1 << beta) - 1);
    }
};

// FP32 input: D = M * 2^sh with a 24-bit M.  For sh >= 0 the bottom
// zd = floor(sh / beta) digits are zero and the rest come from the 32-bit
// m = M * 2^(sh mod beta) (below 2^(24 + beta - 1) <= 2^30); for sh < 0, D
// itself is below 2^25.  All steps are 32-bit.
template <>
struct DigitGen<float> {
    int m;
    int zd;
    __device__ void start(float x, int k, int beta) {
        const uint32_t b = __float_as_uint(x);
        const int ex = static_cast<int>((b >> 23) & 0xFF);
        uint32_t mant = b & 0x7FFFFFu;
        int E = -149;
        if (ex != 0) {
            mant |= 1u << 23;
            E = ex - 150;
        }
        const int sh = E + k;
        uint32_t mag;
        if (mant == 0) {
            mag = 0;
            zd = 0;
        } else if (sh >= 0) {
            zd = sh / beta;
            mag = mant << (sh - zd * beta);
        } else {
            zd = 0;
            const int kk = -sh;
            if (kk > 25) {
                mag = 0;
            } else {
                const uint32_t q = mant >> kk;
                const uint32_t rem = mant & ((1u << kk) - 1u);
                const uint32_t half = 1u << (kk - 1);
                mag = q + ((rem > half || (rem == half && (q & 1u))) ? 1u : 0u);
            }
        }
        m = (b >> 31) ? -static_cast<int>(mag) : static_cast<int>(mag);
    }
    __device__ int next(int s, int beta, int S) {
        const int pos = S - 1 - s;   // digit position from the bottom
        if (pos < zd) return 0;
        if (s == 0) return m;
        const int radix = 1 << beta;
        int low = m & (radix - 1);
        low -= (low & (radix >> 1)) << 1;
        m = (m - low) >> beta;
        return low;
    }
    __device__ int next_biased(int s, int beta, int S) {
        const int half = 1 << (beta - 1);
        const int t = m + half;
        const bool zero = S - 1 - s < zd;
        if (s == 0) return zero ? half : t;
        m = zero ? m : (t >> beta);
        return zero ? half : (t & ((1 << beta) - 1));
    }
};

// One warp per row: exponent of max |A[i,:]| plus `bias` (headroom bits).
template <typename T>
__device__ void row_exp_part(const T* __restrict__ X, int64_t rows, int64_t cols, int bias,
                             int* __restrict__ e_out, int* status, int64_t bid, int64_t nblk) {
    using B = Bits<T>;
    const int lane = threadIdx.x & 31;
    const int64_t warps = nblk * (blockDim.x >> 5);
    bool bad = false;
    for (int64_t r = bid * (blockDim.x >> 5) + (threadIdx.x >> 5); r < rows; r += warps) {
        typename B::U mx = 0;
        for (int64_t c = lane; c < cols; c += 32) mx = max(mx, B::abs_bits(X[r * cols + c]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const typename B::U other = __shfl_xor_sync(0xffffffffu, mx, o);
            mx = max(mx, other);
        }
        if (lane == 0) {
            bad |= mx >= B::kInf;
            e_out[r] = B::frexp_exp(mx) + bias;
        }
    }
    if (bad) atomicCAS(status, kDevOk, kDevNonFinite);
}

// Column maxima of |B| (bit patterns), by atomicMax over row chunks: block
// bid covers columns 256 (bid % gx) .. + 255 and rows chunk (bid / gx) ..
template <typename T>
__device__ void col_max_part(const T* __restrict__ X, int64_t rows, int64_t cols, int64_t chunk,
                             typename Bits<T>::U* __restrict__ cmax, int64_t bid, int64_t gx) {
    using B = Bits<T>;
    const int64_t c = (bid % gx) * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    const int64_t r0 = (bid / gx) * chunk;
    const int64_t r1 = min(rows, r0 + chunk);
    typename B::U mx = 0;
    for (int64_t r = r0; r < r1; ++r) mx = max(mx, B::abs_bits(X[r * cols + c]));
    atomicMax(&cmax[c], mx);
}

// Exponent of a column of B from its max bit pattern (plus `bias`); flags
// NaN/Inf in *status unless status is null.
template <typename T>
__device__ __forceinline__ int col_exp(typename Bits<T>::U M, int bias, int* status) {
    if (status && M >= Bits<T>::kInf) atomicCAS(status, kDevOk, kDevNonFinite);
    return Bits<T>::frexp_exp(M) + bias;
}

// Blocks [0, rblocks): row exponents of A; the next cblocks: column maxima
// of B; the last zblocks (split K only): clear z0[0 .. n0) and z1[0 .. n1)
// (the int64 totals in C and the finished-unit counters).
template <typename T>
__global__ void __launch_bounds__(256)
    exps_kernel(const T* __restrict__ A, int64_t m, int64_t n, const T* __restrict__ B, int64_t p,
                int64_t chunk, int bias, int* __restrict__ eA, typename Bits<T>::U* __restrict__ cmax,
                int* status, int rblocks, int64_t gx, int cblocks, unsigned long long* z0,
                int64_t n0, unsigned long long* z1, int64_t n1) {
    const int b = static_cast<int>(blockIdx.x);
    if (b < rblocks) {
        row_exp_part(A, m, n, bias, eA, status, b, rblocks);
    } else if (b < rblocks + cblocks) {
        col_max_part(B, n, p, chunk, cmax, b - rblocks, gx);
    } else {
        const int64_t zb = b - rblocks - cblocks, nz = gridDim.x - rblocks - cblocks;
        for (int64_t i = zb * blockDim.x + threadIdx.x; i < n0 + n1; i += nz * blockDim.x) {
            if (i < n0)
                z0[i] = 0ull;
            else
                z1[i - n0] = 0ull;
        }
    }
}

// Loads X[r, c0 .. c0+7] of an FP64 matrix (zero past `cols`).
__device__ __forceinline__ void load8(const double* __restrict__ X, int64_t r, int64_t cols,
                                      int64_t c0, bool vec, double (&x)[8]) {
    const double* src = X + r * cols + c0;
    if (vec && c0 + 8 <= cols) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const double2 d = reinterpret_cast<const double2*>(src)[v];
            x[2 * v] = d.x;
            x[2 * v + 1] = d.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = (c0 + i < cols) ? src[i] : 0.0;
    }
}

// Integer digits of every element into S BF16 planes (row pitch ld, a
// multiple of 8; zero pad); 8 consecutive elements per thread, one 16-byte
// store per digit plane.  AXIS 0: exponent per row, read from e[r].  AXIS 1:
// exponent per column, formed here from the column maximum cmax[c] plus
// `bias`; the threads of row 0 store it to e[c] and flag NaN/Inf.  vec: X
// rows start 16-byte aligned (16-byte loads).
template <typename T, int AXIS>
__device__ void digits_part(const T* __restrict__ X, int64_t rows, int64_t cols, int64_t ld,
                            int* __restrict__ e, const typename Bits<T>::U* __restrict__ cmax,
                            int bias, int* status, int S, int vec,
                            __nv_bfloat16* __restrict__ out, int64_t plane, int64_t bid,
                            int64_t nblk) {
    const int64_t gpr = ld / 8;
    const int64_t total = rows * gpr;
    for (int64_t g = bid * blockDim.x + threadIdx.x; g < total; g += nblk * blockDim.x) {
        const int64_t r = g / gpr, c0 = (g - r * gpr) * 8;
        T x[8];
        load8(X, r, cols, c0, vec != 0, x);
        DigitGen<T> D[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int64_t c = c0 + i;
            int ex = 0;
            if (c < cols) {
                if (AXIS == 0) {
                    ex = e[r];
                } else {
                    ex = col_exp<T>(cmax[c], bias, r == 0 ? status : nullptr);
                    if (r == 0) e[c] = ex;
                }
            }
            D[i].start(x[i], kBeta * S - ex, kBeta);
        }
        const int64_t o = r * ld + c0;
        for (int s = S - 1; s >= 0; --s) {
            uint32_t w[4];
#pragma unroll
            for (int i = 0; i < 8; i += 2)   // |d| <= 2^kBeta: exact BF16 values
                w[i / 2] = small_ints_bf16x2(D[i].next(s, kBeta, S), D[i + 1].next(s, kBeta, S));
            *reinterpret_cast<uint4*>(out + s * plane + o) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// Blocks [0, ga): digits of A (row exponents eA); the rest: digits of B
// (column exponents from cmax, stored to eB).
template <typename T>
__global__ void __launch_bounds__(256)
    digits_pair_kernel(const T* __restrict__ A, int64_t m, int64_t n, int64_t lda, int va,
                       const int* __restrict__ eA, const T* __restrict__ B, int64_t p, int64_t ldb,
                       int vb, int* __restrict__ eB, const typename Bits<T>::U* __restrict__ cmax,
                       int bias, int* status, int S, __nv_bfloat16* __restrict__ a_out,
                       int64_t a_plane, __nv_bfloat16* __restrict__ b_out, int64_t b_plane, int ga) {
    if (static_cast<int>(blockIdx.x) < ga)
        digits_part<T, 0>(A, m, n, lda, const_cast<int*>(eA), nullptr, 0, status, S, va, a_out,
                          a_plane, blockIdx.x, ga);
    else
        digits_part<T, 1>(B, n, p, ldb, eB, cmax, bias, status, S, vb, b_out, b_plane,
                          blockIdx.x - ga, gridDim.x - ga);
}

// E4M3 bit pattern of an integer v with |v| <= 16 (exact in E4M3: sign,
// 4 exponent bits with bias 7, 3 stored mantissa bits).  |v| in [2^q, 2^(q+1))
// has exponent field q + 7 and mantissa bits (|v| * 2^(3 - q)) mod 8.
__device__ __forceinline__ uint32_t e4m3_of_small_int(int v) {
    const uint32_t a = static_cast<uint32_t>(v < 0 ? -v : v);
    const int q = 31 - __clz(static_cast<int>(a | 1u));       // a = 0 gives q = 0
    const uint32_t bits = (static_cast<uint32_t>(q + 7) << 3) | (((a << 3) >> q) & 7u);
    return a == 0 ? 0u : (bits | (v < 0 ? 0x80u : 0u));
}

// Shared-memory table of the E4M3 codes of the biased digits: lut[i] is the
// code of i - 2^(beta-1), i in [0, 2^beta].  Filled by the first threads of
// the block; the caller synchronises before use.
__device__ __forceinline__ void fill_e4m3_lut(uint8_t* lut, int beta) {
    const int half = 1 << (beta - 1);
    if (threadIdx.x <= 2 * half) lut[threadIdx.x] = static_cast<uint8_t>(e4m3_of_small_int(
                                     static_cast<int>(threadIdx.x) - half));
}

// Integer digits (radix 2^beta) of a row-major matrix whose exponent is per
// row, as E4M3 bytes in S planes of row pitch ld (a multiple of 16; zero
// pad): 16 consecutive elements per thread, one 16-byte store per plane.
// lut: the block's E4M3 code table (fill_e4m3_lut, synchronised).
template <typename T>
__device__ void digits_e4m3_rows_part(const T* __restrict__ X, int64_t rows, int64_t cols,
                                      int64_t ld, const int* __restrict__ e, int S, int beta,
                                      int vec, uint8_t* __restrict__ out, int64_t plane,
                                      const uint8_t* lut, int64_t bid, int64_t nblk) {
    const int64_t gpr = ld / 16;
    const int64_t total = rows * gpr;
    for (int64_t g = bid * blockDim.x + threadIdx.x; g < total; g += nblk * blockDim.x) {
        const int64_t r = g / gpr, c0 = (g - r * gpr) * 16;
        const int ex = e[r];
        DigitGen<T> D[16];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            T x[8];
            load8(X, r, cols, c0 + 8 * h, vec != 0, x);
#pragma unroll
            for (int i = 0; i < 8; ++i) D[8 * h + i].start(x[i], beta * S - ex, beta);
        }
        const int64_t o = r * ld + c0;
        for (int s = S - 1; s >= 0; --s) {
            uint32_t w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint32_t word = 0;
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    word |= static_cast<uint32_t>(lut[D[4 * q + b].next_biased(s, beta, S)])
                            << (8 * b);
                w[q] = word;
            }
            *reinterpret_cast<uint4*>(out + s * plane + o) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// Integer digits of B (n x p row-major, exponent per column j, formed from
// the column maximum cmax[j] plus `bias`; the tiles at k = 0 store it to e[j]
// and flag NaN/Inf) written transposed as E4M3 bytes: plane s holds B_s^T, p
// rows of pitch ld (a multiple of 16; zero pad past n), so that the slice
// GEMM reads B K-major.
// One 64 (k) x 64 (j) tile per block pass, 256 threads; thread (j, q) holds
// the 16 consecutive k of quarter q in column j.  Reads are coalesced along j;
// each plane goes through a padded shared-memory tile (one 32-bit store per
// 4 bytes) and is written as 16-byte row segments along k.
constexpr int kTT = 64;
// tile: kTT * (kTT / 4 + 1) words of shared memory; lut as above.  Every
// thread of the block runs this part (it synchronises the block).
constexpr int kTileWords = kTT * (kTT / 4 + 1);
template <typename T>
__device__ void digits_e4m3_cols_t_part(const T* __restrict__ X, int64_t rows, int64_t cols,
                                        int64_t ld, int* __restrict__ e,
                                        const typename Bits<T>::U* __restrict__ cmax, int bias,
                                        int* status, int S, int beta, uint8_t* __restrict__ out,
                                        int64_t plane, uint32_t* tile, const uint8_t* lut,
                                        int64_t bid, int64_t nblk) {
    const int t = threadIdx.x;
    const int64_t tk = (rows + kTT - 1) / kTT, tj = (cols + kTT - 1) / kTT;
    for (int64_t b = bid; b < tk * tj; b += nblk) {
        const int64_t k0 = (b / tj) * kTT, j0 = (b % tj) * kTT;
        const int jl = t % kTT, kq = t / kTT;          // column in tile, k quarter 0..3
        const int64_t j = j0 + jl;
        const bool first = k0 == 0 && kq == 0;
        const int ex = j < cols ? col_exp<T>(cmax[j], bias, first ? status : nullptr) : 0;
        if (first && j < cols) e[j] = ex;
        DigitGen<T> D[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int64_t k = k0 + 16 * kq + i;
            const T x = (j < cols && k < rows) ? X[k * cols + j] : T(0);
            D[i].start(x, beta * S - ex, beta);
        }
        for (int s = S - 1; s >= 0; --s) {
            __syncthreads();   // the previous plane's tile has been written out
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint32_t word = 0;
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    word |= static_cast<uint32_t>(lut[D[4 * q + b].next_biased(s, beta, S)])
                            << (8 * b);
                tile[jl * (kTT / 4 + 1) + 4 * kq + q] = word;
            }
            __syncthreads();
            // thread t writes row jr = t / 4, bytes [16 c, 16 c + 16) of the tile
            const int jr = t / 4, c = t % 4;
            const int64_t kk = k0 + 16 * c;
            if (j0 + jr < cols && kk < ld) {
                const uint32_t* row = tile + jr * (kTT / 4 + 1) + 4 * c;
                *reinterpret_cast<uint4*>(out + s * plane + (j0 + jr) * ld + kk) =
                    make_uint4(row[0], row[1], row[2], row[3]);
            }
        }
        __syncthreads();
    }
}

// Blocks [0, ga): E4M3 digits of A by rows; the rest: transposed E4M3 digits
// of B (column exponents from cmax, stored to eB).  The branch is uniform per
// block, so the block-wide barriers of the B part are safe.
template <typename T>
__global__ void __launch_bounds__(256)
    digits_e4m3_pair_kernel(const T* __restrict__ A, int64_t m, int64_t n, int64_t lda, int va,
                            const int* __restrict__ eA, const T* __restrict__ B, int64_t p,
                            int64_t ldb, int* __restrict__ eB,
                            const typename Bits<T>::U* __restrict__ cmax, int bias, int* status,
                            int S, int beta, uint8_t* __restrict__ a_out, int64_t a_plane,
                            uint8_t* __restrict__ b_out, int64_t b_plane, int ga) {
    __shared__ uint32_t tile[kTileWords];   // [j][k/4], 17 words per row
    __shared__ uint8_t lut[64];
    fill_e4m3_lut(lut, beta);
    __syncthreads();
    if (static_cast<int>(blockIdx.x) < ga)
        digits_e4m3_rows_part<T>(A, m, n, lda, eA, S, beta, va, a_out, a_plane, lut, blockIdx.x,
                                 ga);
    else
        digits_e4m3_cols_t_part<T>(B, n, p, ldb, eB, cmax, bias, status, S, beta, b_out, b_plane,
                                   tile, lut, blockIdx.x - ga, gridDim.x - ga);
}

// 1 when every row of a row-major matrix with `cols` columns starts on a
// 16-byte boundary (base aligned, row length a multiple of `per16` elements).
int vec_rows(const void* X, int64_t cols, int per16) {
    return (cols % per16 == 0) && (reinterpret_cast<uintptr_t>(X) % 16 == 0);
}

int grid_for(int64_t total, int threads) {
    const int64_t want = ceil_div(total, threads);
    const int64_t cap = 16L * num_sms();
    return static_cast<int>(std::max<int64_t>(1, std::min(want, cap)));
}

}  // namespace

// ====================================================================== slice GEMM
namespace {

constexpr int kBM = 128, kBK = 64;                // kBK: BF16 elements per K block
constexpr int kABytes = kBM * 128;                 // 128 rows x 128 bytes of K
constexpr int kMaxLevels = 12;
// Largest tile count (at width 128) for which the workspace holds the split-K
// counters and fine-level sums.
constexpr int64_t kSplitKMaxTiles = 320;
// Digit-plane formats of the slice GEMM.  kFmtBF16: kind::f16, B planes
// MN-major (n x p, read as 64-column chunks).  kFmtE4M3: kind::f8f6f4, B
// planes hold B^T (p x n, K-major, one box per stage).  A K block is 128
// bytes of K either way: 64 BF16 or 128 E4M3 elements.
// kFmtBF16KB (FP32 accuracy only): all three BF16 slices of A and of B of
// one 32-deep K block share a stage (A K-major with 64-byte rows, 64-byte
// swizzle), and the six slice products of that K block run from it: every
// staged byte feeds two or three products, half the operand bytes per MMA
// cycle of one (A slice, B slice) pair per stage.
constexpr int kFmtBF16 = 0, kFmtE4M3 = 1, kFmtBF16KB = 2;
template <int FMT>
constexpr int block_k() { return FMT == kFmtE4M3 ? 128 : (FMT == kFmtBF16KB ? 32 : 64); }

// Kernel variants (tile width BN x epilogue mode):
//   kModeF32     FP32 accuracy; two chunk accumulators; each epilogue warp keeps
//                FP32 running sums of 64 columns in registers (BN / 16 warps).
//   kModeF64Reg  FP64 accuracy; two chunk accumulators; exact int32 level sums
//                of 64 columns per warp in registers (BN 128 or 192).
//   kModeF64Tmem FP64 accuracy at BN = 256: one chunk accumulator (TMEM columns
//                0..255) and the exact int32 level sums in TMEM (256..511);
//                8 epilogue warps of 128 columns each.
// The FP64 modes keep the tile's int64 fixed-point total in C itself.
constexpr int kModeF32 = 0, kModeF64Reg = 1, kModeF64Tmem = 2;

template <int BN, int MODE, int FMT>
struct SplitCfg {
    static constexpr int kBKe = block_k<FMT>();   // K elements per stage
    static constexpr bool kKB = FMT == kFmtBF16KB;
    // A part of a stage: one slice (128 rows x 128 B) or, kb-major, three
    // slices of 128 rows x 64 B; B part: BN / 64 chunks of 64 columns x kBKe
    // K rows per slice staged.
    static constexpr int kASlice = kKB ? kBM * 64 : kABytes;
    static constexpr int kAStage = kKB ? 3 * kASlice : kABytes;
    static constexpr int kBChunk = kBKe * 128;   // MN-major chunk (BF16 formats)
    static constexpr int kBSlice = FMT == kFmtE4M3 ? BN * 128 : (BN / 64) * kBChunk;
    static constexpr int kBBytes = kKB ? 3 * kBSlice : kBSlice;
    static constexpr int kStageBytes = kAStage + kBBytes;
    static constexpr int kColsPerWarp = MODE == kModeF64Tmem ? 128 : 64;
    static constexpr int kEpiWarps = 4 * (BN / kColsPerWarp);
    // FP64 modes: a 2 KB staging tile per epilogue warp for the folds
    static constexpr int kEpiStageWarp = 2048;
    static constexpr int kEpiStage = MODE == kModeF32 ? 0 : kEpiWarps * kEpiStageWarp;
    static constexpr int kStagesWant =
        kKB ? (BN == 256 ? 3 : 4) : (BN == 256 ? 4 : (BN == 192 ? 5 : 6));
    static constexpr int kStagesFit = (227 * 1024 - 1024 - 256 - kEpiStage) / kStageBytes;
    static constexpr int kStages = kStagesWant < kStagesFit ? kStagesWant : kStagesFit;
    static constexpr int kSmem = 1024 + kStages * kStageBytes + kEpiStage + 256;
    static_assert(kStages >= 2 && kSmem <= 227 * 1024, "split kernel shared memory");
    static constexpr int kThreads = 64 + 32 * kEpiWarps;
    static constexpr int kNBuf = MODE == kModeF64Tmem ? 1 : 2;
    static constexpr int kTmemCols = (MODE == kModeF64Tmem || BN > 128) ? 512 : 256;
    // A/B format fields: BF16 = 1 (kind::f16), E4M3 = 0 (kind::f8f6f4); B is
    // MN-major for BF16, K-major for E4M3.
    static constexpr uint32_t kIdesc =
        FMT == kFmtE4M3 ? make_idesc(0u, kBM, BN, 0u, 0u) : make_idesc(1u, kBM, BN, 0u, 1u);
};

struct SplitArgs {
    void* C;
    int64_t m, n, p;
    int tiles_m, tiles_n, num_kb;
    int group_m;
    int f64;            // 0: FP32-accuracy (one level of 6 pairs); 1: FP64-accuracy levels
    int levels;         // number of levels
    int kc[kMaxLevels]; // chunk length per level, in K blocks
    int S;
    int beta;           // digit radix 2^beta (FP64 mode)
    int drop;           // fixed-point bits dropped from the int64 total (FP64 mode)
    const int* eA;
    const int* eB;
    int vec_ok;
    uint64_t wait_limit_ns;
    int* status;
    // FP64 modes, split K: every tile's K range is cut into `ksplit` slices
    // run as separate work units; their folds add into C atomically (exact
    // int64 adds, order-free), and cnt[tile * epilogue warps + warp] counts
    // the units that have finished a warp's region (zeroed before launch).
    int ksplit;
    // and the levels of a tile into `lgroups` groups (bit L of lmask[g] set:
    // level L belongs to group g), each run as a separate work unit
    int lgroups;
    uint32_t lmask[kMaxLevels];
    int* cnt;
    // split K: levels finer than the total's grid (shift below 0) add their
    // exact sums, scaled to the finest level, into fine[m x p] instead of
    // rounding them into C; the region's last unit rounds them in once.
    long long* fine;
    // FP32-accuracy split K: slice s's partial tile at part[s * m * p + i * p + j]
    float* part;
    // grouped FP32-accuracy launches: the problems (sorted by unit_begin) and
    // their TMA descriptors (A slices, B slices per problem, global memory)
    const struct SplitGProb* probs;
    const CUtensorMap* maps;
    int nprob;
    int num_units;
};

// One problem of a grouped FP32-accuracy split GEMM (device table).
struct SplitGProb {
    float* C;
    int64_t m, p;
    int tiles_m, tiles_n, num_kb, group_m;
    int bn;                 // tile width (the MMA N extent): 128 or 256
    int vec_ok;             // C rows allow 16-byte stores
    int unit_begin, pad;    // first unit (tile) of the problem in the work list
};

// What the roles need about a unit of a grouped launch: the problem and the
// tile (one K slice, every level).
struct SplitGUnit {
    int g, tm, tn, bn, vec_ok;
    int64_t m, p;
    float* C;
};
__device__ __forceinline__ SplitGUnit split_gresolve(const SplitArgs& a, int u) {
    int lo = 0, hi = a.nprob - 1;
    while (lo < hi) {   // last problem with unit_begin <= u
        const int mid = (lo + hi + 1) >> 1;
        if (a.probs[mid].unit_begin <= u) lo = mid; else hi = mid - 1;
    }
    const SplitGProb& pr = a.probs[lo];
    SplitGUnit x;
    x.g = lo;
    const int t = u - pr.unit_begin;
    const int per_group = pr.group_m * pr.tiles_n;
    const int gi = t / per_group;
    const int first_m = gi * pr.group_m;
    const int gsize = min(pr.tiles_m - first_m, pr.group_m);
    const int r = t - gi * per_group;
    x.tm = first_m + r % gsize;
    x.tn = r / gsize;
    x.bn = pr.bn;
    x.vec_ok = pr.vec_ok;
    x.m = pr.m;
    x.p = pr.p;
    x.C = pr.C;
    return x;
}

// Work unit u: tile t and the K blocks [kb_lo, kb_hi) of its K slice (SK:
// the split-K kernel variant; without it every unit is a whole tile).
template <bool SK>
__device__ __forceinline__ void split_unit(const SplitArgs& a, int u, int& t, int& kb_lo,
                                           int& kb_hi, uint32_t& lmask, int* slice = nullptr) {
    if constexpr (!SK) {
        t = u;
        kb_lo = 0;
        kb_hi = a.num_kb;
        lmask = 0xFFFFFFFFu;
        if (slice) *slice = 0;
        return;
    }
    const int ks = a.ksplit;
    const int lg = a.lgroups;
    t = u / (ks * lg);
    const int rem = u - t * (ks * lg);
    const int sl = rem / lg;
    lmask = a.lmask[rem - sl * lg];
    if (slice) *slice = sl;
    kb_lo = static_cast<int>(static_cast<long long>(sl) * a.num_kb / ks);
    kb_hi = static_cast<int>(static_cast<long long>(sl + 1) * a.num_kb / ks);
}

__device__ __forceinline__ void split_tile_coords(int t, int tiles_m, int tiles_n, int group_m,
                                                  int& tm, int& tn) {
    const int per_group = group_m * tiles_n;
    const int g = t / per_group;
    const int first_m = g * group_m;
    const int gsize = min(tiles_m - first_m, group_m);
    const int r = t - g * per_group;
    tm = first_m + r % gsize;
    tn = r / gsize;
}

// Pairs (slice of A, slice of B) of one level.  FP32 mode: the six products
// with t + u <= 2, larger first.  FP64 mode: level L holds (s, L - s).
__device__ __forceinline__ int level_pairs(const SplitArgs& a, int L) {
    return a.f64 ? L + 1 : 6;
}
__device__ __forceinline__ void pair_at(const SplitArgs& a, int L, int q, int& s, int& t) {
    if (a.f64) {
        s = q;
        t = L - q;
    } else {
        // (0,0) (0,1) (1,0) (0,2) (1,1) (2,0), one nibble per pair
        s = (0x210100 >> (4 * q)) & 15;
        t = (0x012010 >> (4 * q)) & 15;
    }
}

// v * 2^sh for sh >= 0; else v / 2^-sh rounded to nearest (ties up): the
// fixed-point alignment of a level sum to the int64 total.
__device__ __forceinline__ long long align_level64(long long x, int sh) {
    return sh >= 0 ? x * (1ll << sh) : (x + (1ll << (-sh - 1))) >> (-sh);
}
__device__ __forceinline__ long long align_level(int v, int sh) {
    return align_level64(static_cast<long long>(v), sh);
}

// Folds a 32 x 16 block of exact level sums into the int64 fixed-point
// totals T kept in C (FP64 modes): T += align_level(R, sh) (T = 0 before the
// tile's first fold, !t_init); with `last` the sum is converted once to FP64,
// scaled by 2^(eA_i + eB_j + ebias) and stored over T.  Lane l holds row l of
// the block in v (16 int32 values).  The block goes through this warp's 2 KB
// staging tile (16-byte chunks XOR-swizzled by row) so that each warp access
// to C moves 16-byte pairs covering 4 rows x 128 contiguous bytes, instead
// of one 8-byte element in each of 32 rows.  row0, col0: the block's origin
// in C (pitch ld elements); rows_left / cols_left: its rows and columns
// inside C; er: the lane's row exponent eA (lane = row); vec: C is 16-byte
// aligned and ld even.
// `atomic` (split K): T += align_level(R, sh) by atomic adds into a C that
// was zeroed before the launch (t_init and last are ignored).
__device__ __forceinline__ void fold_block16(uint8_t* stage, const uint32_t (&v)[16],
                                             long long* C64, int64_t ld, int64_t row0,
                                             int rows_left, int64_t col0, int64_t cols_left,
                                             int sh, bool t_init, bool last, int er,
                                             const int* __restrict__ eB, int ebias, bool vec,
                                             bool atomic) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < 4; ++c)
        *reinterpret_cast<uint4*>(stage + lane * 64 + ((c ^ (lane & 3)) << 4)) =
            make_uint4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
    __syncwarp();
    // lane -> (row in a group of 4, column pair): columns 2 c2, 2 c2 + 1 of
    // rows 4 i + r4, i = 0..7
    const int r4 = lane >> 3, c2 = lane & 7;
    const int64_t col = col0 + 2 * c2;
    const int64_t cl = cols_left - 2 * c2;
    if (atomic) {
#pragma unroll 4
        for (int i = 0; i < 8; ++i) {
            const int rr = 4 * i + r4;
            if (rr >= rows_left || cl <= 0) continue;
            const uint2 sv = *reinterpret_cast<const uint2*>(
                stage + rr * 64 + (((c2 >> 1) ^ (rr & 3)) << 4) + (c2 & 1) * 8);
            auto* dst = reinterpret_cast<unsigned long long*>(C64 + (row0 + rr) * ld + col);
            atomicAdd(dst, static_cast<unsigned long long>(align_level(static_cast<int>(sv.x), sh)));
            if (cl > 1)
                atomicAdd(dst + 1,
                          static_cast<unsigned long long>(align_level(static_cast<int>(sv.y), sh)));
        }
        __syncwarp();
        return;
    }
    int eb0 = 0, eb1 = 0;
    if (last) {
        if (cl > 0) eb0 = eB[col];
        if (cl > 1) eb1 = eB[col + 1];
    }
    const bool pair = vec && cl >= 2;
    constexpr int kBatch = 4;   // row groups whose totals are loaded together
#pragma unroll
    for (int i0 = 0; i0 < 8; i0 += kBatch) {
        long long t0[kBatch], t1[kBatch];
#pragma unroll
        for (int i = 0; i < kBatch; ++i) {
            const int rr = 4 * (i0 + i) + r4;
            t0[i] = 0;
            t1[i] = 0;
            if (t_init && rr < rows_left && cl > 0) {
                const long long* src = C64 + (row0 + rr) * ld + col;
                if (pair) {
                    const longlong2 x = *reinterpret_cast<const longlong2*>(src);
                    t0[i] = x.x;
                    t1[i] = x.y;
                } else {
                    t0[i] = src[0];
                    if (cl > 1) t1[i] = src[1];
                }
            }
        }
#pragma unroll
        for (int i = 0; i < kBatch; ++i) {
            const int rr = 4 * (i0 + i) + r4;
            const int er_r = __shfl_sync(0xffffffffu, er, rr);
            if (rr >= rows_left || cl <= 0) continue;
            const uint2 sv = *reinterpret_cast<const uint2*>(
                stage + rr * 64 + (((c2 >> 1) ^ (rr & 3)) << 4) + (c2 & 1) * 8);
            const long long tot0 = t0[i] + align_level(static_cast<int>(sv.x), sh);
            const long long tot1 = t1[i] + align_level(static_cast<int>(sv.y), sh);
            long long* dst = C64 + (row0 + rr) * ld + col;
            if (last) {
                const double d0 = ldexp(__ll2double_rn(tot0), er_r + eb0 + ebias);
                const double d1 = ldexp(__ll2double_rn(tot1), er_r + eb1 + ebias);
                double* dd = reinterpret_cast<double*>(dst);
                if (pair) {
                    *reinterpret_cast<double2*>(dd) = make_double2(d0, d1);
                } else {
                    dd[0] = d0;
                    if (cl > 1) dd[1] = d1;
                }
            } else {
                if (pair) {
                    *reinterpret_cast<longlong2*>(dst) = make_longlong2(tot0, tot1);
                } else {
                    dst[0] = tot0;
                    if (cl > 1) dst[1] = tot1;
                }
            }
        }
    }
    __syncwarp();   // the staging tile is free for the next block
}

// Split K, last unit of a warp's region: converts the region's int64 totals
// (32 rows x `cols` columns from (row0, col0), every unit's adds complete)
// once to FP64, scaled by 2^(eA_i + eB_j + ebias), in place.  Loads bypass
// L1 (the other units' adds happened in L2).
__device__ __forceinline__ void convert_region(long long* C64, const long long* fine, int drop,
                                               int64_t ld, int64_t row0, int rows_left,
                                               int64_t col0, int64_t cols_left, int cols, int er,
                                               const int* __restrict__ eB, int ebias, bool vec) {
    const int lane = threadIdx.x & 31;
    const int r4 = lane >> 3, c2 = lane & 7;
    for (int b = 0; b < cols; b += 16) {
        const int64_t col = col0 + b + 2 * c2;
        const int64_t cl = cols_left - b - 2 * c2;
        const bool pair = vec && cl >= 2;
        const int eb0 = cl > 0 ? eB[col] : 0;
        const int eb1 = cl > 1 ? eB[col + 1] : 0;
#pragma unroll 4
        for (int i = 0; i < 8; ++i) {
            const int rr = 4 * i + r4;
            const int er_r = __shfl_sync(0xffffffffu, er, rr);
            if (rr >= rows_left || cl <= 0) continue;
            long long* src = C64 + (row0 + rr) * ld + col;
            const long long* fsrc = fine + (row0 + rr) * ld + col;
            long long t0, t1 = 0, f0, f1 = 0;
            if (pair) {
                const longlong2 x = __ldcg(reinterpret_cast<const longlong2*>(src));
                t0 = x.x;
                t1 = x.y;
            } else {
                t0 = __ldcg(src);
                if (cl > 1) t1 = __ldcg(src + 1);
            }
            f0 = __ldcg(fsrc);   // 8-byte aligned only: fine is packed m x p
            if (cl > 1) f1 = __ldcg(fsrc + 1);
            // the fine levels, rounded once onto the total's grid
            t0 += align_level64(f0, -drop);
            t1 += align_level64(f1, -drop);
            const double d0 = ldexp(__ll2double_rn(t0), er_r + eb0 + ebias);
            const double d1 = ldexp(__ll2double_rn(t1), er_r + eb1 + ebias);
            double* dd = reinterpret_cast<double*>(src);
            if (pair) {
                *reinterpret_cast<double2*>(dd) = make_double2(d0, d1);
            } else {
                dd[0] = d0;
                if (cl > 1) dd[1] = d1;
            }
        }
    }
}

// GROUPED (FP32 mode, kb-major stages, no split K only): units are the tiles
// of all problems of args.probs, each with its own TMA descriptors, C and
// tile width (runtime MMA N; narrow tiles leave the last epilogue warps idle).
template <int BN, int MODE, int FMT, bool SK, bool GROUPED = false>
__global__ void __launch_bounds__(SplitCfg<BN, MODE, FMT>::kThreads, 1)
    split_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                      const SplitArgs args) {
    static_assert(!GROUPED || (MODE == kModeF32 && FMT == kFmtBF16KB && !SK),
                  "grouped split launches take FP32-accuracy problems without split K");
    using Cfg = SplitCfg<BN, MODE, FMT>;
    constexpr int kBKe = Cfg::kBKe;
    constexpr bool F64 = MODE != kModeF32;
    constexpr int kNBuf = Cfg::kNBuf;
    constexpr int kStages = Cfg::kStages;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                               ~static_cast<uintptr_t>(1023));
    uint8_t* sA = smem;
    uint8_t* sB = smem + kStages * Cfg::kAStage;
    uint8_t* epi = sB + kStages * Cfg::kBBytes;   // FP64 fold staging, 4 KB per epilogue warp
    uint64_t* bars = reinterpret_cast<uint64_t*>(epi + Cfg::kEpiStage);
    uint64_t* full = bars;
    uint64_t* empty = bars + kStages;
    uint64_t* tfull = bars + 2 * kStages;
    uint64_t* tempty = tfull + 2;
    uint64_t* drain = tempty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    CtaCtl* ctl = reinterpret_cast<CtaCtl*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint64_t limit = args.wait_limit_ns;
    int* status = args.status;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], Cfg::kEpiWarps);
        }
        mbar_init(drain, 1);
        ctl->abort = 0;
        fence_barrier_init();
    }
    if (!GROUPED && warp == 0 && lane == 0) {
        prefetch_tmap(&tmA);
        prefetch_tmap(&tmB);
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, Cfg::kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    const int num_units = GROUPED ? args.num_units
                                  : args.tiles_m * args.tiles_n * (SK ? args.ksplit * args.lgroups : 1);

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer: (tile, level, kb, pair)
            int stage = 0;
            uint32_t phase = 0;
            long issued = 0;
            bool ok = true;
            int g_prev = -1;
            for (int u = blockIdx.x; u < num_units && ok; u += gridDim.x) {
                int t, kb_lo, kb_hi, tm, tn;
                uint32_t lmask;
                int bn = BN;
                const CUtensorMap* mA = &tmA;
                const CUtensorMap* mB = &tmB;
                if constexpr (GROUPED) {
                    const SplitGUnit x = split_gresolve(args, u);
                    tm = x.tm;
                    tn = x.tn;
                    bn = x.bn;
                    kb_lo = 0;
                    kb_hi = args.probs[x.g].num_kb;
                    lmask = 0xFFFFFFFFu;
                    t = 0;
                    mA = args.maps + 2 * x.g;
                    mB = args.maps + 2 * x.g + 1;
                    if (x.g != g_prev) {
                        prefetch_tmap(mA);
                        prefetch_tmap(mB);
                        g_prev = x.g;
                    }
                } else {
                    split_unit<SK>(args, u, t, kb_lo, kb_hi, lmask);
                    split_tile_coords(t, args.tiles_m, args.tiles_n, args.group_m, tm, tn);
                }
                for (int L = 0; L < args.levels && ok; ++L) {
                    if constexpr (SK)
                        if (!((lmask >> L) & 1u)) continue;
                    const int np = level_pairs(args, L);
                    if constexpr (Cfg::kKB) {
                        // kb-major: the three slices of A and of B of K block kb
                        const uint32_t bytes =
                            GROUPED ? 3u * (Cfg::kASlice + static_cast<uint32_t>(bn / 64) * Cfg::kBChunk)
                                    : static_cast<uint32_t>(Cfg::kStageBytes);
                        for (int kb = kb_lo; kb < kb_hi && ok; ++kb) {
                            if (!mbar_wait(&empty[stage], phase ^ 1u, ctl, limit, status)) {
                                ok = false;
                                break;
                            }
                            mbar_arrive_expect_tx(&full[stage], bytes);
                            uint8_t* a_st = sA + stage * Cfg::kAStage;
                            uint8_t* b_st = sB + stage * Cfg::kBBytes;
#pragma unroll
                            for (int sl = 0; sl < 3; ++sl) {
                                tma_load_3d(a_st + sl * Cfg::kASlice, mA, &full[stage],
                                            kb * kBKe, tm * kBM, sl);
#pragma unroll
                                for (int c = 0; c < BN / 64; ++c)
                                    if (!GROUPED || c < bn / 64)
                                        tma_load_3d(b_st + sl * Cfg::kBSlice + c * Cfg::kBChunk, mB,
                                                    &full[stage], tn * bn + c * 64, kb * kBKe, sl);
                            }
                            ++issued;
                            if (++stage == kStages) {
                                stage = 0;
                                phase ^= 1u;
                            }
                        }
                    } else {
                    for (int kb = kb_lo; kb < kb_hi && ok; ++kb) {
                        for (int q = 0; q < np; ++q) {
                            int s, u;
                            pair_at(args, L, q, s, u);
                            if (!mbar_wait(&empty[stage], phase ^ 1u, ctl, limit, status)) {
                                ok = false;
                                break;
                            }
                            mbar_arrive_expect_tx(&full[stage], Cfg::kStageBytes);
                            tma_load_3d(sA + stage * Cfg::kAStage, &tmA, &full[stage], kb * kBKe,
                                        tm * kBM, s);
                            if constexpr (FMT == kFmtE4M3) {
                                // B^T plane u: BN rows (j) x 128 bytes (k)
                                tma_load_3d(sB + stage * Cfg::kBBytes, &tmB, &full[stage],
                                            kb * kBKe, tn * BN, u);
                            } else {
#pragma unroll
                                for (int c = 0; c < BN / 64; ++c)
                                    tma_load_3d(sB + stage * Cfg::kBBytes + c * Cfg::kBChunk, &tmB,
                                                &full[stage], tn * BN + c * 64, kb * kBKe, u);
                            }
                            ++issued;
                            if (++stage == kStages) {
                                stage = 0;
                                phase ^= 1u;
                            }
                        }
                    }
                    }   // kb-major or one pair per stage
                }
            }
            if (!ok) {
                // Let the loads already in flight land before the CTA exits.
                CtaCtl local{0};
                const long outstanding = issued < kStages ? issued : kStages;
                for (long q = 1; q <= outstanding; ++q) {
                    const long idx = issued - q;
                    mbar_wait(&full[idx % kStages], static_cast<uint32_t>((idx / kStages) & 1),
                              &local, limit, status);
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer: one TMEM chunk accumulator per chunk
            int stage = 0;
            uint32_t phase = 0;
            long cnt = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < num_units && ok; u += gridDim.x) {
                int t, kb_lo, kb_hi;
                uint32_t lmask;
                uint32_t idesc = Cfg::kIdesc;
                if constexpr (GROUPED) {
                    const SplitGUnit x = split_gresolve(args, u);
                    kb_lo = 0;
                    kb_hi = args.probs[x.g].num_kb;
                    lmask = 0xFFFFFFFFu;
                    t = 0;
                    idesc = make_idesc(1u, kBM, static_cast<uint32_t>(x.bn), 0u, 1u);
                } else {
                    split_unit<SK>(args, u, t, kb_lo, kb_hi, lmask);
                }
                (void)t;
                for (int L = 0; L < args.levels && ok; ++L) {
                    if constexpr (SK)
                        if (!((lmask >> L) & 1u)) continue;
                    const int np = level_pairs(args, L);
                    const int kc = args.kc[L];
                    for (int kb0 = kb_lo; kb0 < kb_hi && ok; kb0 += kc, ++cnt) {
                        const int buf = static_cast<int>(cnt % kNBuf);
                        const uint32_t bph = static_cast<uint32_t>((cnt / kNBuf) & 1);
                        if (!mbar_wait(&tempty[buf], bph ^ 1u, ctl, limit, status)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t d = tmem_base + static_cast<uint32_t>(buf * BN);
                        const int kb1 = min(kb_hi, kb0 + kc);
                        bool first = true;
                        for (int kb = kb0; kb < kb1 && ok; ++kb) {
                            if constexpr (Cfg::kKB) {
                                // the six slice products of K block kb from one stage
                                if (!mbar_wait(&full[stage], phase, ctl, limit, status)) {
                                    ok = false;
                                    break;
                                }
                                tc_fence_after();
                                const uint8_t* a_st = sA + stage * Cfg::kAStage;
                                const uint8_t* b_st = sB + stage * Cfg::kBBytes;
#pragma unroll
                                for (int q = 0; q < 6; ++q) {
                                    int sl, u;
                                    pair_at(args, 0, q, sl, u);
                                    const uint64_t adesc = smem_desc_sw64(
                                        smem_u32(a_st + sl * Cfg::kASlice), 16, 512);
                                    const uint64_t bdesc = smem_desc_sw128(
                                        smem_u32(b_st + u * Cfg::kBSlice), Cfg::kBChunk, 1024);
#pragma unroll
                                    for (int k = 0; k < kBKe / 16; ++k)
                                        mma_f16(d, adesc + static_cast<uint64_t>((k * 32) >> 4),
                                                bdesc + static_cast<uint64_t>((k * 16 * 128) >> 4),
                                                idesc, (first && q == 0 && k == 0) ? 0u : 1u);
                                }
                                first = false;
                                mma_commit(&empty[stage]);
                                if (++stage == kStages) {
                                    stage = 0;
                                    phase ^= 1u;
                                }
                            } else {
                            for (int q = 0; q < np; ++q) {
                                if (!mbar_wait(&full[stage], phase, ctl, limit, status)) {
                                    ok = false;
                                    break;
                                }
                                tc_fence_after();
                                const uint64_t adesc =
                                    smem_desc_sw128(smem_u32(sA + stage * Cfg::kAStage), 16, 1024);
                                const uint64_t bdesc = smem_desc_sw128(
                                    smem_u32(sB + stage * Cfg::kBBytes),
                                    FMT == kFmtE4M3 ? 16 : Cfg::kBChunk, 1024);
                                // four MMAs of 32 bytes of K each
#pragma unroll
                                for (int k = 0; k < 4; ++k) {
                                    const uint64_t a_off = static_cast<uint64_t>((k * 32) >> 4);
                                    if constexpr (FMT == kFmtE4M3)
                                        mma_f8f6f4(d, adesc + a_off, bdesc + a_off, Cfg::kIdesc,
                                                   (first && k == 0) ? 0u : 1u);
                                    else
                                        mma_f16(d, adesc + a_off,
                                                bdesc + static_cast<uint64_t>((k * 16 * 128) >> 4),
                                                Cfg::kIdesc, (first && k == 0) ? 0u : 1u);
                                }
                                first = false;
                                mma_commit(&empty[stage]);
                                if (++stage == kStages) {
                                    stage = 0;
                                    phase ^= 1u;
                                }
                            }
                            }   // kb-major or one pair per stage
                        }
                        if (!ok) break;
                        mma_commit(&tfull[buf]);
                    }
                }
            }
            // Every MMA issued above must finish before TMEM is released.
            mma_commit(drain);
            CtaCtl local{0};
            mbar_wait(drain, 0, &local, limit, status);
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: quadrant q = warp % 4, column group h
        constexpr int kCols = Cfg::kColsPerWarp;
        const int q = warp & 3;
        const int h = (warp - 2) >> 2;
        const uint32_t lane_base = static_cast<uint32_t>(q * 32) << 16;
        uint8_t* epi_stage = epi + (F64 ? (warp - 2) * Cfg::kEpiStageWarp : 0);
        long cnt = 0;
        bool ok = true;
        constexpr bool atomic = SK;
        for (int u = blockIdx.x; u < num_units && ok; u += gridDim.x) {
            int t, kb_lo, kb_hi, tm, tn, kslice;
            uint32_t lmask;
            // the unit's problem: its C, sizes and tile width
            int64_t um = args.m, up = args.p;
            float* uC = static_cast<float*>(args.C);
            int uvec = args.vec_ok, bn = BN;
            if constexpr (GROUPED) {
                const SplitGUnit x = split_gresolve(args, u);
                tm = x.tm;
                tn = x.tn;
                kb_lo = 0;
                kb_hi = args.probs[x.g].num_kb;
                lmask = 0xFFFFFFFFu;
                kslice = 0;
                t = 0;
                um = x.m;
                up = x.p;
                uC = x.C;
                uvec = x.vec_ok;
                bn = x.bn;
            } else {
                split_unit<SK>(args, u, t, kb_lo, kb_hi, lmask, &kslice);
                split_tile_coords(t, args.tiles_m, args.tiles_n, args.group_m, tm, tn);
            }
            // narrow tiles of a grouped launch leave the last column warps idle
            const bool cols_live = !GROUPED || h * kCols < bn;
            // the unit's last level (its folds end there)
            const int l_last =
                SK ? 31 - __clz(static_cast<int>(lmask & ((1u << args.levels) - 1u)))
                   : args.levels - 1;
            const int64_t row = static_cast<int64_t>(tm) * kBM + q * 32 + lane;
            const int64_t col_base = static_cast<int64_t>(tn) * bn + h * kCols;
            const bool row_ok = row < um;
            // FP64 modes keep the tile's int64 fixed-point total T in C itself
            // (same 8 bytes per element as the final FP64 value).
            const int er = (F64 && row_ok) ? args.eA[row] : 0;
            bool t_init = false;
            // Register running sums (kModeF32, kModeF64Reg): FP32 bits or the
            // exact int32 sum of the current level; 0 is zero in both.
            constexpr int kRegs = MODE == kModeF64Tmem ? 1 : 64;
            uint32_t acc[kRegs];
#pragma unroll
            for (int i = 0; i < kRegs; ++i) acc[i] = 0u;
            const uint32_t r_base = tmem_base + lane_base + 256u + static_cast<uint32_t>(h * kCols);
            bool r_valid = false;   // kModeF64Tmem: TMEM level sums hold data
            for (int L = 0; L < args.levels && ok; ++L) {
                if constexpr (SK)
                    if (!((lmask >> L) & 1u)) continue;
                const int kc = args.kc[L];
                int since_fold = 0;
                for (int kb0 = kb_lo; kb0 < kb_hi; kb0 += kc, ++cnt) {
                    const int buf = static_cast<int>(cnt % kNBuf);
                    const uint32_t bph = static_cast<uint32_t>((cnt / kNBuf) & 1);
                    ok = mbar_wait(&tfull[buf], bph, ctl, limit, status);
                    if (!__all_sync(0xffffffffu, ok)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a_base = tmem_base + lane_base +
                                            static_cast<uint32_t>(buf * BN + h * kCols);
                    if constexpr (MODE == kModeF64Tmem) {
#pragma unroll 2
                        for (int g = 0; g < kCols / 16; ++g) {
                            uint32_t a16[16], r16[16];
                            tmem_ld16(a_base + 16u * g, a16);
                            if (r_valid) tmem_ld16(r_base + 16u * g, r16);
                            tmem_ld_wait();
#pragma unroll
                            for (int i = 0; i < 16; ++i)
                                r16[i] = static_cast<uint32_t>(
                                    (r_valid ? static_cast<int>(r16[i]) : 0) +
                                    __float2int_rn(__uint_as_float(a16[i])));
                            tmem_st16(r_base + 16u * g, r16);
                        }
                        tmem_st_wait();
                        r_valid = true;
                    } else if (cols_live) {
#pragma unroll
                        for (int g = 0; g < 4; ++g) {
                            uint32_t r[16];
                            tmem_ld16(a_base + 16u * g, r);
                            tmem_ld_wait();
                            if constexpr (F64) {
#pragma unroll
                                for (int i = 0; i < 16; ++i)
                                    acc[g * 16 + i] = static_cast<uint32_t>(
                                        static_cast<int>(acc[g * 16 + i]) +
                                        __float2int_rn(__uint_as_float(r[i])));
                            } else {
#pragma unroll
                                for (int i = 0; i < 16; ++i)
                                    acc[g * 16 + i] = __float_as_uint(
                                        __uint_as_float(acc[g * 16 + i]) + __uint_as_float(r[i]));
                            }
                        }
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&tempty[buf]);
                    ++since_fold;
                    const bool level_end = kb0 + kc >= kb_hi;
                    if (F64 && (level_end || since_fold == 64)) {
                        // fold the level's exact sum into the int64 total:
                        // T += round(R * 2^(beta(S-1-L) - drop)); the last fold
                        // of the tile converts once to FP64 and scales by
                        // 2^(eA_i + eB_j - beta(S+1) + drop).
                        const int sh = args.beta * (args.S - 1 - L) - args.drop;
                        const bool last = level_end && L == l_last;
                        const int64_t row0 = static_cast<int64_t>(tm) * kBM + q * 32;
                        const int64_t rl = args.m - row0;
                        const int rows_left = rl < 0 ? 0 : (rl > 32 ? 32 : static_cast<int>(rl));
#pragma unroll
                        for (int b = 0; b < kCols / 16; ++b) {
                            uint32_t rv[16];
                            if constexpr (MODE == kModeF64Tmem) {
                                tmem_ld16(r_base + 16u * b, rv);
                                tmem_ld_wait();
                            } else {
#pragma unroll
                                for (int i = 0; i < 16; ++i) rv[i] = acc[(b * 16 + i) % kRegs];
                            }
                            const int64_t c0 = col_base + b * 16;
                            // split K: a level finer than the total's grid goes,
                            // exact, into the fine-level sums
                            const bool to_fine = atomic && sh < 0;
                            fold_block16(epi_stage, rv,
                                         to_fine ? args.fine
                                                 : reinterpret_cast<long long*>(args.C),
                                         args.p, row0, rows_left, c0, args.p - c0,
                                         to_fine ? sh + args.drop : sh, t_init, last, er,
                                         args.eB, args.drop - args.beta * (args.S + 1),
                                         args.vec_ok != 0 && !to_fine, atomic);
                        }
                        if (atomic && last) {
                            // this unit's adds to the warp's region are done;
                            // the region's last unit converts it to FP64
                            __threadfence();
                            __syncwarp();
                            int old = 0;
                            if (lane == 0)
                                old = atomicAdd(&args.cnt[static_cast<int64_t>(t) * Cfg::kEpiWarps +
                                                          (warp - 2)],
                                                1);
                            old = __shfl_sync(0xffffffffu, old, 0);
                            if (old == args.ksplit * args.lgroups - 1) {
                                __threadfence();
                                const int64_t left = args.p - col_base;
                                convert_region(reinterpret_cast<long long*>(args.C), args.fine,
                                               args.drop, args.p, row0, rows_left, col_base,
                                               left, kCols, er, args.eB,
                                               args.drop - args.beta * (args.S + 1),
                                               args.vec_ok != 0);
                            }
                        }
                        t_init = true;
                        r_valid = false;
#pragma unroll
                        for (int i = 0; i < kRegs; ++i) acc[i] = 0u;
                        since_fold = 0;
                    }
                }
            }
            if (!ok) break;
            // ---------------- FP32 mode, split K: this unit's partial tile goes to
            // the workspace; the last unit of the warp's region sums the slices
            // in slice order (deterministic) into C
            if constexpr (!F64 && SK) {
                const int64_t plane = args.m * args.p;
                if (row_ok) {   // the lane's row of the partial tile
                    float* prow = args.part + kslice * plane + row * args.p;
                    if (args.vec_ok && col_base + 64 <= args.p) {
                        float4* dst = reinterpret_cast<float4*>(prow + col_base);
#pragma unroll
                        for (int v = 0; v < 16; ++v)
                            dst[v] = make_float4(__uint_as_float(acc[4 * v]),
                                                 __uint_as_float(acc[4 * v + 1]),
                                                 __uint_as_float(acc[4 * v + 2]),
                                                 __uint_as_float(acc[4 * v + 3]));
                    } else {
#pragma unroll
                        for (int i = 0; i < 64; ++i)
                            if (col_base + i < args.p) prow[col_base + i] = __uint_as_float(acc[i]);
                    }
                }
                __threadfence();
                __syncwarp();
                int old = 0;
                if (lane == 0)
                    old = atomicAdd(&args.cnt[static_cast<int64_t>(t) * Cfg::kEpiWarps + (warp - 2)], 1);
                old = __shfl_sync(0xffffffffu, old, 0);
                if (old == args.ksplit - 1) {
                    // the region's 32 rows x 64 columns, lanes along the columns
                    // (coalesced), the slices summed in order
                    __threadfence();
                    const int64_t row0 = static_cast<int64_t>(tm) * kBM + q * 32;
#pragma unroll 4
                    for (int r = 0; r < 32; ++r) {
                        const int64_t grow = row0 + r;
                        if (grow >= args.m) break;
#pragma unroll
                        for (int hc = 0; hc < 2; ++hc) {
                            const int64_t col = col_base + hc * 32 + lane;
                            if (col >= args.p) continue;
                            const float* src = args.part + grow * args.p + col;
                            float sum = 0.f;
                            for (int s2 = 0; s2 < args.ksplit; ++s2) sum += __ldcg(src + s2 * plane);
                            static_cast<float*>(args.C)[grow * args.p + col] = sum;
                        }
                    }
                }
                continue;
            }
            // ---------------- FP32 mode: store the tile
            if (!F64 && row_ok && cols_live) {
                float* crow = uC + row * up;
                if (uvec && col_base + 64 <= up) {
                    float4* dst = reinterpret_cast<float4*>(crow + col_base);
#pragma unroll
                    for (int v = 0; v < 16; ++v)
                        dst[v] = make_float4(__uint_as_float(acc[(4 * v) % kRegs]),
                                             __uint_as_float(acc[(4 * v + 1) % kRegs]),
                                             __uint_as_float(acc[(4 * v + 2) % kRegs]),
                                             __uint_as_float(acc[(4 * v + 3) % kRegs]));
                } else {
#pragma unroll
                    for (int i = 0; i < 64; ++i)
                        if (col_base + i < up) crow[col_base + i] = __uint_as_float(acc[i % kRegs]);
                }
            }
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, Cfg::kTmemCols);
    }
}

}  // namespace

// ====================================================================== host side
// FP32-accuracy chunk length in K blocks of `bk` elements
// (MOA_F32_SPLIT_CHUNK_K elements, default 256).
static int f32_split_chunk_kb(int bk) {
    static long k = 0;
    if (k == 0) {
        const char* env = std::getenv("MOA_F32_SPLIT_CHUNK_K");
        k = env ? std::strtol(env, nullptr, 10) : 256;
        if (k < 1) k = 256;
    }
    return static_cast<int>(std::max<long>(1, (k + bk - 1) / bk));
}

int split_slices(moa_dtype dt, int slices) {
    if (dt == MOA_F32_SPLIT) return (slices == 0 || slices == 3) ? 3 : -1;
    if (is_e4m3_split(dt)) {
        if (slices == 0) return kDefaultSlicesE4M3;
        return (slices < kMinSlicesE4M3 || slices > kMaxSlicesE4M3) ? -1 : slices;
    }
    if (slices == 0) return kDefaultSlices;
    if (slices < kMinSlices || slices > kMaxSlices) return -1;
    return slices;
}

SplitLayout split_layout(int64_t m, int64_t n, int64_t p, moa_dtype dt, int S) {
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    SplitLayout L{};
    L.S = S;
    L.esize = is_e4m3_split(dt) ? 1 : 2;
    L.b_trans = is_e4m3_split(dt);
    // row pitches: multiples of 16 bytes (TMA strides)
    L.lda = round_up(n, 16 / L.esize);
    L.ldb = L.b_trans ? round_up(n, 16) : round_up(p, 8);
    const int64_t b_rows = L.b_trans ? p : n;
    size_t off = 0;
    L.a_off = off;
    off += al(static_cast<size_t>(S) * m * L.lda * L.esize);
    L.b_off = off;
    off += al(static_cast<size_t>(S) * b_rows * L.ldb * L.esize);
    if (dt == MOA_F32_SPLIT) {
        // split K for few tiles (at most 160 SMs' worth of units of 128 x 256)
        const int64_t tiles256 = ceil_div(m, kBM) * ceil_div(p, 256);
        const int64_t by_k = std::max<int64_t>(1, ceil_div(n, 32) * 32 / 1024);
        const int64_t ks = std::min<int64_t>({160 / std::max<int64_t>(1, tiles256), by_k, 64});
        if (ks >= 2) {
            L.f32_ks = static_cast<int>(ks);
            L.cnt_bytes = static_cast<size_t>(ceil_div(m, kBM) * ceil_div(p, 128)) * 16 * 4;
            L.cnt_off = off;
            off += al(L.cnt_bytes);
            L.part_bytes = static_cast<size_t>(ks) * m * p * 4;
            L.part_off = off;
            off += al(L.part_bytes);
        }
    }
    if (dt != MOA_F32_SPLIT) {
        L.ea_off = off;
        off += al(static_cast<size_t>(m) * 4);
        L.eb_off = off;
        off += al(static_cast<size_t>(p) * 4);
        L.cmax_off = off;
        off += al(static_cast<size_t>(p) * 8);
        // split K (few tiles only): counters for at most ceil(m/128) x
        // ceil(p/128) tiles of 16 epilogue warps, and the fine-level sums
        const int64_t tiles128 = ceil_div(m, kBM) * ceil_div(p, 128);
        if (tiles128 <= kSplitKMaxTiles) {
            L.cnt_bytes = static_cast<size_t>(tiles128) * 16 * 4;
            L.cnt_off = off;
            off += al(L.cnt_bytes);
            L.fine_bytes = static_cast<size_t>(m) * p * 8;
            L.fine_off = off;
            off += al(L.fine_bytes);
        }
    }
    L.total = off;
    return L;
}

size_t split_workspace_bytes(int64_t m, int64_t n, int64_t p, moa_dtype dt, int slices) {
    const int S = split_slices(dt, slices);
    if (S < 0) return 0;
    return split_layout(m, n, p, dt, S).total;
}

template <int BN, int MODE, int FMT, bool SK = false, bool GROUPED = false>
static int launch_split_cfg(const SplitArgs& a, const CUtensorMap& tmA, const CUtensorMap& tmB,
                            cudaStream_t s, moa_stats* st) {
    using Cfg = SplitCfg<BN, MODE, FMT>;
    static std::atomic<uint64_t> attr_done{0};   // per instantiation, per device
    {
        const int rc = smem_attr_once(
            reinterpret_cast<const void*>(split_gemm_kernel<BN, MODE, FMT, SK, GROUPED>),
            Cfg::kSmem, attr_done, "cudaFuncSetAttribute(split_gemm)");
        if (rc != MOA_OK) return rc;
    }
    const long tiles = GROUPED ? a.num_units : static_cast<long>(a.tiles_m) * a.tiles_n;
    const int grid =
        static_cast<int>(std::min<long>(tiles * (SK ? a.ksplit * a.lgroups : 1), num_sms()));
    prof_begin(s);
    split_gemm_kernel<BN, MODE, FMT, SK, GROUPED><<<grid, Cfg::kThreads, Cfg::kSmem, s>>>(tmA, tmB,
                                                                                         a);
    cudaError_t e = cudaGetLastError();
    prof_end(s);
    if (e != cudaSuccess) return cuda_fail(e, "split_gemm_kernel launch");
    log_msg(2, "split mode %d fmt %d m=%lld n=%lld p=%lld tile %dx%d levels %d K slices %d "
            "level groups %d grid %d tiles %ld", MODE, FMT, static_cast<long long>(a.m),
            static_cast<long long>(a.n), static_cast<long long>(a.p), kBM, BN, a.levels,
            SK ? a.ksplit : 1, SK ? a.lgroups : 1, grid, tiles);
    if (st) {
        st->block_m = kBM;
        st->block_n = BN;
        st->block_k = Cfg::kBKe;
        st->grid = grid;
        st->tiles = tiles;
    }
    return MOA_OK;
}

// Tile width of the slice GEMM by a wave-count cost model: each width costs
// ceil(tiles / SMs) waves of (width / its relative efficiency), measured on
// the B300 for the split kernels (FP32 accuracy: 128 at 0.8 of 256; FP64
// accuracy: 192 at 0.97, 128 at 0.9); the cheapest wins, the wider on a
// tie.  moa_set_block_n(128 | 192 | 256) forces it (192: FP64 accuracy only).
static int split_block_n(int64_t m, int64_t p, bool f64) {
    const int ov = tile_override();
    if (ov == 128 || ov == 256 || (ov == 192 && f64)) return ov;
    const long sms = num_sms();
    auto cost = [&](int bn, double eff) {
        const long tiles = ceil_div(m, kBM) * ceil_div(p, bn);
        return static_cast<double>((tiles + sms - 1) / sms) * bn / eff;
    };
    int best = 256;
    double c = cost(256, 1.0);
    if (f64) {
        const double c192 = cost(192, 0.97);
        if (c192 < c) {
            best = 192;
            c = c192;
        }
    }
    if (cost(128, f64 ? 0.9 : 0.8) < c) best = 128;
    return best;
}

// K slices per tile of the FP64-accuracy slice GEMM: when the tiles fill at
// most half of the SMs, each tile's K range is cut so that the work units
// (tiles x slices) fill them, keeping at least 1024 K elements per unit
// (every unit folds each level into C once).  MOA_SPLIT_K forces a factor.
static int split_k_factor(long tiles, int num_kb, int bk) {
    static long env = -1;
    if (env < 0) {
        const char* e = std::getenv("MOA_SPLIT_K");
        env = e ? std::max(0L, std::strtol(e, nullptr, 10)) : 0;
    }
    long ks = 1;
    if (env > 0) {
        ks = env;
    } else {
        const long sms = num_sms();
        if (tiles * 2 <= sms) ks = std::min(sms / tiles, static_cast<long>(num_kb) * bk / 1024);
    }
    return static_cast<int>(std::max(1L, std::min({ks, static_cast<long>(num_kb), 64L})));
}

// Level groups of the FP64-accuracy slice GEMM: when the (tile, K slice)
// units still fill at most half of the SMs, the S levels of a tile (level L
// holds L + 1 slice products) are dealt longest first onto up to S groups,
// each a separate work unit, so that the units fill the SMs.  Returns the
// group count and sets mask[g] (bit L: level L in group g).
static int split_level_groups(long units, int S, uint32_t* mask) {
    const long sms = num_sms();
    int G = 1;
    if (units * 2 <= sms) G = static_cast<int>(std::min<long>(S, sms / units));
    if (G <= 1) {
        mask[0] = 0xFFFFFFFFu;
        return 1;
    }
    int load[kMaxLevels] = {0};
    for (int g = 0; g < G; ++g) mask[g] = 0;
    for (int L = S - 1; L >= 0; --L) {   // largest level (L + 1 products) first
        int best = 0;
        for (int g = 1; g < G; ++g)
            if (load[g] < load[best]) best = g;
        load[best] += L + 1;
        mask[best] |= 1u << L;
    }
    return G;
}

// Exponent and digit pre-passes of the FP64-accuracy modes for input type T.
template <typename T>
static void digit_prepasses(const SplitLayout& L, int64_t m, int64_t n, int64_t p, const T* A,
                            const T* B, int beta, int headroom, int* eA, int* eB, void* cmax,
                            uint8_t* a_sl, uint8_t* b_sl, int* status, cudaStream_t s,
                            void* zero_c, void* zero_cnt) {
    using U = typename Bits<T>::U;
    constexpr int per16 = 16 / sizeof(T);
    const int S = L.S;
    // launch 1: row exponents of A (one warp per row) beside the column
    // maxima of B (256 columns x 256 rows per block)
    const int rows_per_block = 8;   // 8 warps of 32 threads
    const int64_t rblocks = std::min<int64_t>(ceil_div(m, rows_per_block), 16L * num_sms());
    const int64_t chunk = 256;
    const int64_t gx = ceil_div(p, 256);
    const int64_t cblocks = gx * ceil_div(n, chunk);
    // split K: C (int64 totals, m x p) and the unit counters start at zero
    const int64_t n0 = zero_c ? m * p : 0;
    // (the counters and the fine-level sums are adjacent in the workspace)
    const int64_t n1 =
        zero_c ? static_cast<int64_t>((L.fine_off - L.cnt_off + L.fine_bytes) / 8) : 0;
    const int64_t zblocks = zero_c ? std::min<int64_t>(ceil_div(n0 + n1, 256 * 8), 4L * num_sms()) : 0;
    exps_kernel<T><<<static_cast<unsigned>(rblocks + cblocks + zblocks), 256, 0, s>>>(
        A, m, n, B, p, chunk, headroom, eA, static_cast<U*>(cmax), status,
        static_cast<int>(rblocks), gx, static_cast<int>(cblocks),
        static_cast<unsigned long long*>(zero_c), n0, static_cast<unsigned long long*>(zero_cnt),
        n1);
    // launch 2: digit planes of A and of B (B's column exponents formed there)
    const int64_t a_plane = m * L.lda;
    const U* cm = static_cast<const U*>(cmax);
    if (L.esize == 1) {
        const int64_t b_plane = p * L.ldb;
        const int ga = grid_for(a_plane / 16, 256);
        const int64_t tiles = ceil_div(n, kTT) * ceil_div(p, kTT);
        const int gb = static_cast<int>(std::min<int64_t>(tiles, 8L * num_sms()));
        digits_e4m3_pair_kernel<T><<<ga + gb, 256, 0, s>>>(
            A, m, n, L.lda, vec_rows(A, n, per16), eA, B, p, L.ldb, eB, cm, headroom, status, S,
            beta, a_sl, a_plane, b_sl, b_plane, ga);
    } else {
        const int64_t b_plane = n * L.ldb;
        const int ga = grid_for(a_plane / 8, 256);
        const int gb = grid_for(b_plane / 8, 256);
        digits_pair_kernel<T><<<ga + gb, 256, 0, s>>>(
            A, m, n, L.lda, vec_rows(A, n, per16), eA, B, p, L.ldb, vec_rows(B, p, per16), eB, cm,
            headroom, status, S, reinterpret_cast<__nv_bfloat16*>(a_sl), a_plane,
            reinterpret_cast<__nv_bfloat16*>(b_sl), b_plane, ga);
    }
}

// K slices of an FP32-accuracy split GEMM of tile width bn (1: no split K),
// as split_gemm plans it.
static int f32_split_ks(const SplitLayout& L, int64_t m, int64_t n, int64_t p, int bn) {
    const int bke = block_k<kFmtBF16KB>();
    if (L.f32_ks < 2) return 1;
    const long tiles = static_cast<long>(ceil_div(m, kBM)) * ceil_div(p, bn);
    return std::min(L.f32_ks, split_k_factor(tiles, static_cast<int>(ceil_div(n, bke)), bke));
}

int split_gemm(int64_t m, int64_t n, int64_t p, moa_dtype dt, const void* A, const void* B,
               void* C, int slices, void* ws, size_t ws_bytes, cudaStream_t s, moa_stats* st) {
    const int S = split_slices(dt, slices);
    if (S < 0) return fail(MOA_ERR_DTYPE, "slice count not supported for this mode");
    const SplitLayout L = split_layout(m, n, p, dt, S);
    if (ws_bytes < L.total) return fail(MOA_ERR_WORKSPACE, "workspace too small for split mode");
    int* status = launch_status_ptr();
    if (!status) return MOA_ERR_CUDA;
    const bool e4m3 = is_e4m3_split(dt);
    const int bke = e4m3 ? block_k<kFmtE4M3>()
                         : (dt == MOA_F32_SPLIT ? block_k<kFmtBF16KB>() : block_k<kFmtBF16>());
    uint8_t* base = static_cast<uint8_t*>(ws);
    uint8_t* a_sl = base + L.a_off;
    uint8_t* b_sl = base + L.b_off;
    const int64_t a_plane = m * L.lda;
    const int64_t b_plane = (L.b_trans ? p : n) * L.ldb;
    int kernels = 0;

    SplitArgs a{};
    a.C = C;
    a.m = m;
    a.n = n;
    a.p = p;
    const int bn = split_block_n(m, p, dt != MOA_F32_SPLIT);
    a.tiles_m = static_cast<int>(ceil_div(m, kBM));
    a.tiles_n = static_cast<int>(ceil_div(p, bn));
    a.num_kb = static_cast<int>(ceil_div(n, bke));
    a.group_m = split_raster_group(n);
    a.S = S;
    a.wait_limit_ns = wait_limit_ns();
    a.status = status;
    a.vec_ok = (p % 4 == 0) && (reinterpret_cast<uintptr_t>(C) % 16 == 0);
    if (dt == MOA_F32_SPLIT)
        a.ksplit = f32_split_ks(L, m, n, p, bn);
    else
        a.ksplit = L.fine_bytes == 0
                       ? 1
                       : split_k_factor(static_cast<long>(a.tiles_m) * a.tiles_n, a.num_kb, bke);
    a.lgroups = 1;
    a.lmask[0] = 0xFFFFFFFFu;
    if (dt != MOA_F32_SPLIT && L.fine_bytes > 0)
        a.lgroups = split_level_groups(static_cast<long>(a.tiles_m) * a.tiles_n * a.ksplit, S,
                                       a.lmask);
    const bool split_units = a.ksplit > 1 || a.lgroups > 1;
    a.cnt = split_units ? reinterpret_cast<int*>(base + L.cnt_off) : nullptr;
    a.fine = (split_units && dt != MOA_F32_SPLIT) ? reinterpret_cast<long long*>(base + L.fine_off)
                                                   : nullptr;
    a.part = (split_units && dt == MOA_F32_SPLIT) ? reinterpret_cast<float*>(base + L.part_off)
                                                   : nullptr;

    if (dt == MOA_F32_SPLIT) {
        auto* a16 = reinterpret_cast<__nv_bfloat16*>(a_sl);
        auto* b16 = reinterpret_cast<__nv_bfloat16*>(b_sl);
        const int ga = grid_for(a_plane / 8, 256);
        split3_pair_kernel<<<ga + grid_for(b_plane / 8, 256), 256, 0, s>>>(
            static_cast<const float*>(A), m, n, L.lda, a16, a_plane, vec_rows(A, n, 4),
            static_cast<const float*>(B), p, L.ldb, b16, b_plane, vec_rows(B, p, 4), status, ga);
        kernels += 1;
        if (split_units) {
            cudaError_t e = cudaMemsetAsync(a.cnt, 0, L.cnt_bytes, s);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(split-K counters)");
        }
        a.f64 = 0;
        a.levels = 1;
        a.beta = 0;
        // Flush the FP32 TMEM accumulator into the epilogue's FP32 running sum
        // every kc K blocks: shorter chunks bound the accumulation error of
        // the tensor core's FP32 adds (MOA_F32_SPLIT_CHUNK_K, default 256).
        a.kc[0] = f32_split_chunk_kb(bke);
        a.drop = 0;
    } else {
        int* eA = reinterpret_cast<int*>(base + L.ea_off);
        int* eB = reinterpret_cast<int*>(base + L.eb_off);
        void* cmax = base + L.cmax_off;
        const int beta = e4m3 ? kBetaE4M3 : kBeta;
        const int h = e4m3 ? kHeadroomE4M3 : kHeadroomBF16;
        if (ceil_div(n, 256) * ceil_div(p, 256) > (1L << 30))
            return fail(MOA_ERR_ARG, "n x p too large for the column-max grid");
        cudaError_t e = cudaMemsetAsync(cmax, 0, static_cast<size_t>(p) * 8, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(colmax)");
        if (dt == MOA_F64_SPLIT_F64IN || dt == MOA_F64_SPLIT_F64IN_E4M3)
            digit_prepasses<double>(L, m, n, p, static_cast<const double*>(A),
                                    static_cast<const double*>(B), beta, h, eA, eB, cmax, a_sl,
                                    b_sl, status, s, split_units ? C : nullptr, a.cnt);
        else
            digit_prepasses<float>(L, m, n, p, static_cast<const float*>(A),
                                   static_cast<const float*>(B), beta, h, eA, eB, cmax, a_sl, b_sl,
                                   status, s, split_units ? C : nullptr, a.cnt);
        kernels += 2;   // the exponent pass and the digit pass (the column-max clear is a memset)
        a.f64 = 1;
        a.levels = S;
        a.beta = beta;
        a.eA = eA;
        a.eB = eB;
        // Chunk lengths: every FP32 partial sum of a level must stay an
        // integer of magnitude <= 2^24.  With |d_0| <= 2^(beta-h) and
        // |d_s| <= 2^(beta-1), per k level 0 adds at most 2^(2(beta-h)) and
        // level L >= 1 at most 2 * 2^(2 beta - 1 - h) + (L - 1) * 2^(2 beta - 2)
        // = (L + 3 - 2h) * 2^(2 beta - 2).
        for (int lev = 0; lev < S; ++lev) {
            const long long per_k = lev == 0
                                        ? (1ll << (2 * (beta - h)))
                                        : static_cast<long long>(lev + 3 - 2 * h) << (2 * beta - 2);
            const long long kmax = (1ll << 24) / per_k;
            a.kc[lev] = static_cast<int>(std::max(1ll, kmax / bke));
        }
        // int64 total: |T| <= n * 2^(beta(S+1) - 2h) * 1.07 in units of the
        // finest level before dropping `drop` bits; keep it below 2^62.
        int nbits = 0;
        while ((1ll << nbits) < n) ++nbits;
        a.drop = std::max(0, nbits + beta * (S + 1) - 2 * h + 1 - 62);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "split pre-pass launch");

    CUtensorMap tmA, tmB;
    int rc;
    if (e4m3) {
        // A planes: m rows x n bytes; B^T planes: p rows x n bytes; box
        // 128 bytes of K x (128 | BN) rows.
        rc = make_tmap_3d(&tmA, CU_TENSOR_MAP_DATA_TYPE_UINT8, a_sl, static_cast<uint64_t>(n),
                          static_cast<uint64_t>(m), static_cast<uint64_t>(S),
                          static_cast<uint64_t>(L.lda), static_cast<uint64_t>(a_plane), 128, kBM);
        if (rc != MOA_OK) return rc;
        rc = make_tmap_3d(&tmB, CU_TENSOR_MAP_DATA_TYPE_UINT8, b_sl, static_cast<uint64_t>(n),
                          static_cast<uint64_t>(p), static_cast<uint64_t>(S),
                          static_cast<uint64_t>(L.ldb), static_cast<uint64_t>(b_plane), 128,
                          static_cast<uint32_t>(bn));
        if (rc != MOA_OK) return rc;
        if (split_units)
            rc = bn == 256   ? launch_split_cfg<256, kModeF64Tmem, kFmtE4M3, true>(a, tmA, tmB, s, st)
                 : bn == 192 ? launch_split_cfg<192, kModeF64Reg, kFmtE4M3, true>(a, tmA, tmB, s, st)
                             : launch_split_cfg<128, kModeF64Reg, kFmtE4M3, true>(a, tmA, tmB, s, st);
        else
            rc = bn == 256   ? launch_split_cfg<256, kModeF64Tmem, kFmtE4M3>(a, tmA, tmB, s, st)
                 : bn == 192 ? launch_split_cfg<192, kModeF64Reg, kFmtE4M3>(a, tmA, tmB, s, st)
                             : launch_split_cfg<128, kModeF64Reg, kFmtE4M3>(a, tmA, tmB, s, st);
    } else if (dt == MOA_F32_SPLIT) {
        // kb-major stages: A slices 32 K x 128 rows (64-byte swizzle), B
        // slices 64 columns x 32 K rows per chunk
        rc = make_tmap_3d(&tmA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, a_sl, static_cast<uint64_t>(n),
                          static_cast<uint64_t>(m), static_cast<uint64_t>(S),
                          static_cast<uint64_t>(L.lda) * 2, static_cast<uint64_t>(a_plane) * 2, bke,
                          kBM, 64);
        if (rc != MOA_OK) return rc;
        rc = make_tmap_3d(&tmB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, b_sl, static_cast<uint64_t>(p),
                          static_cast<uint64_t>(n), static_cast<uint64_t>(S),
                          static_cast<uint64_t>(L.ldb) * 2, static_cast<uint64_t>(b_plane) * 2, 64,
                          bke);
        if (rc != MOA_OK) return rc;
        if (split_units)
            rc = bn == 256 ? launch_split_cfg<256, kModeF32, kFmtBF16KB, true>(a, tmA, tmB, s, st)
                           : launch_split_cfg<128, kModeF32, kFmtBF16KB, true>(a, tmA, tmB, s, st);
        else
            rc = bn == 256 ? launch_split_cfg<256, kModeF32, kFmtBF16KB>(a, tmA, tmB, s, st)
                           : launch_split_cfg<128, kModeF32, kFmtBF16KB>(a, tmA, tmB, s, st);
    } else {
        rc = make_tmap_3d(&tmA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, a_sl, static_cast<uint64_t>(n),
                          static_cast<uint64_t>(m), static_cast<uint64_t>(S),
                          static_cast<uint64_t>(L.lda) * 2, static_cast<uint64_t>(a_plane) * 2, 64,
                          kBM);
        if (rc != MOA_OK) return rc;
        rc = make_tmap_3d(&tmB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, b_sl, static_cast<uint64_t>(p),
                          static_cast<uint64_t>(n), static_cast<uint64_t>(S),
                          static_cast<uint64_t>(L.ldb) * 2, static_cast<uint64_t>(b_plane) * 2, 64,
                          kBK);
        if (rc != MOA_OK) return rc;
        if (split_units)
            rc = bn == 256   ? launch_split_cfg<256, kModeF64Tmem, kFmtBF16, true>(a, tmA, tmB, s, st)
                 : bn == 192 ? launch_split_cfg<192, kModeF64Reg, kFmtBF16, true>(a, tmA, tmB, s, st)
                             : launch_split_cfg<128, kModeF64Reg, kFmtBF16, true>(a, tmA, tmB, s, st);
        else
            rc = bn == 256   ? launch_split_cfg<256, kModeF64Tmem, kFmtBF16>(a, tmA, tmB, s, st)
                 : bn == 192 ? launch_split_cfg<192, kModeF64Reg, kFmtBF16>(a, tmA, tmB, s, st)
                             : launch_split_cfg<128, kModeF64Reg, kFmtBF16>(a, tmA, tmB, s, st);
    }
    if (st) {
        st->slices = S;
        st->products = dt == MOA_F32_SPLIT ? 6 : S * (S + 1) / 2;
        st->kernels = kernels + 1;
    }
    return rc;
}


// ---------------------------------------------------------------- grouped FP32-accuracy
namespace {

struct SplitGPlan {
    size_t pass_off, prob_off, maps_off, head_bytes;   // tables, one upload
    std::vector<size_t> region;                         // per taken problem: its slice planes
    size_t total;
};

struct STaken {
    int idx;        // index in the caller's descriptors
    int bn;         // the lone call's tile width
    SplitLayout L;  // offsets within the problem's region (slice planes only)
};

SplitGPlan split_grouped_plan(int count, const moa_gemm_desc* d, std::vector<STaken>* taken) {
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    std::vector<STaken> tk;
    for (int g = 0; g < count; ++g) {
        if (!split_grouped_ok(d[g])) continue;
        STaken x{};
        x.idx = g;
        x.bn = split_block_n(d[g].m, d[g].p, false);
        x.L = split_layout(d[g].m, d[g].n, d[g].p, MOA_F32_SPLIT, 3);
        tk.push_back(x);
    }
    const size_t G = tk.size();
    SplitGPlan P{};
    size_t off = 0;
    P.pass_off = off;
    off += al(sizeof(SplitGPass) * G);
    P.prob_off = off;
    off += al(sizeof(SplitGProb) * G);
    P.maps_off = off;
    off += al(sizeof(CUtensorMap) * 2 * G);
    P.head_bytes = off;
    for (const STaken& x : tk) {
        P.region.push_back(off);
        off += al(x.L.b_off + static_cast<size_t>(3) * d[x.idx].n * x.L.ldb * 2);
    }
    P.total = G ? off : 0;
    if (taken) *taken = tk;
    return P;
}

}  // namespace

bool split_grouped_ok(const moa_gemm_desc& d) {
    const int64_t lim = int64_t(1) << 31;
    if (d.dt != MOA_F32_SPLIT || d.m <= 0 || d.n <= 0 || d.p <= 0 || d.m >= lim || d.n >= lim ||
        d.p >= lim || d.C == nullptr || reinterpret_cast<uintptr_t>(d.A) % 16 != 0 ||
        reinterpret_cast<uintptr_t>(d.B) % 16 != 0 || reinterpret_cast<uintptr_t>(d.C) % 4 != 0)
        return false;
    // only what the lone call would run without split K: the same sums in
    // the same order, so a grouped result equals the lone one bit for bit
    const int bn = split_block_n(d.m, d.p, false);
    return f32_split_ks(split_layout(d.m, d.n, d.p, MOA_F32_SPLIT, 3), d.m, d.n, d.p, bn) == 1;
}

size_t split_grouped_workspace(int count, const moa_gemm_desc* d) {
    return split_grouped_plan(count, d, nullptr).total;
}

int split_grouped_launch(int count, const moa_gemm_desc* d, void* ws, size_t ws_bytes,
                         cudaStream_t s, int* const* status_of) {
    std::vector<STaken> tk;
    const SplitGPlan P = split_grouped_plan(count, d, &tk);
    const int G = static_cast<int>(tk.size());
    if (G == 0) return MOA_OK;
    if (ws == nullptr || ws_bytes < P.total)
        return fail(MOA_ERR_WORKSPACE, "workspace too small for the grouped split path");
    int* status = launch_status_ptr();
    if (!status) return MOA_ERR_CUDA;
    const int bke = block_k<kFmtBF16KB>();
    uint8_t* base = static_cast<uint8_t*>(ws);
    int slot = 0;
    uint8_t* host = static_cast<uint8_t*>(staging_get(P.head_bytes, &slot));
    if (!host) return fail(MOA_ERR_CUDA, "pinned staging buffer unavailable");
    std::memset(host, 0, P.head_bytes);
    auto* pass = reinterpret_cast<SplitGPass*>(host + P.pass_off);
    auto* probs = reinterpret_cast<SplitGProb*>(host + P.prob_off);
    auto* maps = reinterpret_cast<CUtensorMap*>(host + P.maps_off);
    int pre_blocks = 0;
    for (int i = 0; i < G; ++i) {
        const STaken& x = tk[i];
        const moa_gemm_desc& dd = d[x.idx];
        uint8_t* r = base + P.region[i];
        SplitGPass& q = pass[i];
        q.A = static_cast<const float*>(dd.A);
        q.B = static_cast<const float*>(dd.B);
        q.a_sl = reinterpret_cast<__nv_bfloat16*>(r + x.L.a_off);
        q.b_sl = reinterpret_cast<__nv_bfloat16*>(r + x.L.b_off);
        q.m = dd.m;
        q.n = dd.n;
        q.p = dd.p;
        q.lda = x.L.lda;
        q.ldb = x.L.ldb;
        q.a_plane = dd.m * x.L.lda;
        q.b_plane = dd.n * x.L.ldb;
        q.status = (status_of && status_of[x.idx]) ? status_of[x.idx] : status;
        q.va = vec_rows(dd.A, dd.n, 4);
        q.vb = vec_rows(dd.B, dd.p, 4);
        q.ga = grid_for(q.a_plane / 8, 256);
        q.gb = grid_for(q.b_plane / 8, 256);
        q.begin = pre_blocks;
        pre_blocks += q.ga + q.gb;
    }
    // GEMM problems, longest K first, each with its TMA descriptors
    std::vector<int> order(G);
    for (int i = 0; i < G; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return d[tk[a].idx].n > d[tk[b].idx].n; });
    long units = 0;
    for (int j = 0; j < G; ++j) {
        const int i = order[j];
        const STaken& x = tk[i];
        const moa_gemm_desc& dd = d[x.idx];
        SplitGProb& g = probs[j];
        g.C = static_cast<float*>(dd.C);
        g.m = dd.m;
        g.p = dd.p;
        g.bn = x.bn;
        g.tiles_m = static_cast<int>(ceil_div(dd.m, kBM));
        g.tiles_n = static_cast<int>(ceil_div(dd.p, x.bn));
        g.num_kb = static_cast<int>(ceil_div(dd.n, bke));
        g.group_m = split_raster_group(dd.n);
        g.vec_ok = (dd.p % 4 == 0) && (reinterpret_cast<uintptr_t>(dd.C) % 16 == 0);
        g.unit_begin = static_cast<int>(units);
        units += static_cast<long>(g.tiles_m) * g.tiles_n;
        int rc = make_tmap_3d(&maps[2 * j], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, pass[i].a_sl,
                              static_cast<uint64_t>(dd.n), static_cast<uint64_t>(dd.m), 3,
                              static_cast<uint64_t>(x.L.lda) * 2,
                              static_cast<uint64_t>(pass[i].a_plane) * 2, bke, kBM, 64);
        if (rc == MOA_OK)
            rc = make_tmap_3d(&maps[2 * j + 1], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, pass[i].b_sl,
                              static_cast<uint64_t>(dd.p), static_cast<uint64_t>(dd.n), 3,
                              static_cast<uint64_t>(x.L.ldb) * 2,
                              static_cast<uint64_t>(pass[i].b_plane) * 2, 64, bke);
        if (rc != MOA_OK) {
            staging_release(slot, s);
            return rc;
        }
    }
    if (units > (1L << 30)) {
        staging_release(slot, s);
        return fail(MOA_ERR_ARG, "too many tiles in one grouped call");
    }
    cudaError_t e = cudaMemcpyAsync(base, host, P.head_bytes, cudaMemcpyHostToDevice, s);
    staging_release(slot, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(grouped split tables)");
    split3_g_kernel<<<pre_blocks, 256, 0, s>>>(reinterpret_cast<const SplitGPass*>(base + P.pass_off),
                                               G);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "grouped split pre-pass launch");
    SplitArgs a{};
    a.f64 = 0;
    a.levels = 1;
    a.S = 3;
    a.kc[0] = f32_split_chunk_kb(bke);
    a.ksplit = 1;
    a.lgroups = 1;
    a.lmask[0] = 0xFFFFFFFFu;
    a.wait_limit_ns = wait_limit_ns();
    a.status = status;
    a.probs = reinterpret_cast<const SplitGProb*>(base + P.prob_off);
    a.maps = reinterpret_cast<const CUtensorMap*>(base + P.maps_off);
    a.nprob = G;
    a.num_units = static_cast<int>(units);
    CUtensorMap unused{};
    const int rc = launch_split_cfg<256, kModeF32, kFmtBF16KB, false, true>(a, unused, unused, s,
                                                                            nullptr);
    if (rc != MOA_OK) return rc;
    log_msg(2, "grouped split: %d problems, %ld tiles", G, units);
    return MOA_OK;
}

}  // namespace moa
