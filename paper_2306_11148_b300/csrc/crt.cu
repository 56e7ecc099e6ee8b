// crt.cu -- FP64-accuracy ONF GEMM from modular slices (MOA_F64_CRT_F32IN,
// MOA_F64_CRT_F64IN).
//
// The result is Eq. (eq:dnf) of Sec. 2, C[(i*p)+j] := sum_k A[(i*n)+k] *
// B[(k*p)+j], to FP64 accuracy; the slicing is not in the paper (it is the
// residue-number form of error-free slicing, "Ozaki scheme II" of Ozaki,
// Uchino & Imamura, 2025):
//
// * each row i of A is scaled by 2^(t - eA_i) (eA_i the frexp exponent of
//   max_k |A[i,k]|) and rounded to the nearest integer A'[i,k], |A'| <= 2^t;
//   each column j of B likewise by 2^(t - eB_j) to B'[k,j];
// * for M pairwise-coprime moduli q_l <= 256 (product P), the symmetric
//   residues A' mod q_l and B' mod q_l are integers of magnitude <= 128,
//   exact in BF16; one BF16 tensor-core GEMM per modulus forms
//   sum_k (A' mod q_l)(B' mod q_l), exact in FP32 over K chunks of 1024
//   (1024 * 128^2 = 2^24), reduced modulo q_l after every chunk;
// * the Chinese remainder theorem recovers C' = A'B' itself from its M
//   residues, because t is chosen so that n * 2^(2t) < P / 2; C' is rounded
//   once to FP64 and scaled by 2^(eA_i + eB_j - 2t).
//
// The result is therefore exactly fl(2^(eA_i + eB_j - 2t) * (A'B')[i,j]):
// deterministic, independent of the K order, with M slice GEMMs (14 for
// n <= 36639 at t >= 47) instead of the S(S+1)/2 = 28 of the integer-digit
// form.
//
// Launches per call: a clear of the column maxima, the exponent pass, the
// residue pass (A and B in one launch), the residue GEMM (one persistent
// launch over (modulus, tile, K slice) units, modulus-major so that the L2
// holds one modulus's planes at a time) and the reconstruction pass.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "crt.h"
#include "fastdiv.cuh"
#include "fpbits.cuh"
#include "internal.h"
#include "ptx.cuh"

namespace moa {

namespace {

// The moduli: 256, 255, 254, ... keeping each integer coprime to every one
// taken before it (254 = 2 * 127 shares 2 with 256, 252 likewise, 249 = 3 * 83
// shares 3 with 255, ...).  Every symmetric residue lies in [-128, 128].
__host__ __device__ constexpr uint32_t crt_mod(int l) {
    return l == 0 ? 256u : l == 1 ? 255u : l == 2 ? 253u : l == 3 ? 251u : l == 4 ? 247u
         : l == 5 ? 241u : l == 6 ? 239u : l == 7 ? 233u : l == 8 ? 229u : l == 9 ? 227u
         : l == 10 ? 223u : l == 11 ? 217u : l == 12 ? 211u : l == 13 ? 199u : l == 14 ? 197u
         : 193u;
}

using u128 = unsigned __int128;
using i128 = __int128;

// Per-call constants of the reconstruction (kernel parameter).
struct CrtConsts {
    int M;                               // moduli in use
    int t;                               // operand bits
    uint32_t w[kCrtMaxModuli][4];        // CRT weights W_l = (P / q_l) * ((P / q_l)^-1 mod q_l)
                                         //   mod P, as 32-bit limbs, least significant first
    uint64_t P_lo, P_hi;                 // P = prod q_l
    int sP;                              // quotient estimate: floor(X / 2^sP) * kq ~ X / P,
    float kq;                            //   sP = bit length of P - 32, kq = 2^sP / P rounded
};

// ---------------------------------------------------------------- host arithmetic
u128 crt_product(int M) {
    u128 P = 1;
    for (int l = 0; l < M; ++l) P *= crt_mod(l);
    return P;
}

// x^-1 mod q for x coprime to q (extended Euclid on small integers).
int64_t inv_mod(int64_t x, int64_t q) {
    int64_t a = ((x % q) + q) % q, b = q, u = 1, v = 0;
    while (b != 0) {
        const int64_t k = a / b;
        a -= k * b;
        u -= k * v;
        int64_t tmp = a; a = b; b = tmp;
        tmp = u; u = v; v = tmp;
    }
    return ((u % q) + q) % q;
}

CrtConsts crt_consts(int M, int t) {
    CrtConsts c{};
    c.M = M;
    c.t = t;
    const u128 P = crt_product(M);
    c.P_lo = static_cast<uint64_t>(P);
    c.P_hi = static_cast<uint64_t>(P >> 64);
    auto as_double = [](u128 v) {
        return static_cast<double>(static_cast<uint64_t>(v >> 64)) * 18446744073709551616.0 +
               static_cast<double>(static_cast<uint64_t>(v));
    };
    for (int l = 0; l < M; ++l) {
        const u128 Ml = P / crt_mod(l);
        const int64_t Ml_mod = static_cast<int64_t>(Ml % crt_mod(l));
        const int64_t y = inv_mod(Ml_mod, crt_mod(l));
        const u128 W = (Ml * static_cast<u128>(y)) % P;   // Ml * y < P * 256 < 2^128
        for (int k = 0; k < 4; ++k) c.w[l][k] = static_cast<uint32_t>(W >> (32 * k));
    }
    int bits = 0;
    while (bits < 128 && (P >> bits) != 0) ++bits;
    c.sP = bits > 32 ? bits - 32 : 0;
    c.kq = static_cast<float>(std::ldexp(1.0, c.sP) / as_double(P));
    return c;
}

// ---------------------------------------------------------------- exponent pass
// One warp per row: eA[r] = frexp exponent of max_k |A[r,k]|.  Flags NaN/Inf.
template <typename T>
__device__ void crt_row_exp_part(const T* __restrict__ X, int64_t rows, int64_t cols,
                                 int* __restrict__ e_out, int* status, int64_t bid, int64_t nblk) {
    using B = Bits<T>;
    const int lane = threadIdx.x & 31;
    const int64_t warps = nblk * (blockDim.x >> 5);
    bool bad = false;
    for (int64_t r = bid * (blockDim.x >> 5) + (threadIdx.x >> 5); r < rows; r += warps) {
        typename B::U mx = 0;
        for (int64_t c = lane; c < cols; c += 32) mx = max(mx, B::abs_bits(X[r * cols + c]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) {
            bad |= mx >= B::kInf;
            e_out[r] = B::frexp_exp(mx);
        }
    }
    if (bad) atomicCAS(status, kDevOk, kDevNonFinite);
}

// Column maxima of |B| (bit patterns) by atomicMax over chunks of rows: block
// bid covers 256 columns from 256 (bid % gx) and rows chunk * (bid / gx) ..
template <typename T>
__device__ void crt_col_max_part(const T* __restrict__ X, int64_t rows, int64_t cols,
                                 int64_t chunk, typename Bits<T>::U* __restrict__ cmax,
                                 int64_t bid, int64_t gx) {
    using B = Bits<T>;
    const int64_t c = (bid % gx) * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    const int64_t r0 = (bid / gx) * chunk;
    const int64_t r1 = min(rows, r0 + chunk);
    typename B::U mx = 0;
    for (int64_t r = r0; r < r1; ++r) mx = max(mx, B::abs_bits(X[r * cols + c]));
    if (mx != 0) atomicMax(&cmax[c], mx);
}

template <typename T>
__global__ void __launch_bounds__(256)
    crt_exps_kernel(const T* __restrict__ A, int64_t m, int64_t n, const T* __restrict__ B,
                    int64_t p, int64_t chunk, int* __restrict__ eA,
                    typename Bits<T>::U* __restrict__ cmax, int* status, int rblocks, int64_t gx) {
    const int b = static_cast<int>(blockIdx.x);
    if (b < rblocks)
        crt_row_exp_part(A, m, n, eA, status, b, rblocks);
    else
        crt_col_max_part(B, n, p, chunk, cmax, b - rblocks, gx);
}

// ---------------------------------------------------------------- residue pass
// 2^s mod q_l for s < 128 (kernel parameter; copied to shared memory as FP32).
constexpr int kPow2Cols = 128;
struct CrtPow2 {
    uint8_t v[kCrtMaxModuli][kPow2Cols];
};

// x (an integer-valued float) minus the nearest multiple of q: rint(x / q)
// by the magic-number addition (exact for |x / q| < 2^22), the product
// subtracted by one fused multiply-add (the result is an exact integer).  The
// quotient comes from x * RN(1/q), off from x / q by at most 2^-23 x / q: for
// |x| <= 2^24 the result lies within 0.51 q + 1 of zero, and for |x| < 2^21
// (the estimate's error is then below 1/(2q), the least distance of x / q from
// a half-integer it is not on) it is the symmetric residue, |result| <= q/2.
__device__ __forceinline__ float mod_reduce(float x, float q, float qinv) {
    const float y = __fmul_rn(x, qinv);
    const float k = __fsub_rn(__fadd_rn(y, 12582912.0f), 12582912.0f);
    return __fmaf_rn(-k, q, x);
}

// An integer 0 <= v < 2^23 as an FP32 value (the float with bits 2^23 | v is
// 2^23 + v exactly).
__device__ __forceinline__ float small_uint_to_float(uint32_t v) {
    return __fsub_rn(__uint_as_float(0x4B000000u | v), 8388608.0f);
}

// The scaled integer D = rint(x * 2^k) of one element as (sign, 12-bit
// pieces as exact floats, shift): |D| = sum_i p[i] 2^(12 i + s).  FP32
// inputs: two pieces of the 24-bit significand (or of the rounded D when k
// shifts it right) and a shift s < 64; FP64 inputs: six pieces of |D| < 2^63
// and s = 0.
template <int NP>
struct ScaledParts {
    float p[NP];
    int s;
    bool neg;
};
__device__ __forceinline__ ScaledParts<2> scaled_parts(float x, int k) {
    ScaledParts<2> r;
    const uint32_t b = __float_as_uint(x);
    r.neg = (b >> 31) != 0;
    r.s = 0;
    const int ex = static_cast<int>((b >> 23) & 0xFF);
    uint32_t mant = b & 0x7FFFFFu;
    int E = -149;
    if (ex != 0) {
        mant |= 1u << 23;
        E = ex - 150;
    }
    const int sh = E + k;
    uint32_t base;
    if (sh >= 0) {
        base = mant;
        r.s = sh;
    } else {
        const int kk = -sh;
        if (kk > 25) {
            base = 0;
        } else {
            const uint32_t q = mant >> kk;
            const uint32_t rem = mant & ((1u << kk) - 1u);
            const uint32_t half = 1u << (kk - 1);
            base = q + ((rem > half || (rem == half && (q & 1u))) ? 1u : 0u);
        }
    }
    // the pieces carry the sign, so every residue comes out signed
    const uint32_t sgn = r.neg ? 0x80000000u : 0u;
    r.p[0] = __uint_as_float(__float_as_uint(small_uint_to_float(base & 0xFFFu)) ^ sgn);
    r.p[1] = __uint_as_float(__float_as_uint(small_uint_to_float(base >> 12)) ^ sgn);   // base <= 2^24
    return r;
}
__device__ __forceinline__ ScaledParts<6> scaled_parts(double x, int k) {
    ScaledParts<6> r;
    const long long D = Bits<double>::round_scaled(x, k);
    r.neg = D < 0;
    r.s = 0;
    const uint64_t v = static_cast<uint64_t>(r.neg ? -D : D);
    const uint32_t sgn = r.neg ? 0x80000000u : 0u;
#pragma unroll
    for (int i = 0; i < 6; ++i)
        r.p[i] = __uint_as_float(
            __float_as_uint(small_uint_to_float(static_cast<uint32_t>((v >> (12 * i)) & 0xFFFu))) ^ sgn);
    return r;
}

// Symmetric residue (|r| <= q/2, an integer-valued float with the element's
// sign applied) of one element modulo q = crt_mod(L); tab: the block's shared
// table row of 2^s mod q.
// tab: the block's shared table row of modulus L, tab[s] = (2^s mod q,
// 2^(s+12) mod q) for s < 64.  The pieces carry the element's sign.
template <int L, int NP>
__device__ __forceinline__ float residue_of(const ScaledParts<NP>& e, const float2* tab) {
    constexpr float q = static_cast<float>(crt_mod(L));
    constexpr float qinv = 1.0f / static_cast<float>(crt_mod(L));
    if constexpr (NP == 2) {
        // two pieces below 2^12 times 2^s mod q (< 2^8): the sum is below 2^21,
        // one reduction gives the symmetric residue
        const float2 c = tab[e.s];
        return mod_reduce(__fmaf_rn(e.p[1], c.y, __fmul_rn(e.p[0], c.x)), q, qinv);
    } else {
        // six pieces at 2^0, 2^12, ..., 2^60: the sum is below 2^23, reduced
        // within 0.51 q + 1, then reduced once more to the symmetric residue
        float t = __fmul_rn(e.p[0], tab[0].x);
        t = __fmaf_rn(e.p[1], tab[0].y, t);
        t = __fmaf_rn(e.p[2], tab[24].x, t);
        t = __fmaf_rn(e.p[3], tab[24].y, t);
        t = __fmaf_rn(e.p[4], tab[48].x, t);
        t = __fmaf_rn(e.p[5], tab[48].y, t);
        return mod_reduce(mod_reduce(t, q, qinv), q, qinv);
    }
}

// BF16 patterns of two integer-valued floats of magnitude <= 256 (exact in
// BF16: at most 8 significant bits, so the upper 16 bits are the pattern),
// packed low half first.
__device__ __forceinline__ uint32_t bf16x2_of_ints(float lo, float hi) {
    return (__float_as_uint(lo) >> 16) | (__float_as_uint(hi) & 0xFFFF0000u);
}

// Loads X[r, c0 .. c0+3] (zero past `cols`); 16-byte loads when allowed.
template <typename T>
__device__ __forceinline__ void load4(const T* __restrict__ X, int64_t r, int64_t cols, int64_t c0,
                                      bool vec, T (&x)[4]) {
    const T* src = X + r * cols + c0;
    if (vec && c0 + 4 <= cols) {
        if constexpr (sizeof(T) == 4) {
            const float4 a = reinterpret_cast<const float4*>(src)[0];
            x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
        } else {
#pragma unroll
            for (int v = 0; v < 2; ++v) {
                const double2 d = reinterpret_cast<const double2*>(src)[v];
                x[2 * v] = d.x;
                x[2 * v + 1] = d.y;
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) x[i] = (c0 + i < cols) ? src[i] : T(0);
    }
}

// Writes the residues of 4 elements at element offset o of planes L .. M-1
// (one 8-byte store per plane).
template <int L, int NP>
__device__ __forceinline__ void store_planes(const ScaledParts<NP> (&v)[4], int M,
                                             const float2* tab, __nv_bfloat16* __restrict__ out,
                                             int64_t plane, int64_t o) {
    if constexpr (L < kCrtMaxModuli) {
        if (L >= M) return;
        const float2* row = tab + L * 64;
        const uint32_t w0 = bf16x2_of_ints(residue_of<L, NP>(v[0], row), residue_of<L, NP>(v[1], row));
        const uint32_t w1 = bf16x2_of_ints(residue_of<L, NP>(v[2], row), residue_of<L, NP>(v[3], row));
        *reinterpret_cast<uint2*>(out + L * plane + o) = make_uint2(w0, w1);
        store_planes<L + 1, NP>(v, M, tab, out, plane, o);
    }
}

// Residue planes of X (rows x cols, row-major) into M BF16 planes of row
// pitch ld (a multiple of 8; zero pad); 4 consecutive elements per thread.
// AXIS 0: exponent per row from e[r]; AXIS 1: exponent per column from the
// column maximum cmax[c] (the threads of row 0 store it to e[c] and flag
// NaN/Inf).
template <typename T, int AXIS>
__device__ void crt_residue_part(const T* __restrict__ X, int64_t rows, int64_t cols, int64_t ld,
                                 int* __restrict__ e, const typename Bits<T>::U* __restrict__ cmax,
                                 int* status, int t, int M, int vec, const float2* tab,
                                 __nv_bfloat16* __restrict__ out, int64_t plane, int64_t bid,
                                 int64_t nblk) {
    const int64_t gpr = ld / 4;
    const int64_t total = rows * gpr;
    const int64_t step = nblk * blockDim.x;
    const bool small = total + step < (int64_t(1) << 31);
    const FastDiv fd{static_cast<uint32_t>(gpr),
                     gpr <= 1 ? 0xFFFFFFFFu : static_cast<uint32_t>((uint64_t(1) << 32) / gpr)};
    for (int64_t g = bid * blockDim.x + threadIdx.x; g < total; g += step) {
        int64_t r, c0;
        if (small) {
            uint32_t rem;
            r = fdiv(static_cast<uint32_t>(g), fd, rem);
            c0 = static_cast<int64_t>(rem) * 4;
        } else {
            r = g / gpr;
            c0 = (g - r * gpr) * 4;
        }
        T x[4];
        load4(X, r, cols, c0, vec != 0, x);
        ScaledParts<sizeof(T) == 8 ? 6 : 2> v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t c = c0 + i;
            int ex = 0;
            if (c < cols) {
                if (AXIS == 0) {
                    ex = e[r];
                } else {
                    const typename Bits<T>::U mx = cmax[c];
                    if (r == 0 && mx >= Bits<T>::kInf) atomicCAS(status, kDevOk, kDevNonFinite);
                    ex = Bits<T>::frexp_exp(mx);
                    if (r == 0) e[c] = ex;
                }
            }
            v[i] = scaled_parts(x[i], t - ex);
        }
        store_planes<0, sizeof(T) == 8 ? 6 : 2>(v, M, tab, out, plane, r * ld + c0);
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
    crt_residue_kernel(const T* __restrict__ A, int64_t m, int64_t n, int64_t lda, int va,
                       const int* __restrict__ eA, const T* __restrict__ B, int64_t p, int64_t ldb,
                       int vb, int* __restrict__ eB, const typename Bits<T>::U* __restrict__ cmax,
                       int* status, int t, int M, __nv_bfloat16* __restrict__ a_out,
                       int64_t a_plane, __nv_bfloat16* __restrict__ b_out, int64_t b_plane,
                       int ga, const CrtPow2 pow2) {
    // tab[l * 64 + s] = (2^s mod q_l, 2^(s+12) mod q_l): a row per modulus, so
    // threads of a warp that read different s of one row mostly hit different banks
    __shared__ float2 tab[kCrtMaxModuli * 64];
    for (int i = threadIdx.x; i < kCrtMaxModuli * 64; i += blockDim.x)
        tab[i] = make_float2(static_cast<float>(pow2.v[i / 64][i % 64]),
                             static_cast<float>(pow2.v[i / 64][i % 64 + 12]));
    __syncthreads();
    if (static_cast<int>(blockIdx.x) < ga)
        crt_residue_part<T, 0>(A, m, n, lda, const_cast<int*>(eA), nullptr, status, t, M, va, tab,
                               a_out, a_plane, blockIdx.x, ga);
    else
        crt_residue_part<T, 1>(B, n, p, ldb, eB, cmax, status, t, M, vb, tab, b_out, b_plane,
                               blockIdx.x - ga, gridDim.x - ga);
}

// ---------------------------------------------------------------- residue GEMM
constexpr int kBM = 128;
constexpr int kBK = 64;            // BF16 elements per K block (128 bytes)
constexpr int kChunkKB = 16;       // K blocks per exact FP32 chunk: 1024 * 128^2 = 2^24

template <int BN>
struct CrtCfg {
    static constexpr int kAStage = kBM * 128;                // 128 rows x 128 B
    static constexpr int kBChunk = kBK * 128;                // 64 K rows x 64 columns (MN-major)
    static constexpr int kBStage = (BN / 64) * kBChunk;
    static constexpr int kStageBytes = kAStage + kBStage;
    static constexpr int kStages = BN == 256 ? 4 : 6;
    static constexpr int kSmem = 1024 + kStages * kStageBytes + 256;
    static_assert(kSmem <= 227 * 1024, "crt kernel shared memory");
    static constexpr int kEpiWarps = 4 * (BN / 64);          // 32 rows x 64 columns each
    static constexpr int kThreads = 64 + 32 * kEpiWarps;
    static constexpr int kTmemCols = 2 * BN;                 // two chunk accumulators
    static constexpr uint32_t kIdesc = make_idesc(1u, kBM, BN, 0u, 1u);
};

// One problem of a grouped residue GEMM (device table).
struct CrtGProb {
    uint8_t* R;                   // its residue planes: l x m x ldr bytes (one K slice)
    int64_t m, p, ldr;
    int tiles_m, tiles_n, num_kb, group_m;
    int M, bn;                    // moduli; tile width (128 or 256)
    int unit_begin, pad;          // first unit of the problem in the work list
};

struct CrtGemmArgs {
    uint8_t* R;                   // residue planes: (l * ks + s) x r_rows x ldr bytes
    int64_t m, n, p, ldr;
    int64_t r_rows;               // rows a residue plane holds (m, or more for a band of rows)
    int tiles_m, tiles_n, num_kb, group_m;
    int M, ks;
    float qf[kCrtMaxModuli];      // moduli and their rounded reciprocals
    float qinv[kCrtMaxModuli];
    uint64_t wait_limit_ns;
    int* status;
    // grouped launches: the problems (sorted by unit_begin) and their TMA
    // descriptors (A, B per problem, global memory, 64-byte aligned)
    const CrtGProb* probs;
    const CUtensorMap* maps;
    int nprob;
    int num_units;
};

__device__ __forceinline__ void crt_tile_coords(int t, int tiles_m, int tiles_n, int group_m,
                                                int& tm, int& tn) {
    const int per_group = group_m * tiles_n;
    const int g = t / per_group;
    const int first_m = g * group_m;
    const int gsize = min(tiles_m - first_m, group_m);
    const int r = t - g * per_group;
    tm = first_m + r % gsize;
    tn = r / gsize;
}

// What every role needs to know about work unit u.
struct CrtUnit {
    int g;                 // problem (0 for a single GEMM)
    int l, tm, tn, s;      // modulus, tile, K slice
    int kb_lo, kb_hi;      // K blocks
    int bn;                // tile width (the MMA N extent)
    uint8_t* R;
    int64_t m, p, ldr, r_rows;
    int ks;
};

// Single GEMM: unit u = modulus l (slowest), tile t, K slice s (fastest).
// Grouped: the problem by binary search over the units' starts, then modulus
// and tile within it (one K slice).
template <bool GROUPED>
__device__ __forceinline__ CrtUnit crt_resolve(const CrtGemmArgs& a, int u) {
    CrtUnit x;
    if constexpr (!GROUPED) {
        const int per_l = a.tiles_m * a.tiles_n * a.ks;
        x.g = 0;
        x.l = u / per_l;
        const int r = u - x.l * per_l;
        const int t = r / a.ks;
        x.s = r - t * a.ks;
        x.kb_lo = static_cast<int>(static_cast<long long>(x.s) * a.num_kb / a.ks);
        x.kb_hi = static_cast<int>(static_cast<long long>(x.s + 1) * a.num_kb / a.ks);
        crt_tile_coords(t, a.tiles_m, a.tiles_n, a.group_m, x.tm, x.tn);
        x.bn = 0;   // the kernel's BN
        x.R = a.R;
        x.m = a.m;
        x.p = a.p;
        x.ldr = a.ldr;
        x.r_rows = a.r_rows;
        x.ks = a.ks;
    } else {
        int lo = 0, hi = a.nprob - 1;
        while (lo < hi) {   // last problem with unit_begin <= u
            const int mid = (lo + hi + 1) >> 1;
            if (a.probs[mid].unit_begin <= u) lo = mid; else hi = mid - 1;
        }
        const CrtGProb& pr = a.probs[lo];
        x.g = lo;
        const int r0 = u - pr.unit_begin;
        const int per_l = pr.tiles_m * pr.tiles_n;
        x.l = r0 / per_l;
        crt_tile_coords(r0 - x.l * per_l, pr.tiles_m, pr.tiles_n, pr.group_m, x.tm, x.tn);
        x.s = 0;
        x.kb_lo = 0;
        x.kb_hi = pr.num_kb;
        x.bn = pr.bn;
        x.R = pr.R;
        x.m = pr.m;
        x.p = pr.p;
        x.ldr = pr.ldr;
        x.r_rows = pr.m;
        x.ks = 1;
    }
    return x;
}

template <int BN, bool GROUPED>
__global__ void __launch_bounds__(CrtCfg<BN>::kThreads, 1)
    crt_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    const CrtGemmArgs args) {
    using Cfg = CrtCfg<BN>;
    constexpr int kStages = Cfg::kStages;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                               ~static_cast<uintptr_t>(1023));
    uint8_t* sA = smem;
    uint8_t* sB = smem + kStages * Cfg::kAStage;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + kStages * Cfg::kBStage);
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
    const int num_units =
        GROUPED ? args.num_units : args.M * args.tiles_m * args.tiles_n * args.ks;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer: (unit, K block)
            int stage = 0;
            uint32_t phase = 0;
            long issued = 0;
            bool ok = true;
            int g_prev = -1;
            for (int u = blockIdx.x; u < num_units && ok; u += gridDim.x) {
                const CrtUnit x = crt_resolve<GROUPED>(args, u);
                const int bn = GROUPED ? x.bn : BN;
                const CUtensorMap* mA = GROUPED ? args.maps + 2 * x.g : &tmA;
                const CUtensorMap* mB = GROUPED ? args.maps + 2 * x.g + 1 : &tmB;
                if (GROUPED && x.g != g_prev) {
                    prefetch_tmap(mA);
                    prefetch_tmap(mB);
                    g_prev = x.g;
                }
                const uint32_t bytes = Cfg::kAStage + static_cast<uint32_t>(bn / 64) * Cfg::kBChunk;
                for (int kb = x.kb_lo; kb < x.kb_hi; ++kb) {
                    if (!mbar_wait(&empty[stage], phase ^ 1u, ctl, limit, status)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[stage], bytes);
                    tma_load_3d(sA + stage * Cfg::kAStage, mA, &full[stage], kb * kBK, x.tm * kBM,
                                x.l);
                    for (int c = 0; c < bn / 64; ++c)
                        tma_load_3d(sB + stage * Cfg::kBStage + c * Cfg::kBChunk, mB, &full[stage],
                                    x.tn * bn + c * 64, kb * kBK, x.l);
                    ++issued;
                    if (++stage == kStages) {
                        stage = 0;
                        phase ^= 1u;
                    }
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
                const CrtUnit x = crt_resolve<GROUPED>(args, u);
                const int kb_lo = x.kb_lo, kb_hi = x.kb_hi;
                const uint32_t idesc =
                    GROUPED ? make_idesc(1u, kBM, static_cast<uint32_t>(x.bn), 0u, 1u) : Cfg::kIdesc;
                for (int kb0 = kb_lo; kb0 < kb_hi && ok; kb0 += kChunkKB, ++cnt) {
                    const int buf = static_cast<int>(cnt & 1);
                    const uint32_t bph = static_cast<uint32_t>((cnt >> 1) & 1);
                    if (!mbar_wait(&tempty[buf], bph ^ 1u, ctl, limit, status)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem_base + static_cast<uint32_t>(buf * BN);
                    const int kb1 = min(kb_hi, kb0 + kChunkKB);
                    for (int kb = kb0; kb < kb1; ++kb) {
                        if (!mbar_wait(&full[stage], phase, ctl, limit, status)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint64_t adesc =
                            smem_desc_sw128(smem_u32(sA + stage * Cfg::kAStage), 16, 1024);
                        const uint64_t bdesc =
                            smem_desc_sw128(smem_u32(sB + stage * Cfg::kBStage), Cfg::kBChunk, 1024);
                        // four MMAs of 16 K elements (32 bytes of A's rows) each
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            mma_f16(d, adesc + static_cast<uint64_t>((k * 32) >> 4),
                                    bdesc + static_cast<uint64_t>((k * 16 * 128) >> 4), idesc,
                                    (kb == kb0 && k == 0) ? 0u : 1u);
                        mma_commit(&empty[stage]);
                        if (++stage == kStages) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                    if (!ok) break;
                    mma_commit(&tfull[buf]);
                }
            }
            // Every MMA issued above must finish before TMEM is released.
            mma_commit(drain);
            CtaCtl local{0};
            mbar_wait(drain, 0, &local, limit, status);
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: quadrant q = warp % 4 (32 rows), column group h
        const int q = warp & 3;
        const int h = (warp - 2) >> 2;
        const uint32_t lane_base = static_cast<uint32_t>(q * 32) << 16;
        long cnt = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < num_units && ok; u += gridDim.x) {
            const CrtUnit x = crt_resolve<GROUPED>(args, u);
            const int l = x.l, tm = x.tm, tn = x.tn, s = x.s;
            const int bn = GROUPED ? x.bn : BN;
            const bool cols_live = h * 64 < bn;   // narrow tiles leave the last warps idle
            const float qf = args.qf[l], qinv = args.qinv[l];
            float acc[64];
#pragma unroll
            for (int i = 0; i < 64; ++i) acc[i] = 0.f;
            for (int kb0 = x.kb_lo; kb0 < x.kb_hi; kb0 += kChunkKB, ++cnt) {
                const int buf = static_cast<int>(cnt & 1);
                const uint32_t bph = static_cast<uint32_t>((cnt >> 1) & 1);
                ok = mbar_wait(&tfull[buf], bph, ctl, limit, status);
                if (!__all_sync(0xffffffffu, ok)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t a_base =
                    tmem_base + lane_base + static_cast<uint32_t>(buf * BN + h * 64);
                if (!GROUPED || cols_live) {
#pragma unroll
                    for (int g = 0; g < 4; ++g) {
                        uint32_t r[16];
                        tmem_ld16(a_base + 16u * g, r);
                        tmem_ld_wait();
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            acc[g * 16 + i] = __fadd_rn(acc[g * 16 + i],
                                                        mod_reduce(__uint_as_float(r[i]), qf, qinv));
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[buf]);
            }
            if (!ok) break;
            // the unit's residues in [0, q) as bytes of plane (l, s)
            const int64_t row = static_cast<int64_t>(tm) * kBM + q * 32 + lane;
            const int64_t col0 = static_cast<int64_t>(tn) * bn + h * 64;
            if (cols_live && row < x.m && col0 < x.p) {
                uint32_t w[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    uint32_t word = 0;
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        float r = mod_reduce(acc[4 * i + b], qf, qinv);   // |r| <= q/2 + 1
                        r = r < 0.f ? __fadd_rn(r, qf) : r;
                        r = r >= qf ? __fsub_rn(r, qf) : r;
                        word |= (__float_as_uint(__fadd_rn(r, 8388608.0f)) & 0xFFu) << (8 * b);
                    }
                    w[i] = word;
                }
                uint8_t* dst =
                    x.R + ((static_cast<int64_t>(l) * x.ks + s) * x.r_rows + row) * x.ldr + col0;
                if (col0 + 64 <= x.ldr) {
#pragma unroll
                    for (int v = 0; v < 4; ++v)
                        reinterpret_cast<uint4*>(dst)[v] =
                            make_uint4(w[4 * v], w[4 * v + 1], w[4 * v + 2], w[4 * v + 3]);
                } else {
                    for (int i = 0; i < 64 && col0 + i < x.ldr; ++i)
                        dst[i] = static_cast<uint8_t>((w[i >> 2] >> (8 * (i & 3))) & 0xFFu);
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

// ---------------------------------------------------------------- residue GEMM, CTA pairs
// The same units over 256 x 256 output tiles, each computed by a cluster of
// two CTAs (CTA r: rows 128 r .. 128 r + 127 of the tile) with cta_group::2
// MMAs of M = 256, N = 256.  Each CTA stages its 128 rows of A and its half
// (128 columns) of B: 32 KB a K block instead of 48 KB, so six stages are in
// flight, and the L2 serves a third less operand traffic per product.
//   * producer (warp 0 of each CTA): its own halves into its own stages; the
//     loads of both CTAs complete on the even CTA's `full` barrier (which
//     the even CTA's producer arms for both: 64 KB a stage);
//   * the even CTA's warp 1 issues the MMAs; its commits release the stage
//     in both CTAs (`empty`) and hand each chunk accumulator to both CTAs'
//     epilogues (`tfull`);
//   * epilogue (16 warps of each CTA): its 128 x 256 accumulator, as in the
//     one-CTA kernel; both CTAs' warps report the drain to the even CTA's
//     `tempty` barrier.
// Every wait is bounded; both CTAs pass a cluster barrier before TMEM is
// released and before either exits, so neither leaves while the other's MMAs
// or arrivals may still reach it.
struct CrtPairCfg {
    static constexpr int kAStage = kBM * 128;                 // this CTA's 128 rows x 128 B
    static constexpr int kBChunk = kBK * 128;                 // 64 K rows x 64 columns
    static constexpr int kBStage = 2 * kBChunk;               // this CTA's 128 columns
    static constexpr int kStageBytes = kAStage + kBStage;
    static constexpr int kStages = 6;
    static constexpr int kSmem = 1024 + kStages * kStageBytes + 256;
    static_assert(kSmem <= 227 * 1024, "crt pair kernel shared memory");
    static constexpr int kEpiWarps = 16;                      // 32 rows x 64 columns each
    static constexpr int kThreads = 64 + 32 * kEpiWarps;
    static constexpr int kTmemCols = 512;                     // two 256-column accumulators
    static constexpr uint32_t kIdesc = make_idesc(1u, 2 * kBM, 256, 0u, 1u);
};
constexpr int kPairRows = 2 * kBM;

// Unit u of the pair kernel: modulus l (slowest), then the 256 x 256 tile.
__device__ __forceinline__ void crt_pair_unit(const CrtGemmArgs& a, int u, int& l, int& tm,
                                              int& tn) {
    const int per_l = a.tiles_m * a.tiles_n;
    l = u / per_l;
    crt_tile_coords(u - l * per_l, a.tiles_m, a.tiles_n, a.group_m, tm, tn);
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(CrtPairCfg::kThreads, 1)
    crt_gemm_pair_kernel(const __grid_constant__ CUtensorMap tmA,
                         const __grid_constant__ CUtensorMap tmB, const CrtGemmArgs args) {
    using Cfg = CrtPairCfg;
    constexpr int kStages = Cfg::kStages;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                               ~static_cast<uintptr_t>(1023));
    uint8_t* sA = smem;
    uint8_t* sB = smem + kStages * Cfg::kAStage;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + kStages * Cfg::kBStage);
    uint64_t* full = bars;                   // (even CTA) both CTAs' stage has landed
    uint64_t* empty = bars + kStages;        // the pair's MMAs are done with the stage
    uint64_t* tfull = bars + 2 * kStages;    // a chunk accumulator is complete
    uint64_t* tempty = tfull + 2;            // (even CTA) both epilogues drained it
    uint64_t* drain = tempty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    CtaCtl* ctl = reinterpret_cast<CtaCtl*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint32_t rank = cluster_ctarank();
    const uint64_t limit = args.wait_limit_ns;
    int* status = args.status;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 2 * Cfg::kEpiWarps);
        }
        mbar_init(drain, 1);
        ctl->abort = 0;
        fence_barrier_init();
    }
    if (warp == 0 && lane == 0) {
        prefetch_tmap(&tmA);
        prefetch_tmap(&tmB);
    }
    if (warp == 1) {
        tmem_alloc_pair(tmem_slot, Cfg::kTmemCols);
        tmem_relinquish_pair();
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();   // both CTAs' barriers exist before any arrival crosses over
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const int cid = static_cast<int>(blockIdx.x) >> 1;
    const int ncl = static_cast<int>(gridDim.x) >> 1;
    const int num_units = args.M * args.tiles_m * args.tiles_n;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer: this CTA's rows of A, columns of B,
            // completing on the even CTA's full barrier
            const uint32_t full0 = mapa_shared(smem_u32(full), 0);
            int stage = 0;
            uint32_t phase = 0;
            long issued = 0;
            bool ok = true;
            for (int u = cid; u < num_units && ok; u += ncl) {
                int l, tm, tn;
                crt_pair_unit(args, u, l, tm, tn);
                const int row0 = tm * kPairRows + static_cast<int>(rank) * kBM;
                const int col0 = tn * 256 + static_cast<int>(rank) * 128;
                for (int kb = 0; kb < args.num_kb; ++kb) {
                    if (!mbar_wait(&empty[stage], phase ^ 1u, ctl, limit, status)) {
                        ok = false;
                        break;
                    }
                    if (rank == 0) mbar_arrive_expect_tx(&full[stage], 2 * Cfg::kStageBytes);
                    const uint32_t fb = full0 + 8u * static_cast<uint32_t>(stage);
                    tma_load_3d_pair(sA + stage * Cfg::kAStage, &tmA, fb, kb * kBK, row0, l);
                    for (int c = 0; c < 2; ++c)
                        tma_load_3d_pair(sB + stage * Cfg::kBStage + c * Cfg::kBChunk, &tmB, fb,
                                         col0 + c * 64, kb * kBK, l);
                    ++issued;
                    if (++stage == kStages) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) {
                // Let the loads already in flight land before the CTA exits:
                // the even CTA waits on its full barriers (which count both
                // CTAs' loads); the odd CTA, which cannot see them, gives its
                // own at most kStages loads a millisecond.
                CtaCtl local{0};
                if (rank == 0) {
                    const long outstanding = issued < kStages ? issued : kStages;
                    for (long q = 1; q <= outstanding; ++q) {
                        const long idx = issued - q;
                        mbar_wait(&full[idx % kStages], static_cast<uint32_t>((idx / kStages) & 1),
                                  &local, limit, status);
                    }
                } else {
                    const uint64_t t0 = global_timer_ns();
                    while (global_timer_ns() - t0 < 1000000ull) {
                    }
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0 && rank == 0) {
            // ---------------- even CTA: MMA issuer for the pair
            int stage = 0;
            uint32_t phase = 0;
            long cnt = 0;
            bool ok = true;
            for (int u = cid; u < num_units && ok; u += ncl) {
                for (int kb0 = 0; kb0 < args.num_kb && ok; kb0 += kChunkKB, ++cnt) {
                    const int buf = static_cast<int>(cnt & 1);
                    const uint32_t bph = static_cast<uint32_t>((cnt >> 1) & 1);
                    if (!mbar_wait(&tempty[buf], bph ^ 1u, ctl, limit, status)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem_base + static_cast<uint32_t>(buf * 256);
                    const int kb1 = min(args.num_kb, kb0 + kChunkKB);
                    for (int kb = kb0; kb < kb1; ++kb) {
                        if (!mbar_wait(&full[stage], phase, ctl, limit, status)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint64_t adesc =
                            smem_desc_sw128(smem_u32(sA + stage * Cfg::kAStage), 16, 1024);
                        const uint64_t bdesc =
                            smem_desc_sw128(smem_u32(sB + stage * Cfg::kBStage), Cfg::kBChunk, 1024);
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            mma_f16_pair(d, adesc + static_cast<uint64_t>((k * 32) >> 4),
                                         bdesc + static_cast<uint64_t>((k * 16 * 128) >> 4),
                                         Cfg::kIdesc, (kb == kb0 && k == 0) ? 0u : 1u);
                        mma_commit_pair_mc(&empty[stage], 0x3);
                        if (++stage == kStages) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                    if (!ok) break;
                    mma_commit_pair_mc(&tfull[buf], 0x3);
                }
            }
            // Every MMA issued above must finish before either CTA releases
            // TMEM or exits.
            mma_commit_pair(drain);
            CtaCtl local{0};
            mbar_wait(drain, 0, &local, limit, status);
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: quadrant q = warp % 4 (32 rows), column group h
        const int q = warp & 3;
        const int h = (warp - 2) >> 2;
        const uint32_t lane_base = static_cast<uint32_t>(q * 32) << 16;
        const uint32_t tempty0 = rank == 0 ? 0u : mapa_shared(smem_u32(tempty), 0);
        long cnt = 0;
        bool ok = true;
        for (int u = cid; u < num_units && ok; u += ncl) {
            int l, tm, tn;
            crt_pair_unit(args, u, l, tm, tn);
            const float qf = args.qf[l], qinv = args.qinv[l];
            float acc[64];
#pragma unroll
            for (int i = 0; i < 64; ++i) acc[i] = 0.f;
            for (int kb0 = 0; kb0 < args.num_kb; kb0 += kChunkKB, ++cnt) {
                const int buf = static_cast<int>(cnt & 1);
                const uint32_t bph = static_cast<uint32_t>((cnt >> 1) & 1);
                ok = mbar_wait(&tfull[buf], bph, ctl, limit, status);
                if (!__all_sync(0xffffffffu, ok)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t a_base = tmem_base + lane_base + static_cast<uint32_t>(buf * 256 + h * 64);
#pragma unroll
                for (int g = 0; g < 4; ++g) {
                    uint32_t r[16];
                    tmem_ld16(a_base + 16u * g, r);
                    tmem_ld_wait();
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        acc[g * 16 + i] =
                            __fadd_rn(acc[g * 16 + i], mod_reduce(__uint_as_float(r[i]), qf, qinv));
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    if (rank == 0)
                        mbar_arrive(&tempty[buf]);
                    else
                        mbar_arrive_remote(tempty0 + 8u * static_cast<uint32_t>(buf));
                }
            }
            if (!ok) break;
            // the unit's residues in [0, q) as bytes of plane l
            const int64_t row = static_cast<int64_t>(tm) * kPairRows + rank * kBM + q * 32 + lane;
            const int64_t col0 = static_cast<int64_t>(tn) * 256 + h * 64;
            if (row < args.m && col0 < args.p) {
                uint32_t w[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    uint32_t word = 0;
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        float r = mod_reduce(acc[4 * i + b], qf, qinv);   // |r| <= q/2 + 1
                        r = r < 0.f ? __fadd_rn(r, qf) : r;
                        r = r >= qf ? __fsub_rn(r, qf) : r;
                        word |= (__float_as_uint(__fadd_rn(r, 8388608.0f)) & 0xFFu) << (8 * b);
                    }
                    w[i] = word;
                }
                uint8_t* dst = args.R + (static_cast<int64_t>(l) * args.r_rows + row) * args.ldr + col0;
                if (col0 + 64 <= args.ldr) {
#pragma unroll
                    for (int v = 0; v < 4; ++v)
                        reinterpret_cast<uint4*>(dst)[v] =
                            make_uint4(w[4 * v], w[4 * v + 1], w[4 * v + 2], w[4 * v + 3]);
                } else {
                    for (int i = 0; i < 64 && col0 + i < args.ldr; ++i)
                        dst[i] = static_cast<uint8_t>((w[i >> 2] >> (8 * (i & 3))) & 0xFFu);
                }
            }
        }
    }
    __syncthreads();
    cluster_sync_all();   // the pair's MMAs and cross-CTA arrivals are over
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc_pair(tmem_base, Cfg::kTmemCols);
    }
}

// ---------------------------------------------------------------- reconstruction
// mag * 2^e rounded to the nearest FP64 value, ties to even: the top 64 bits
// normalised, the top 53 of them rounded half to even with the rest (and a
// sticky bit for anything below), the FP64 pattern assembled directly (no
// FP64 arithmetic); results outside the normal range go through ldexp (one
// more rounding when subnormal).
__device__ __forceinline__ double u128_to_double_scaled(uint64_t hi, uint64_t lo, int e) {
    uint64_t top;
    bool sticky;
    int e0;   // mag = top * 2^(e0 - 63) + (the sticky part)
    if (hi != 0) {
        const int sh = __clzll(static_cast<long long>(hi));
        top = sh ? (hi << sh) | (lo >> (64 - sh)) : hi;
        sticky = (lo << sh) != 0;
        e0 = 127 - sh;
    } else if (lo != 0) {
        const int sh = __clzll(static_cast<long long>(lo));
        top = lo << sh;
        sticky = false;
        e0 = 63 - sh;
    } else {
        return 0.0;
    }
    uint64_t m53 = top >> 11;                 // in [2^52, 2^53)
    const uint32_t rbits = static_cast<uint32_t>(top & 0x7FFu);
    if (rbits > 0x400u || (rbits == 0x400u && (sticky || (m53 & 1u)))) ++m53;
    int e2 = e + e0 - 52;                      // value = m53 * 2^e2
    if (m53 == (uint64_t(1) << 53)) {
        m53 >>= 1;
        ++e2;
    }
    const int biased = e2 + 52 + 1023;
    if (biased >= 1 && biased <= 2046)
        return __longlong_as_double(static_cast<long long>(
            (static_cast<uint64_t>(biased) << 52) | (m53 & ((uint64_t(1) << 52) - 1))));
    return ldexp(static_cast<double>(m53), e2);
}

// Residues of modulus L for 4 consecutive outputs (w: their bytes, summed
// over the K slices and reduced when there are several), then X += r W_L as
// four 32-bit limbs, each product (r < 2^8 times a limb < 2^32) added in a
// 64-bit sum by one wide multiply-add (16 of them stay below 2^44).
template <int L>
__device__ __forceinline__ void crt_accumulate(const uint32_t (&w)[kCrtMaxModuli], int M,
                                               const CrtConsts& k, uint64_t (&acc)[4][4]) {
    if constexpr (L < kCrtMaxModuli) {
        if (L >= M) return;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const uint32_t r = (w[L] >> (8 * e)) & 0xFFu;
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[e][j] += static_cast<uint64_t>(r) * k.w[L][j];
        }
        crt_accumulate<L + 1>(w, M, k, acc);
    }
}

// The residue bytes of modulus L and its successors, 4 outputs per word:
// the K slices summed and reduced modulo q_L (a compile-time constant).
template <int L>
__device__ __forceinline__ void crt_load(const uint8_t* __restrict__ R, int64_t plane_stride,
                                         int ks, int M, uint32_t (&w)[kCrtMaxModuli]) {
    if constexpr (L < kCrtMaxModuli) {
        if (L >= M) return;
        const uint8_t* src = R + static_cast<int64_t>(L) * ks * plane_stride;
        w[L] = __ldg(reinterpret_cast<const uint32_t*>(src));
        if (ks > 1) {
            constexpr uint32_t q = crt_mod(L);
            uint32_t r[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) r[e] = (w[L] >> (8 * e)) & 0xFFu;
            for (int s = 1; s < ks; ++s) {
                const uint32_t v = __ldg(reinterpret_cast<const uint32_t*>(src + s * plane_stride));
#pragma unroll
                for (int e = 0; e < 4; ++e) r[e] += (v >> (8 * e)) & 0xFFu;
            }
            w[L] = (r[0] % q) | ((r[1] % q) << 8) | ((r[2] % q) << 16) | ((r[3] % q) << 24);
        }
        crt_load<L + 1>(R, plane_stride, ks, M, w);
    }
}

// C[i, j] for 4 consecutive j per thread: r_l = sum_s R[l, s, i, j] mod q_l;
// X = sum_l r_l W_l (four 64-bit limb sums, then carried into 32-bit words;
// X < 2^12 P and P < 2^126, so X has at most 138 bits: words 0..3 hold X mod
// 2^128 and the carry out of word 3 its top bits); the quotient q =
// floor(X / P) estimated in FP32 from floor(X / 2^sP) (off by at most one);
// C' = X - q P (exact modulo 2^128, and within (-P, 2P)) corrected into
// [0, P), then into [-P/2, P/2), rounded once and scaled by
// 2^(eA_i + eB_j - 2t); the FP64 pattern is assembled with integer
// operations only.  The thread takes the groups of 4 outputs g0, g0 + gstep,
// ... of the m x ceil(p / 4) groups.  A residue plane holds r_rows >= m rows
// of ldr bytes.
__device__ __forceinline__ void crt_recon_range(const uint8_t* __restrict__ R, int64_t m, int64_t p,
                                                int64_t ldr, int64_t r_rows, int ks, int t,
                                                const int* __restrict__ eA,
                                                const int* __restrict__ eB,
                                                double* __restrict__ C, int vec,
                                                const CrtConsts& k, int64_t g0, int64_t gstep) {
    const int64_t gpr = (p + 3) / 4;
    const int64_t total = m * gpr;
    const int64_t plane_stride = r_rows * ldr;
    const u128 P = (static_cast<u128>(k.P_hi) << 64) | k.P_lo;
    const u128 halfP = P >> 1;
    // 32-bit index arithmetic by reciprocal when the group count allows
    const bool small = total + gstep < (int64_t(1) << 31);
    const FastDiv fd{static_cast<uint32_t>(gpr),
                     gpr <= 1 ? 0xFFFFFFFFu : static_cast<uint32_t>((uint64_t(1) << 32) / gpr)};
    for (int64_t g = g0; g < total; g += gstep) {
        int64_t i, j0;
        if (small) {
            uint32_t rem;
            i = fdiv(static_cast<uint32_t>(g), fd, rem);
            j0 = static_cast<int64_t>(rem) * 4;
        } else {
            i = g / gpr;
            j0 = (g - i * gpr) * 4;
        }
        uint32_t w[kCrtMaxModuli];
        crt_load<0>(R + i * ldr + j0, plane_stride, ks, k.M, w);
        uint64_t acc[4][4] = {};
        crt_accumulate<0>(w, k.M, k, acc);
        const int ea = eA[i] - 2 * t;
        uint64_t out[4];   // FP64 bit patterns
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            // X = a0 + a1 2^32 + a2 2^64 + a3 2^96 carried into 32-bit words
            // (every partial sum below 2^45); c holds X's bits from 128 up
            const uint64_t a0 = acc[e][0], a1 = acc[e][1], a2 = acc[e][2], a3 = acc[e][3];
            uint64_t v = (a0 >> 32) + (a1 & 0xFFFFFFFFull);
            const uint64_t lo64 = (a0 & 0xFFFFFFFFull) | (v << 32);
            v = (v >> 32) + (a1 >> 32) + (a2 & 0xFFFFFFFFull);
            const uint32_t w2 = static_cast<uint32_t>(v);
            v = (v >> 32) + (a2 >> 32) + (a3 & 0xFFFFFFFFull);
            const uint64_t hi64 = w2 | (v << 32);
            const uint32_t c = static_cast<uint32_t>((v >> 32) + (a3 >> 32));
            // floor(X / 2^sP) < 2^44 (sP >= 64 when P >= 2^96; the carry c is X >> 128)
            uint64_t top;
            if (k.sP >= 64) {
                const int sh = k.sP - 64;
                top = sh == 0 ? hi64 : ((hi64 >> sh) | (static_cast<uint64_t>(c) << (64 - sh)));
            } else {
                top = (hi64 << (64 - k.sP)) | (lo64 >> k.sP);   // X < 2^76 here: no carry
            }
            // fl(top) without a 64-bit conversion (those run on the FP64
            // pipe): top < 2^44 = hi 2^21 + lo with hi < 2^23, lo < 2^21,
            // both exact as floats, joined by one rounding
            const float top_f = __fmaf_rn(small_uint_to_float(static_cast<uint32_t>(top >> 21)),
                                          2097152.0f,
                                          small_uint_to_float(static_cast<uint32_t>(top) & 0x1FFFFFu));
            const uint32_t qe = static_cast<uint32_t>(__float2int_rd(__fmul_rn(top_f, k.kq)));
            // X - qe P modulo 2^128: the true value lies in (-P, 2P), inside the
            // signed 128-bit range
            const uint64_t ql = qe * k.P_lo;
            const uint64_t qh = __umul64hi(static_cast<uint64_t>(qe), k.P_lo) + qe * k.P_hi;
            const u128 x = (static_cast<u128>(hi64) << 64) | lo64;
            i128 rr = static_cast<i128>(x - ((static_cast<u128>(qh) << 64) | ql));
            if (rr < 0) rr += static_cast<i128>(P);
            if (rr >= static_cast<i128>(P)) rr -= static_cast<i128>(P);
            const bool neg = static_cast<u128>(rr) >= halfP;
            const u128 mag = neg ? P - static_cast<u128>(rr) : static_cast<u128>(rr);
            const int64_t j = j0 + e;
            const uint64_t vb =
                j < p ? static_cast<uint64_t>(__double_as_longlong(u128_to_double_scaled(
                            static_cast<uint64_t>(mag >> 64), static_cast<uint64_t>(mag), ea + eB[j])))
                      : 0ull;
            out[e] = vb | (neg ? 0x8000000000000000ull : 0ull);
        }
        uint64_t* crow = reinterpret_cast<uint64_t*>(C + i * p + j0);
        if (vec && j0 + 4 <= p) {
            reinterpret_cast<ulonglong2*>(crow)[0] = make_ulonglong2(out[0], out[1]);
            reinterpret_cast<ulonglong2*>(crow)[1] = make_ulonglong2(out[2], out[3]);
        } else {
            for (int e = 0; e < 4 && j0 + e < p; ++e) crow[e] = out[e];
        }
    }
}

__global__ void __launch_bounds__(256)
    crt_recon_kernel(const uint8_t* __restrict__ R, int64_t m, int64_t p, int64_t ldr,
                     int64_t r_rows, int ks,
                     const int* __restrict__ eA, const int* __restrict__ eB, double* __restrict__ C,
                     int vec, const CrtConsts k) {
    crt_recon_range(R, m, p, ldr, r_rows, ks, k.t, eA, eB, C, vec, k,
                        static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x,
                        static_cast<int64_t>(gridDim.x) * blockDim.x);
}

// ---------------------------------------------------------------- grouped launches
// One problem of a grouped call, as the pre-pass and reconstruction launches
// see it: operands, its workspace region, and the block range it owns in
// each launch (blocks [*_begin, *_begin + *_blocks)).
struct CrtGPass {
    const void* A;
    const void* B;
    double* C;
    int64_t m, n, p, lda, ldb, ldr, a_plane, b_plane, gx, chunk;
    __nv_bfloat16* a_pl;
    __nv_bfloat16* b_pl;
    int* eA;
    int* eB;
    void* cmax;
    const uint8_t* R;
    int* status;   // where this problem's non-finite inputs are recorded
    int M, t, va, vb, vec_c, f64in;
    int exps_begin, rblocks, cblocks;
    int res_begin, ga, gb;
    int rec_begin, rec_blocks;
};

// The problem whose block range of a launch holds block b (begin(i) ascending).
template <typename F>
__device__ __forceinline__ int find_owner(int count, int b, F begin) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (begin(mid) <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Grouped exponent pass over the problems of one input type.
template <typename T>
__global__ void __launch_bounds__(256)
    crt_g_exps_kernel(const CrtGPass* __restrict__ pr, int count) {
    const int b = static_cast<int>(blockIdx.x);
    const int g = find_owner(count, b, [&](int i) { return pr[i].exps_begin; });
    const CrtGPass& x = pr[g];
    const int local = b - x.exps_begin;
    using U = typename Bits<T>::U;
    if (local < x.rblocks)
        crt_row_exp_part(static_cast<const T*>(x.A), x.m, x.n, x.eA, x.status, local, x.rblocks);
    else if (local < x.rblocks + x.cblocks)
        crt_col_max_part(static_cast<const T*>(x.B), x.n, x.p, x.chunk, static_cast<U*>(x.cmax),
                         local - x.rblocks, x.gx);
}

// Grouped residue pass over the problems of one input type.
template <typename T>
__global__ void __launch_bounds__(256)
    crt_g_residue_kernel(const CrtGPass* __restrict__ pr, int count, const CrtPow2 pow2) {
    // tab[l * 64 + s] = (2^s mod q_l, 2^(s+12) mod q_l): a row per modulus, so
    // threads of a warp that read different s of one row mostly hit different banks
    __shared__ float2 tab[kCrtMaxModuli * 64];
    for (int i = threadIdx.x; i < kCrtMaxModuli * 64; i += blockDim.x)
        tab[i] = make_float2(static_cast<float>(pow2.v[i / 64][i % 64]),
                             static_cast<float>(pow2.v[i / 64][i % 64 + 12]));
    __syncthreads();
    const int b = static_cast<int>(blockIdx.x);
    const int g = find_owner(count, b, [&](int i) { return pr[i].res_begin; });
    const CrtGPass& x = pr[g];
    const int local = b - x.res_begin;
    using U = typename Bits<T>::U;
    if (local < x.ga)
        crt_residue_part<T, 0>(static_cast<const T*>(x.A), x.m, x.n, x.lda, x.eA, nullptr,
                               x.status, x.t, x.M, x.va, tab, x.a_pl, x.a_plane, local, x.ga);
    else if (local < x.ga + x.gb)
        crt_residue_part<T, 1>(static_cast<const T*>(x.B), x.n, x.p, x.ldb, x.eB,
                               static_cast<const U*>(x.cmax), x.status, x.t, x.M, x.vb, tab,
                               x.b_pl, x.b_plane, local - x.ga, x.gb);
}

// Grouped reconstruction: each block serves one problem, with that problem's
// CRT constants (consts[M - kCrtMinModuli]) copied to shared memory.
__global__ void __launch_bounds__(256)
    crt_g_recon_kernel(const CrtGPass* __restrict__ pr, int count,
                       const CrtConsts* __restrict__ consts) {
    __shared__ CrtConsts k;
    const int b = static_cast<int>(blockIdx.x);
    const int g = find_owner(count, b, [&](int i) { return pr[i].rec_begin; });
    const CrtGPass& x = pr[g];
    {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(consts + (x.M - kCrtMinModuli));
        uint32_t* dst = reinterpret_cast<uint32_t*>(&k);
        for (int i = threadIdx.x; i < static_cast<int>(sizeof(CrtConsts) / 4); i += blockDim.x)
            dst[i] = src[i];
    }
    __syncthreads();
    crt_recon_range(x.R, x.m, x.p, x.ldr, x.m, 1, x.t, x.eA, x.eB, x.C, x.vec_c, k,
                       static_cast<int64_t>(b - x.rec_begin) * blockDim.x + threadIdx.x,
                       static_cast<int64_t>(x.rec_blocks) * blockDim.x);
}

// Rows per block of the column-maximum pass: enough blocks to spread over
// the SMs (about 8 per SM), 16 .. 256 rows each.
int64_t colmax_chunk(int64_t n, int64_t p, long sms) {
    const int64_t gx = ceil_div(p, 256);
    const int64_t want = ceil_div(n * gx, 8 * sms);
    return std::max<int64_t>(16, std::min<int64_t>(256, want));
}

int grid_for(int64_t total, int threads) {
    const int64_t want = ceil_div(total, threads);
    const int64_t cap = 16L * num_sms();
    return static_cast<int>(std::max<int64_t>(1, std::min(want, cap)));
}

int vec_rows(const void* X, int64_t cols, int per16) {
    return (cols % per16 == 0) && (reinterpret_cast<uintptr_t>(X) % 16 == 0);
}

// Most K slices per tile the workspace is sized for.
constexpr int kCrtMaxKs = 8;
// Reference SM count of the workspace sizing (the launch uses the device's).
constexpr int kCrtRefSms = 160;

// K slices for `units` (modulus x tile) units over `sms` SMs: cut K only
// when the units fill at most half of the SMs, keeping >= 4 chunks a slice.
int crt_ks(long units, int num_kb, long sms) {
    if (units * 2 > sms) return 1;
    const long by_sms = (sms + units - 1) / units;
    const long by_k = std::max(1L, static_cast<long>(num_kb) / (4 * kChunkKB));
    return static_cast<int>(std::max(1L, std::min({by_sms, by_k, static_cast<long>(kCrtMaxKs)})));
}

// Tile width by a wave-count cost model over (modulus, tile) units: the
// cheapest of ceil(units / SMs) waves of width / efficiency (128-wide tiles
// at 0.9 of 256-wide ones); moa_set_block_n(128 | 256) forces it.
int crt_block_n(int64_t m, int64_t p, int M, long sms) {
    const int ov = tile_override();
    if (ov == 128 || ov == 256) return ov;
    auto cost = [&](int bn, double eff) {
        const long units = M * ceil_div(m, kBM) * ceil_div(p, bn);
        return static_cast<double>((units + sms - 1) / sms) * bn / eff;
    };
    return cost(128, 0.9) < cost(256, 1.0) ? 128 : 256;
}

// Tile shape of a single modular-slice GEMM: 128-row tiles of width 128 or
// 256 on one SM, or 256 x 256 tiles on a CTA pair.  Wave-count cost model:
// ceil(units / slots) waves, each as long as one SM's share of a unit (a
// 128 x bn block) divided by the shape's efficiency (measured: 128 x 256 at
// 0.9 of the pair's rate, 128 x 128 at 0.9 of that).  Pair tiles only while
// one modulus plane of A (m x n) and of B (n x p) each fit in the L2: beyond
// that the pair kernel reads more from DRAM and, under the power cap, runs
// slower (measured, FP32 inputs, square N: pair 0.362 vs 0.386 ms at 2048,
// 5.66 vs 5.76 ms at 6144, even at 8192, 47-48 vs 44 ms at 12288).  K-sliced
// launches (few units) stay on one SM.  moa_set_block_m / moa_set_block_n
// force it.
struct CrtTiles {
    int rows, bn;
};
CrtTiles crt_tile_plan(int64_t m, int64_t n, int64_t p, int M, int ks, long sms, long clusters,
                       int64_t l2_bytes) {
    const int ov_m = tile_m_override(), ov_n = tile_override();
    const int bn1 = crt_block_n(m, p, M, sms);
    if (ks != 1 || ov_n == 128 || ov_m == 128 || clusters < 1) return {kBM, bn1};
    if (ov_m == 256) return {2 * kBM, 256};
    if (2 * std::max(m, p) * n > l2_bytes) return {kBM, bn1};
    const long units2 = M * ceil_div(m, 2 * kBM) * ceil_div(p, 256);
    const double c_pair = static_cast<double>((units2 + clusters - 1) / clusters) * 256.0;
    const long units1 = M * ceil_div(m, kBM) * ceil_div(p, bn1);
    const double eff1 = bn1 == 256 ? 0.9 : 0.81;
    const double c_one = static_cast<double>((units1 + sms - 1) / sms) * bn1 / eff1;
    return c_pair <= c_one ? CrtTiles{2 * kBM, 256} : CrtTiles{kBM, bn1};
}

// The device's L2 size in bytes (cached per device).
int64_t l2_bytes() {
    static std::atomic<int64_t> cache[64];
    int d = -1;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= 64) return 0;
    int64_t v = cache[d].load(std::memory_order_acquire);
    if (v == 0) {
        int b = 0;
        if (cudaDeviceGetAttribute(&b, cudaDevAttrL2CacheSize, d) != cudaSuccess || b <= 0) return 0;
        v = b;
        cache[d].store(v, std::memory_order_release);
    }
    return v;
}

// Clusters of the pair kernel that fit on the device at once (0 when the
// query fails: the one-SM kernels are used).
long crt_pair_clusters() {
    static std::atomic<long> cache[64];
    int d = -1;
    if (cudaGetDevice(&d) != cudaSuccess) d = -1;
    if (d >= 0 && d < 64 && cache[d].load(std::memory_order_acquire) != 0)
        return cache[d].load(std::memory_order_acquire);
    static std::atomic<uint64_t> attr_done{0};
    if (smem_attr_once(reinterpret_cast<const void*>(crt_gemm_pair_kernel), CrtPairCfg::kSmem,
                       attr_done, "cudaFuncSetAttribute(crt_gemm_pair)") != MOA_OK)
        return 0;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(2 * static_cast<unsigned>(num_sms()), 1, 1);
    cfg.blockDim = dim3(CrtPairCfg::kThreads, 1, 1);
    cfg.dynamicSmemBytes = CrtPairCfg::kSmem;
    int n = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&n, crt_gemm_pair_kernel, &cfg);
    if (e != cudaSuccess || n < 1) {
        cudaGetLastError();
        log_msg(1, "crt pair kernel: cluster occupancy query failed (%s); one-SM tiles only",
                e != cudaSuccess ? cudaGetErrorString(e) : "no cluster fits");
        return 0;
    }
    if (d >= 0 && d < 64) cache[d].store(n, std::memory_order_release);
    return n;
}

int launch_crt_pair(const CrtGemmArgs& a, const CUtensorMap& tmA, const CUtensorMap& tmB,
                    long clusters, cudaStream_t s, moa_stats* st) {
    using Cfg = CrtPairCfg;
    const long units = static_cast<long>(a.M) * a.tiles_m * a.tiles_n;
    const int grid = 2 * static_cast<int>(std::min<long>(units, clusters));
    prof_begin(s);
    crt_gemm_pair_kernel<<<grid, Cfg::kThreads, Cfg::kSmem, s>>>(tmA, tmB, a);
    cudaError_t e = cudaGetLastError();
    prof_end(s);
    if (e != cudaSuccess) return cuda_fail(e, "crt_gemm_pair_kernel launch");
    log_msg(2, "crt m=%lld n=%lld p=%lld tile 256x256 (CTA pairs) moduli %d units %ld grid %d",
            static_cast<long long>(a.m), static_cast<long long>(a.n), static_cast<long long>(a.p),
            a.M, units, grid);
    if (st) {
        st->block_m = 2 * kBM;
        st->block_n = 256;
        st->block_k = kBK;
        st->grid = grid;
        st->tiles = static_cast<int64_t>(a.tiles_m) * a.tiles_n;
    }
    return MOA_OK;
}

template <int BN, bool GROUPED = false>
int launch_crt_gemm(const CrtGemmArgs& a, const CUtensorMap& tmA, const CUtensorMap& tmB,
                    cudaStream_t s, moa_stats* st) {
    using Cfg = CrtCfg<BN>;
    static std::atomic<uint64_t> attr_done{0};
    int rc = smem_attr_once(reinterpret_cast<const void*>(crt_gemm_kernel<BN, GROUPED>), Cfg::kSmem,
                            attr_done, "cudaFuncSetAttribute(crt_gemm)");
    if (rc != MOA_OK) return rc;
    const long units =
        GROUPED ? a.num_units : static_cast<long>(a.M) * a.tiles_m * a.tiles_n * a.ks;
    const int grid = static_cast<int>(std::min<long>(units, num_sms()));
    prof_begin(s);
    crt_gemm_kernel<BN, GROUPED><<<grid, Cfg::kThreads, Cfg::kSmem, s>>>(tmA, tmB, a);
    cudaError_t e = cudaGetLastError();
    prof_end(s);
    if (e != cudaSuccess) return cuda_fail(e, "crt_gemm_kernel launch");
    log_msg(2, "crt m=%lld n=%lld p=%lld tile %dx%d moduli %d K slices %d units %ld grid %d",
            static_cast<long long>(a.m), static_cast<long long>(a.n), static_cast<long long>(a.p),
            kBM, BN, a.M, a.ks, units, grid);
    if (st) {
        st->block_m = kBM;
        st->block_n = BN;
        st->block_k = kBK;
        st->grid = grid;
        st->tiles = static_cast<int64_t>(a.tiles_m) * a.tiles_n;
    }
    return MOA_OK;
}

}  // namespace

int crt_moduli_for(moa_dtype dt, int64_t n, int slices) {
    (void)dt;
    if (slices != 0) return (slices < kCrtMinModuli || slices > kCrtMaxModuli) ? -1 : slices;
    // the fewest moduli, from 14, that keep t >= 47 bits per operand
    for (int M = kCrtDefaultModuli; M < kCrtMaxModuli; ++M)
        if (crt_bits(std::max<int64_t>(n, 1), M) >= 47) return M;
    return kCrtMaxModuli;
}

int crt_bits(int64_t n, int M) {
    const u128 P = crt_product(M);
    int best = -1;
    for (int t = 0; t <= 62; ++t) {
        // n * 2^(2t+1) < P
        const int sh = 2 * t + 1;
        if (sh >= 127) break;
        const u128 lhs = static_cast<u128>(n) << sh;
        if ((lhs >> sh) != static_cast<u128>(n) || lhs >= P) break;
        best = t;
    }
    return best;
}

CrtLayout crt_layout(int64_t m, int64_t n, int64_t p, int M) {
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    CrtLayout L{};
    L.M = M;
    L.lda = round_up(n, 8);
    L.ldb = round_up(p, 8);
    L.ldr = round_up(p, 16);
    const long tiles128 = static_cast<long>(ceil_div(m, kBM) * ceil_div(p, 128));
    L.ks_max = crt_ks(static_cast<long>(M) * tiles128, static_cast<int>(ceil_div(n, kBK)),
                      kCrtRefSms);
    size_t off = 0;
    L.a_off = off;
    off += al(static_cast<size_t>(M) * m * L.lda * 2);
    L.b_off = off;
    off += al(static_cast<size_t>(M) * n * L.ldb * 2);
    L.ea_off = off;
    off += al(static_cast<size_t>(m) * 4);
    L.eb_off = off;
    off += al(static_cast<size_t>(p) * 4);
    L.cmax_off = off;
    off += al(static_cast<size_t>(p) * 8);
    L.r_off = off;
    off += al(static_cast<size_t>(M) * L.ks_max * m * L.ldr);
    L.total = off;
    return L;
}

size_t crt_workspace_bytes(int64_t m, int64_t n, int64_t p, moa_dtype dt, int slices) {
    const int M = crt_moduli_for(dt, n, slices);
    if (M < 0) return 0;
    return crt_layout(m, n, p, M).total;
}

namespace {

// One modular-slice GEMM's constants and workspace regions.
struct CrtCall {
    int64_t m, n, p;
    int M, t;
    bool f64in;
    CrtLayout L;
    __nv_bfloat16* a_pl;
    __nv_bfloat16* b_pl;
    int* eA;
    int* eB;
    void* cmax;
    uint8_t* R;
    int64_t a_plane, b_plane;   // elements a residue plane of A (m rows) and of B
    int* status;
    CrtPow2 pow2;
};

int crt_setup(int64_t m, int64_t n, int64_t p, moa_dtype dt, int slices, void* ws,
              size_t ws_bytes, CrtCall& c) {
    c.m = m;
    c.n = n;
    c.p = p;
    c.M = crt_moduli_for(dt, n, slices);
    if (c.M < 0) return fail(MOA_ERR_DTYPE, "modulus count not supported (8..16)");
    c.t = crt_bits(n, c.M);
    if (c.t < 1) return fail(MOA_ERR_ARG, "n too large for this modulus count");
    c.L = crt_layout(m, n, p, c.M);
    if (ws_bytes < c.L.total) return fail(MOA_ERR_WORKSPACE, "workspace too small for crt mode");
    if (ceil_div(n, 256) * ceil_div(p, 256) > (1L << 30))
        return fail(MOA_ERR_ARG, "n x p too large for the column-max grid");
    c.status = launch_status_ptr();
    if (!c.status) return MOA_ERR_CUDA;
    uint8_t* base = static_cast<uint8_t*>(ws);
    c.a_pl = reinterpret_cast<__nv_bfloat16*>(base + c.L.a_off);
    c.b_pl = reinterpret_cast<__nv_bfloat16*>(base + c.L.b_off);
    c.eA = reinterpret_cast<int*>(base + c.L.ea_off);
    c.eB = reinterpret_cast<int*>(base + c.L.eb_off);
    c.cmax = base + c.L.cmax_off;
    c.R = base + c.L.r_off;
    c.a_plane = m * c.L.lda;
    c.b_plane = n * c.L.ldb;
    c.f64in = dt == MOA_F64_CRT_F64IN;
    for (int l = 0; l < kCrtMaxModuli; ++l)
        for (int e2 = 0; e2 < kPow2Cols; ++e2)
            c.pow2.v[l][e2] = static_cast<uint8_t>(
                (e2 < 128 ? (static_cast<u128>(1) << e2) % crt_mod(l) : 0));
    return MOA_OK;
}

// Exponents and residue planes of rows [r0, r0 + mb) of A (A0: A's row r0;
// mb = 0: none) and, when B is not NULL, of all of B (its column maxima
// cleared first).  Two launches (a memset before them when B is taken).
int crt_passes(const CrtCall& c, const void* A0, int64_t r0, int64_t mb, const void* B,
               cudaStream_t s) {
    const int64_t n = c.n, p = c.p;
    if (B) {
        cudaError_t e = cudaMemsetAsync(c.cmax, 0, static_cast<size_t>(p) * 8, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(colmax)");
    }
    const int64_t rblocks = mb > 0 ? std::min<int64_t>(ceil_div(mb, 8), 16L * num_sms()) : 0;
    const int64_t chunk = colmax_chunk(n, p, num_sms());
    const int64_t gx = ceil_div(p, 256);
    const int64_t cblocks = B ? gx * ceil_div(n, chunk) : 0;
    const int ga = mb > 0 ? grid_for(mb * c.L.lda / 4, 256) : 0;
    const int gb = B ? grid_for(c.b_plane / 4, 256) : 0;
    if (rblocks + cblocks == 0) return MOA_OK;
    int* eA = c.eA + r0;
    __nv_bfloat16* a_out = c.a_pl + r0 * c.L.lda;
    if (c.f64in) {
        const double* Ad = static_cast<const double*>(A0);
        const double* Bd = static_cast<const double*>(B);
        auto* cm = static_cast<unsigned long long*>(c.cmax);
        crt_exps_kernel<double><<<static_cast<unsigned>(rblocks + cblocks), 256, 0, s>>>(
            Ad, mb, n, Bd, p, chunk, eA, cm, c.status, static_cast<int>(rblocks), gx);
        crt_residue_kernel<double><<<ga + gb, 256, 0, s>>>(
            Ad, mb, n, c.L.lda, mb > 0 ? vec_rows(Ad, n, 2) : 0, eA, Bd, p, c.L.ldb,
            B ? vec_rows(Bd, p, 2) : 0, c.eB, cm, c.status, c.t, c.M, a_out, c.a_plane, c.b_pl,
            c.b_plane, ga, c.pow2);
    } else {
        const float* Af = static_cast<const float*>(A0);
        const float* Bf = static_cast<const float*>(B);
        auto* cm = static_cast<unsigned int*>(c.cmax);
        crt_exps_kernel<float><<<static_cast<unsigned>(rblocks + cblocks), 256, 0, s>>>(
            Af, mb, n, Bf, p, chunk, eA, cm, c.status, static_cast<int>(rblocks), gx);
        crt_residue_kernel<float><<<ga + gb, 256, 0, s>>>(
            Af, mb, n, c.L.lda, mb > 0 ? vec_rows(Af, n, 4) : 0, eA, Bf, p, c.L.ldb,
            B ? vec_rows(Bf, p, 4) : 0, c.eB, cm, c.status, c.t, c.M, a_out, c.a_plane, c.b_pl,
            c.b_plane, ga, c.pow2);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MOA_OK : cuda_fail(e, "crt pre-pass launch");
}

// The residue GEMM and the reconstruction of rows [r0, r0 + mb) into C0
// (C's row r0), from residue planes that crt_passes wrote.  Two launches.
int crt_product(const CrtCall& c, int64_t r0, int64_t mb, double* C0, cudaStream_t s,
                moa_stats* st) {
    const int64_t n = c.n, p = c.p;
    const int M = c.M;
    const CrtLayout& L = c.L;
    const long sms = num_sms();
    const int bn1 = crt_block_n(mb, p, M, sms);
    const int ks = std::min(L.ks_max, crt_ks(static_cast<long>(M) * ceil_div(mb, kBM) *
                                                 ceil_div(p, bn1),
                                             static_cast<int>(ceil_div(n, kBK)), sms));
    const long clusters = ks == 1 ? crt_pair_clusters() : 0;
    const CrtTiles tiles = crt_tile_plan(mb, n, p, M, ks, sms, clusters, l2_bytes());
    const bool pair = tiles.rows == 2 * kBM;
    const int bn = tiles.bn;
    uint8_t* R0 = c.R + r0 * L.ldr;
    CrtGemmArgs a{};
    a.R = R0;
    a.m = mb;
    a.n = n;
    a.p = p;
    a.ldr = L.ldr;
    a.r_rows = c.m;
    a.tiles_m = static_cast<int>(ceil_div(mb, tiles.rows));
    a.tiles_n = static_cast<int>(ceil_div(p, bn));
    a.num_kb = static_cast<int>(ceil_div(n, kBK));
    // the same number of tile rows a raster group either way: twice the
    // output rows for pair tiles (measured: 16 pair rows a group hold their
    // own against 16 one-SM rows at 8192^2 under the power cap; 8 lose ~2%)
    a.group_m = split_raster_group(n);
    a.M = M;
    a.ks = ks;
    for (int l = 0; l < M; ++l) {
        a.qf[l] = static_cast<float>(crt_mod(l));
        a.qinv[l] = 1.0f / static_cast<float>(crt_mod(l));
    }
    a.wait_limit_ns = wait_limit_ns();
    a.status = c.status;
    CUtensorMap tmA, tmB;
    int rc = make_tmap_3d(&tmA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, c.a_pl + r0 * L.lda,
                          static_cast<uint64_t>(n), static_cast<uint64_t>(mb),
                          static_cast<uint64_t>(M), static_cast<uint64_t>(L.lda) * 2,
                          static_cast<uint64_t>(c.a_plane) * 2, kBK, kBM);
    if (rc != MOA_OK) return rc;
    rc = make_tmap_3d(&tmB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, c.b_pl, static_cast<uint64_t>(p),
                      static_cast<uint64_t>(n), static_cast<uint64_t>(M),
                      static_cast<uint64_t>(L.ldb) * 2, static_cast<uint64_t>(c.b_plane) * 2, 64,
                      kBK);
    if (rc != MOA_OK) return rc;
    rc = pair ? launch_crt_pair(a, tmA, tmB, clusters, s, st)
         : bn == 256 ? launch_crt_gemm<256>(a, tmA, tmB, s, st)
                     : launch_crt_gemm<128>(a, tmA, tmB, s, st);
    if (rc != MOA_OK) return rc;

    const CrtConsts k = crt_consts(M, c.t);
    const int vec = (p % 2 == 0) && (reinterpret_cast<uintptr_t>(C0) % 16 == 0);
    const int rgrid = grid_for(mb * ceil_div(p, 4), 256);
    crt_recon_kernel<<<rgrid, 256, 0, s>>>(R0, mb, p, L.ldr, c.m, a.ks, c.eA + r0, c.eB, C0, vec,
                                           k);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "crt reconstruction launch");
    if (st) {
        st->slices = M;
        st->products = M;
    }
    return MOA_OK;
}

}  // namespace

int crt_gemm(int64_t m, int64_t n, int64_t p, moa_dtype dt, const void* A, const void* B, void* C,
             int slices, void* ws, size_t ws_bytes, cudaStream_t s, moa_stats* st) {
    CrtCall c;
    int rc = crt_setup(m, n, p, dt, slices, ws, ws_bytes, c);
    if (rc != MOA_OK) return rc;
    // launches: clear the column maxima (a memset), row exponents of A beside
    // the column maxima of B, residue planes of A and B, the residue GEMM,
    // the reconstruction
    rc = crt_passes(c, A, 0, m, B, s);
    if (rc != MOA_OK) return rc;
    rc = crt_product(c, 0, m, static_cast<double*>(C), s, st);
    if (rc != MOA_OK) return rc;
    if (st) st->kernels = 4;
    return MOA_OK;
}

int crt_gemm_host(int64_t m, int64_t n, int64_t p, moa_dtype dt, const void* hA, const void* hB,
                  void* hC, int slices, void* dA, void* dB, void* dC, void* ws, size_t ws_bytes,
                  cudaStream_t s, moa_stats* st) {
    CrtCall c;
    int rc = crt_setup(m, n, p, dt, slices, ws, ws_bytes, c);
    if (rc != MOA_OK) return rc;
    const size_t in_b = c.f64in ? 8 : 4;
    // bands of about 2048 rows (at most 8), 256-row multiples
    const int64_t want = std::min<int64_t>(8, std::max<int64_t>(1, ceil_div(m, 2048)));
    const int64_t mb = round_up(ceil_div(m, want), 256);
    const int64_t nb = ceil_div(m, mb);
    if (nb == 1) {
        // one band: nothing to overlap within the call; upload, compute and
        // download in order on the caller's stream (no helper streams)
        cudaError_t e = cudaMemcpyAsync(dA, hA, static_cast<size_t>(m) * n * in_b,
                                        cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dB, hB, static_cast<size_t>(n) * p * in_b, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(A, B to the device)");
        rc = crt_passes(c, dA, 0, m, dB, s);
        if (rc == MOA_OK) rc = crt_product(c, 0, m, static_cast<double*>(dC), s, st);
        if (rc != MOA_OK) return rc;
        e = cudaMemcpyAsync(hC, dC, static_cast<size_t>(m) * p * 8, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(C to the host)");
        if (st) st->kernels = 4;
        return MOA_OK;
    }
    cudaStream_t up = nullptr, down = nullptr;
    std::vector<cudaEvent_t> ev;   // start, b_ready, a_ready[nb], c_ready[nb], up_done, down_done
    auto mk = [&]() {
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return false;
        ev.push_back(e);
        return true;
    };
    bool ok = cudaStreamCreateWithFlags(&up, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&down, cudaStreamNonBlocking) == cudaSuccess;
    for (int64_t i = 0; ok && i < 2 * nb + 4; ++i) ok = mk();
    // Whatever happens below, the caller's stream ends after both helper
    // streams' work, so the workspace and host buffers stay in use until then.
    auto finish = [&](int status) {
        if (up && ev.size() == static_cast<size_t>(2 * nb + 4)) {
            cudaEventRecord(ev[2 * nb + 2], up);
            cudaEventRecord(ev[2 * nb + 3], down);
            cudaStreamWaitEvent(s, ev[2 * nb + 2], 0);
            cudaStreamWaitEvent(s, ev[2 * nb + 3], 0);
        }
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        if (up) cudaStreamDestroy(up);
        if (down) cudaStreamDestroy(down);
        return status;
    };
    if (!ok) return finish(fail(MOA_ERR_CUDA, "stream / event creation for moa_gemm_host"));
    cudaEvent_t start = ev[0], b_ready = ev[1];
    cudaEvent_t* a_ready = ev.data() + 2;
    cudaEvent_t* c_ready = ev.data() + 2 + nb;
    if (cudaEventRecord(start, s) != cudaSuccess || cudaStreamWaitEvent(up, start, 0) != cudaSuccess ||
        cudaStreamWaitEvent(down, start, 0) != cudaSuccess)
        return finish(fail(MOA_ERR_CUDA, "moa_gemm_host stream order"));
    // uploads: all of B, then A band by band
    if (cudaMemcpyAsync(dB, hB, static_cast<size_t>(n) * p * in_b, cudaMemcpyHostToDevice, up) !=
            cudaSuccess ||
        cudaEventRecord(b_ready, up) != cudaSuccess)
        return finish(fail(MOA_ERR_CUDA, "cudaMemcpyAsync(B to the device)"));
    for (int64_t i = 0; i < nb; ++i) {
        const int64_t r0 = i * mb, rows = std::min(mb, m - r0);
        const size_t off = static_cast<size_t>(r0) * n * in_b;
        if (cudaMemcpyAsync(static_cast<uint8_t*>(dA) + off, static_cast<const uint8_t*>(hA) + off,
                            static_cast<size_t>(rows) * n * in_b, cudaMemcpyHostToDevice,
                            up) != cudaSuccess ||
            cudaEventRecord(a_ready[i], up) != cudaSuccess)
            return finish(fail(MOA_ERR_CUDA, "cudaMemcpyAsync(A band to the device)"));
    }
    // compute on the caller's stream: B's passes once, then band by band
    int kernels = 0;
    if (cudaStreamWaitEvent(s, b_ready, 0) != cudaSuccess)
        return finish(fail(MOA_ERR_CUDA, "moa_gemm_host stream order"));
    rc = crt_passes(c, nullptr, 0, 0, dB, s);
    if (rc != MOA_OK) return finish(rc);
    kernels += 2;
    for (int64_t i = 0; i < nb; ++i) {
        const int64_t r0 = i * mb, rows = std::min(mb, m - r0);
        if (cudaStreamWaitEvent(s, a_ready[i], 0) != cudaSuccess)
            return finish(fail(MOA_ERR_CUDA, "moa_gemm_host stream order"));
        rc = crt_passes(c, static_cast<const uint8_t*>(dA) + static_cast<size_t>(r0) * n * in_b,
                        r0, rows, nullptr, s);
        if (rc != MOA_OK) return finish(rc);
        double* C0 = static_cast<double*>(dC) + r0 * p;
        rc = crt_product(c, r0, rows, C0, s, st);
        if (rc != MOA_OK) return finish(rc);
        kernels += 4;
        if (cudaEventRecord(c_ready[i], s) != cudaSuccess)
            return finish(fail(MOA_ERR_CUDA, "moa_gemm_host stream order"));
        // download of the band as soon as it is reconstructed
        if (cudaStreamWaitEvent(down, c_ready[i], 0) != cudaSuccess ||
            cudaMemcpyAsync(static_cast<double*>(hC) + r0 * p, C0,
                            static_cast<size_t>(rows) * p * 8, cudaMemcpyDeviceToHost,
                            down) != cudaSuccess)
            return finish(fail(MOA_ERR_CUDA, "cudaMemcpyAsync(C band to the host)"));
    }
    if (st) {
        st->kernels = kernels;
        st->slices = c.M;
        st->products = c.M;
    }
    return finish(MOA_OK);
}

// ---------------------------------------------------------------- grouped host side
namespace {

struct GroupedPlan {
    size_t consts_off, pass_off, prob_off, maps_off, head_bytes;   // tables, one upload
    size_t cmax_off, cmax_bytes;                                     // one memset
    std::vector<size_t> region;   // per taken problem: its region in the workspace
    size_t total;
};

struct Taken {
    int idx;          // index in the caller's descriptors
    int M, t, bn;
    CrtLayout L;      // offsets within the problem's region (cmax unused)
};

// The problems this path takes, F32-input ones first, and the workspace plan.
GroupedPlan grouped_plan(int count, const moa_gemm_desc* d, std::vector<Taken>* taken) {
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    std::vector<Taken> tk;
    for (int pass = 0; pass < 2; ++pass)
        for (int g = 0; g < count; ++g) {
            if (!crt_grouped_ok(d[g])) continue;
            if ((d[g].dt == MOA_F64_CRT_F64IN) != (pass == 1)) continue;
            Taken x{};
            x.idx = g;
            x.M = crt_moduli_for(d[g].dt, d[g].n, 0);
            x.t = crt_bits(d[g].n, x.M);
            x.L = crt_layout(d[g].m, d[g].n, d[g].p, x.M);
            tk.push_back(x);
        }
    const size_t G = tk.size();
    GroupedPlan P{};
    size_t off = 0;
    P.consts_off = off;
    off += al(sizeof(CrtConsts) * (kCrtMaxModuli - kCrtMinModuli + 1));
    P.pass_off = off;
    off += al(sizeof(CrtGPass) * G);
    P.prob_off = off;
    off += al(sizeof(CrtGProb) * G);
    P.maps_off = off;
    off += al(sizeof(CUtensorMap) * 2 * G);
    P.head_bytes = off;
    P.cmax_off = off;
    for (const Taken& x : tk) off += al(static_cast<size_t>(d[x.idx].p) * 8);
    P.cmax_bytes = off - P.cmax_off;
    for (const Taken& x : tk) {
        P.region.push_back(off);
        // the single-call layout without its column-max block and with one K slice
        off += al(x.L.r_off + static_cast<size_t>(x.M) * d[x.idx].m * x.L.ldr);
    }
    P.total = G ? off : 0;
    if (taken) *taken = tk;
    return P;
}

}  // namespace

bool crt_grouped_ok(const moa_gemm_desc& d) {
    const int64_t lim = int64_t(1) << 31;
    return is_crt(d.dt) && d.m > 0 && d.n > 0 && d.p > 0 && d.m < lim && d.n < lim && d.p < lim &&
           reinterpret_cast<uintptr_t>(d.A) % 16 == 0 && reinterpret_cast<uintptr_t>(d.B) % 16 == 0 &&
           reinterpret_cast<uintptr_t>(d.C) % 8 == 0 && d.C != nullptr &&
           crt_moduli_for(d.dt, d.n, 0) > 0 && crt_bits(d.n, crt_moduli_for(d.dt, d.n, 0)) >= 1 &&
           ceil_div(d.n, 256) * ceil_div(d.p, 256) <= (1L << 30);
}

size_t crt_grouped_workspace(int count, const moa_gemm_desc* d) {
    return grouped_plan(count, d, nullptr).total;
}

int crt_grouped_launch(int count, const moa_gemm_desc* d, void* ws, size_t ws_bytes,
                       cudaStream_t s, int* const* status_of) {
    std::vector<Taken> tk;
    const GroupedPlan P = grouped_plan(count, d, &tk);
    const int G = static_cast<int>(tk.size());
    if (G == 0) return MOA_OK;
    if (ws == nullptr || ws_bytes < P.total)
        return fail(MOA_ERR_WORKSPACE, "workspace too small for the grouped modular-slice path");
    int* status = launch_status_ptr();
    if (!status) return MOA_ERR_CUDA;
    const long sms = num_sms();
    uint8_t* base = static_cast<uint8_t*>(ws);
    int slot = 0;
    uint8_t* host = static_cast<uint8_t*>(staging_get(P.head_bytes, &slot));
    if (!host) return fail(MOA_ERR_CUDA, "pinned staging buffer unavailable");
    std::memset(host, 0, P.head_bytes);
    auto* consts = reinterpret_cast<CrtConsts*>(host + P.consts_off);
    for (int M = kCrtMinModuli; M <= kCrtMaxModuli; ++M) consts[M - kCrtMinModuli] = crt_consts(M, 0);
    auto* pass = reinterpret_cast<CrtGPass*>(host + P.pass_off);
    auto* probs = reinterpret_cast<CrtGProb*>(host + P.prob_off);
    auto* maps = reinterpret_cast<CUtensorMap*>(host + P.maps_off);

    // pre-pass and reconstruction tables (F32-input problems first)
    int n32 = 0;
    int exps_pos[2] = {0, 0}, res_pos[2] = {0, 0}, rec_pos = 0;
    size_t cmax_pos = P.cmax_off;
    for (int i = 0; i < G; ++i) {
        const Taken& x = tk[i];
        const moa_gemm_desc& dd = d[x.idx];
        const int ty = dd.dt == MOA_F64_CRT_F64IN ? 1 : 0;
        n32 += ty == 0;
        uint8_t* r = base + P.region[i];
        CrtGPass& q = pass[i];
        q.A = dd.A;
        q.B = dd.B;
        q.C = static_cast<double*>(dd.C);
        q.m = dd.m;
        q.n = dd.n;
        q.p = dd.p;
        q.lda = x.L.lda;
        q.ldb = x.L.ldb;
        q.ldr = x.L.ldr;
        q.a_plane = dd.m * x.L.lda;
        q.b_plane = dd.n * x.L.ldb;
        q.gx = ceil_div(dd.p, 256);
        q.a_pl = reinterpret_cast<__nv_bfloat16*>(r + x.L.a_off);
        q.b_pl = reinterpret_cast<__nv_bfloat16*>(r + x.L.b_off);
        q.eA = reinterpret_cast<int*>(r + x.L.ea_off);
        q.eB = reinterpret_cast<int*>(r + x.L.eb_off);
        q.cmax = base + cmax_pos;
        cmax_pos += (static_cast<size_t>(dd.p) * 8 + 255) / 256 * 256;
        q.R = r + x.L.r_off;
        q.status = (status_of && status_of[x.idx]) ? status_of[x.idx] : status;
        q.M = x.M;
        q.t = x.t;
        const int per16 = ty ? 2 : 4;
        q.va = vec_rows(dd.A, dd.n, per16);
        q.vb = vec_rows(dd.B, dd.p, per16);
        q.vec_c = (dd.p % 2 == 0) && (reinterpret_cast<uintptr_t>(dd.C) % 16 == 0);
        q.f64in = ty;
        q.rblocks = static_cast<int>(std::min<int64_t>(ceil_div(dd.m, 8), 16L * sms));
        q.chunk = colmax_chunk(dd.n, dd.p, sms);
        q.cblocks = static_cast<int>(q.gx * ceil_div(dd.n, q.chunk));
        q.exps_begin = exps_pos[ty];
        exps_pos[ty] += q.rblocks + q.cblocks;
        q.ga = grid_for(q.a_plane / 4, 256);
        q.gb = grid_for(q.b_plane / 4, 256);
        q.res_begin = res_pos[ty];
        res_pos[ty] += q.ga + q.gb;
        q.rec_blocks = grid_for(dd.m * ceil_div(dd.p, 4), 256);
        q.rec_begin = rec_pos;
        rec_pos += q.rec_blocks;
    }
    // residue-GEMM problems, longest K first, each with its TMA descriptors
    std::vector<int> order(G);
    for (int i = 0; i < G; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return d[tk[a].idx].n > d[tk[b].idx].n; });
    long units = 0;
    for (int j = 0; j < G; ++j) {
        const int i = order[j];
        const Taken& x = tk[i];
        const moa_gemm_desc& dd = d[x.idx];
        CrtGProb& g = probs[j];
        g.R = base + P.region[i] + x.L.r_off;
        g.m = dd.m;
        g.p = dd.p;
        g.ldr = x.L.ldr;
        g.bn = crt_block_n(dd.m, dd.p, x.M, sms);
        g.tiles_m = static_cast<int>(ceil_div(dd.m, kBM));
        g.tiles_n = static_cast<int>(ceil_div(dd.p, g.bn));
        g.num_kb = static_cast<int>(ceil_div(dd.n, kBK));
        g.group_m = split_raster_group(dd.n);
        g.M = x.M;
        g.unit_begin = static_cast<int>(units);
        units += static_cast<long>(x.M) * g.tiles_m * g.tiles_n;
        int rc = make_tmap_3d(&maps[2 * j], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, pass[i].a_pl,
                              static_cast<uint64_t>(dd.n), static_cast<uint64_t>(dd.m),
                              static_cast<uint64_t>(x.M), static_cast<uint64_t>(x.L.lda) * 2,
                              static_cast<uint64_t>(pass[i].a_plane) * 2, kBK, kBM);
        if (rc == MOA_OK)
            rc = make_tmap_3d(&maps[2 * j + 1], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, pass[i].b_pl,
                              static_cast<uint64_t>(dd.p), static_cast<uint64_t>(dd.n),
                              static_cast<uint64_t>(x.M), static_cast<uint64_t>(x.L.ldb) * 2,
                              static_cast<uint64_t>(pass[i].b_plane) * 2, 64, kBK);
        if (rc != MOA_OK) {
            staging_release(slot, s);
            return rc;
        }
    }
    if (units > (1L << 30)) {
        staging_release(slot, s);
        return fail(MOA_ERR_ARG, "too many units in one grouped call");
    }
    cudaError_t e = cudaMemcpyAsync(base, host, P.head_bytes, cudaMemcpyHostToDevice, s);
    staging_release(slot, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(grouped crt tables)");
    e = cudaMemsetAsync(base + P.cmax_off, 0, P.cmax_bytes, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(grouped colmax)");
    const CrtGPass* dpass = reinterpret_cast<const CrtGPass*>(base + P.pass_off);
    CrtPow2 pow2{};
    for (int l = 0; l < kCrtMaxModuli; ++l)
        for (int e2 = 0; e2 < kPow2Cols; ++e2)
            pow2.v[l][e2] = static_cast<uint8_t>((static_cast<u128>(1) << e2) % crt_mod(l));
    const int n64 = G - n32;
    if (n32 > 0) {
        crt_g_exps_kernel<float><<<exps_pos[0], 256, 0, s>>>(dpass, n32);
        crt_g_residue_kernel<float><<<res_pos[0], 256, 0, s>>>(dpass, n32, pow2);
    }
    if (n64 > 0) {
        crt_g_exps_kernel<double><<<exps_pos[1], 256, 0, s>>>(dpass + n32, n64);
        crt_g_residue_kernel<double><<<res_pos[1], 256, 0, s>>>(dpass + n32, n64, pow2);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "grouped crt pre-pass launch");
    CrtGemmArgs a{};
    for (int l = 0; l < kCrtMaxModuli; ++l) {
        a.qf[l] = static_cast<float>(crt_mod(l));
        a.qinv[l] = 1.0f / static_cast<float>(crt_mod(l));
    }
    a.wait_limit_ns = wait_limit_ns();
    a.status = status;
    a.probs = reinterpret_cast<const CrtGProb*>(base + P.prob_off);
    a.maps = reinterpret_cast<const CUtensorMap*>(base + P.maps_off);
    a.nprob = G;
    a.num_units = static_cast<int>(units);
    CUtensorMap unused{};
    int rc = launch_crt_gemm<256, true>(a, unused, unused, s, nullptr);
    if (rc != MOA_OK) return rc;
    crt_g_recon_kernel<<<rec_pos, 256, 0, s>>>(
        dpass, G, reinterpret_cast<const CrtConsts*>(base + P.consts_off));
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "grouped crt reconstruction launch");
    log_msg(2, "grouped crt: %d problems, %ld units", G, units);
    return MOA_OK;
}

}  // namespace moa
