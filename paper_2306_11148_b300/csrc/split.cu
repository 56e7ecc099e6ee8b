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
//   max_k |A[i,k]| in [2^(eA_i - 1), 2^eA_i), each column j of B likewise eB_j;
//   x * 2^(7S - e) is rounded once to an integer D and written as S balanced
//   base-128 digits (|d_0| <= 128, d_s in [-64, 64) for s >= 1), each exactly
//   a BF16 value.  Level L = s + t of the triangular product (s + t <= S - 1)
//   is summed over chunks of K short enough that every FP32 partial sum is an
//   integer below 2^24, hence exact; each chunk is flushed into an int32
//   running sum, folded at the level's end into an int64 fixed-point total in
//   TMEM, which the epilogue converts to FP64 once and scales by
//   2^(eA_i + eB_j - 7(S+1) + drop).
//
// Kernel layout (one persistent CTA per SM, 320 threads): warp 0 issues TMA
// loads of (A slice, B slice) K blocks; warp 1 issues tcgen05.mma into one of
// two TMEM chunk accumulators; warps 2..9 (two per TMEM lane quadrant, 64
// columns each) flush chunks and write C.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>

#include "internal.h"
#include "ptx.cuh"
#include "split.h"

namespace moa {

// ====================================================================== pre-passes
namespace {

__device__ __forceinline__ uint32_t pack_bf16x2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return static_cast<uint32_t>(__bfloat16_as_ushort(lo)) |
           (static_cast<uint32_t>(__bfloat16_as_ushort(hi)) << 16);
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
__global__ void split3_kernel(const float* __restrict__ X, int64_t rows, int64_t cols, int64_t ld,
                              __nv_bfloat16* __restrict__ out, int64_t plane, int vec, int* status) {
    const int64_t gpr = ld / 8;                 // 8-element groups per row
    const int64_t total = rows * gpr;
    bool bad = false;
    for (int64_t g = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; g < total;
         g += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t r = g / gpr, c0 = (g - r * gpr) * 8;
        float x[8];
        load8(X, r, cols, c0, vec != 0, x);
        uint32_t w0[4], w1[4], w2[4];
#pragma unroll
        for (int i = 0; i < 8; i += 2) {
            __nv_bfloat16 a[2], b[2], c[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float v = x[i + h];
                a[h] = __float2bfloat16_rn(v);
                const float av = __bfloat162float(a[h]);
                const float r1 = __fsub_rn(v, av);
                b[h] = __float2bfloat16_rn(r1);
                const float r2 = __fsub_rn(r1, __bfloat162float(b[h]));
                c[h] = __float2bfloat16_rn(r2);
                bad |= !isfinite(v) || !isfinite(av);
            }
            w0[i / 2] = pack_bf16x2(a[0], a[1]);
            w1[i / 2] = pack_bf16x2(b[0], b[1]);
            w2[i / 2] = pack_bf16x2(c[0], c[1]);
        }
        const int64_t o = r * ld + c0;
        *reinterpret_cast<uint4*>(out + o) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
        *reinterpret_cast<uint4*>(out + plane + o) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
        *reinterpret_cast<uint4*>(out + 2 * plane + o) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
    }
    if (bad) atomicCAS(status, kDevOk, kDevNonFinite);
}

template <typename T>
struct Bits;
template <>
struct Bits<double> {
    using U = unsigned long long;
    static constexpr U kAbsMask = 0x7FFFFFFFFFFFFFFFull;
    static constexpr U kInf = 0x7FF0000000000000ull;
    __device__ static U abs_bits(double x) {
        return static_cast<U>(__double_as_longlong(x)) & kAbsMask;
    }
    // frexp exponent of the non-negative value with bit pattern M (0 for 0).
    __device__ static int frexp_exp(U M) {
        if (M == 0) return 0;
        const int ex = static_cast<int>(M >> 52);
        if (ex > 0) return ex - 1022;
        return (64 - __clzll(static_cast<long long>(M))) - 1074;
    }
    // round-half-even(x * 2^k) as an integer; requires |x| * 2^k < 2^62.
    __device__ static long long round_scaled(double x, int k) {
        const U b = static_cast<U>(__double_as_longlong(x));
        const bool neg = (b >> 63) != 0;
        const int ex = static_cast<int>((b >> 52) & 0x7FF);
        U mant = b & 0xFFFFFFFFFFFFFull;
        int E;
        if (ex == 0) {
            E = -1074;
        } else {
            mant |= 1ull << 52;
            E = ex - 1075;
        }
        if (mant == 0) return 0;
        const int sh = E + k;
        U D;
        if (sh >= 0) {
            D = mant << sh;
        } else {
            const int kk = -sh;
            if (kk > 54) {
                D = 0;
            } else {
                const U q = mant >> kk;
                const U rem = mant & ((1ull << kk) - 1);
                const U half = 1ull << (kk - 1);
                D = q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull);
            }
        }
        return neg ? -static_cast<long long>(D) : static_cast<long long>(D);
    }
};
template <>
struct Bits<float> {
    using U = unsigned int;
    static constexpr U kAbsMask = 0x7FFFFFFFu;
    static constexpr U kInf = 0x7F800000u;
    __device__ static U abs_bits(float x) { return __float_as_uint(x) & kAbsMask; }
    __device__ static int frexp_exp(U M) {
        if (M == 0) return 0;
        const int ex = static_cast<int>(M >> 23);
        if (ex > 0) return ex - 126;
        return (32 - __clz(static_cast<int>(M))) - 149;
    }
    __device__ static long long round_scaled(float x, int k) {
        const U b = __float_as_uint(x);
        const bool neg = (b >> 31) != 0;
        const int ex = static_cast<int>((b >> 23) & 0xFF);
        unsigned long long mant = b & 0x7FFFFFu;
        int E;
        if (ex == 0) {
            E = -149;
        } else {
            mant |= 1ull << 23;
            E = ex - 150;
        }
        if (mant == 0) return 0;
        const int sh = E + k;
        unsigned long long D;
        if (sh >= 0) {
            D = mant << sh;
        } else {
            const int kk = -sh;
            if (kk > 25) {
                D = 0;
            } else {
                const unsigned long long q = mant >> kk;
                const unsigned long long rem = mant & ((1ull << kk) - 1);
                const unsigned long long half = 1ull << (kk - 1);
                D = q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull);
            }
        }
        return neg ? -static_cast<long long>(D) : static_cast<long long>(D);
    }
};

// One warp per row: exponent of max |A[i,:]|.
template <typename T>
__global__ void row_exp_kernel(const T* __restrict__ X, int64_t rows, int64_t cols,
                               int* __restrict__ e_out, int* status) {
    using B = Bits<T>;
    const int lane = threadIdx.x & 31;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    bool bad = false;
    for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x >> 5) + (threadIdx.x >> 5);
         r < rows; r += warps) {
        typename B::U mx = 0;
        for (int64_t c = lane; c < cols; c += 32) mx = max(mx, B::abs_bits(X[r * cols + c]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const typename B::U other = __shfl_xor_sync(0xffffffffu, mx, o);
            mx = max(mx, other);
        }
        if (lane == 0) {
            bad |= mx >= B::kInf;
            e_out[r] = B::frexp_exp(mx);
        }
    }
    if (bad) atomicCAS(status, kDevOk, kDevNonFinite);
}

// Column maxima of |B| (bit patterns), by atomicMax over row chunks.
template <typename T>
__global__ void col_max_kernel(const T* __restrict__ X, int64_t rows, int64_t cols, int64_t chunk,
                               typename Bits<T>::U* __restrict__ cmax) {
    using B = Bits<T>;
    const int64_t c = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (c >= cols) return;
    const int64_t r0 = blockIdx.y * chunk;
    const int64_t r1 = min(rows, r0 + chunk);
    typename B::U mx = 0;
    for (int64_t r = r0; r < r1; ++r) mx = max(mx, B::abs_bits(X[r * cols + c]));
    atomicMax(&cmax[c], mx);
}

template <typename T>
__global__ void col_exp_kernel(const typename Bits<T>::U* __restrict__ cmax, int64_t cols,
                               int* __restrict__ e_out, int* status) {
    using B = Bits<T>;
    const int64_t c = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (c >= cols) return;
    const typename B::U M = cmax[c];
    if (M >= B::kInf) atomicCAS(status, kDevOk, kDevNonFinite);
    e_out[c] = B::frexp_exp(M);
}

// Integer digits of every element into S BF16 planes (row pitch ld, a
// multiple of 8; zero pad); 8 consecutive elements per thread, one 16-byte
// store per digit plane.  axis 0: exponent per row (e[r]); axis 1: per
// column (e[c]).
template <typename T>
__global__ void digits_kernel(const T* __restrict__ X, int64_t rows, int64_t cols, int64_t ld,
                              const int* __restrict__ e, int axis, int S,
                              __nv_bfloat16* __restrict__ out, int64_t plane) {
    const int64_t gpr = ld / 8;
    const int64_t total = rows * gpr;
    constexpr long long radix = 1ll << kBeta;
    constexpr long long half = radix / 2;
    for (int64_t g = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; g < total;
         g += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t r = g / gpr, c0 = (g - r * gpr) * 8;
        long long D[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int64_t c = c0 + i;
            D[i] = 0;
            if (c < cols) {
                const int ex = axis == 0 ? e[r] : e[c];
                D[i] = Bits<T>::round_scaled(X[r * cols + c], kBeta * S - ex);
            }
        }
        const int64_t o = r * ld + c0;
        for (int s = S - 1; s >= 0; --s) {
            uint32_t w[4];
#pragma unroll
            for (int i = 0; i < 8; i += 2) {
                __nv_bfloat16 d[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    long long low = D[i + h];
                    if (s > 0) {
                        low = D[i + h] & (radix - 1);
                        if (low >= half) low -= radix;
                        D[i + h] = (D[i + h] - low) >> kBeta;
                    }
                    d[h] = __float2bfloat16_rn(static_cast<float>(low));
                }
                w[i / 2] = pack_bf16x2(d[0], d[1]);
            }
            *reinterpret_cast<uint4*>(out + s * plane + o) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

int grid_for(int64_t total, int threads) {
    const int64_t want = ceil_div(total, threads);
    const int64_t cap = 16L * num_sms();
    return static_cast<int>(std::max<int64_t>(1, std::min(want, cap)));
}

}  // namespace

// ====================================================================== slice GEMM
namespace {

constexpr int kBM = 128, kBK = 64;
constexpr int kABytes = kBM * 128;                 // 128 rows x 64 BF16
constexpr int kBChunkBytes = kBK * 128;            // 64 rows x 64 BF16 columns
constexpr int kMaxLevels = 8;

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

template <int BN, int MODE>
struct SplitCfg {
    static constexpr int kStages = BN == 256 ? 4 : (BN == 192 ? 5 : 6);
    static constexpr int kBBytes = (BN / 64) * kBChunkBytes;
    static constexpr int kStageBytes = kABytes + kBBytes;
    static constexpr int kSmem = 1024 + kStages * kStageBytes + 256;
    static constexpr int kColsPerWarp = MODE == kModeF64Tmem ? 128 : 64;
    static constexpr int kEpiWarps = 4 * (BN / kColsPerWarp);
    static constexpr int kThreads = 64 + 32 * kEpiWarps;
    static constexpr int kNBuf = MODE == kModeF64Tmem ? 1 : 2;
    static constexpr int kTmemCols = (MODE == kModeF64Tmem || BN > 128) ? 512 : 256;
    static constexpr uint32_t kIdesc = make_idesc(1u, kBM, BN, 0u, 1u);
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
    int drop;           // fixed-point bits dropped from the int64 total (FP64 mode)
    const int* eA;
    const int* eB;
    int vec_ok;
    uint64_t wait_limit_ns;
    int* status;
};

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

template <int BN, int MODE>
__global__ void __launch_bounds__(SplitCfg<BN, MODE>::kThreads, 1)
    split_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                      const SplitArgs args) {
    using Cfg = SplitCfg<BN, MODE>;
    constexpr bool F64 = MODE != kModeF32;
    constexpr int kNBuf = Cfg::kNBuf;
    constexpr int kStages = Cfg::kStages;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                               ~static_cast<uintptr_t>(1023));
    uint8_t* sA = smem;
    uint8_t* sB = smem + kStages * kABytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + kStages * Cfg::kBBytes);
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
    if (warp == 0 && lane == 0) {
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

    const int num_tiles = args.tiles_m * args.tiles_n;
    const int num_kb = args.num_kb;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer: (tile, level, kb, pair)
            int stage = 0;
            uint32_t phase = 0;
            long issued = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < num_tiles && ok; t += gridDim.x) {
                int tm, tn;
                split_tile_coords(t, args.tiles_m, args.tiles_n, args.group_m, tm, tn);
                for (int L = 0; L < args.levels && ok; ++L) {
                    const int np = level_pairs(args, L);
                    for (int kb = 0; kb < num_kb && ok; ++kb) {
                        for (int q = 0; q < np; ++q) {
                            int s, u;
                            pair_at(args, L, q, s, u);
                            if (!mbar_wait(&empty[stage], phase ^ 1u, ctl, limit, status)) {
                                ok = false;
                                break;
                            }
                            mbar_arrive_expect_tx(&full[stage], Cfg::kStageBytes);
                            tma_load_3d(sA + stage * kABytes, &tmA, &full[stage], kb * kBK,
                                        tm * kBM, s);
#pragma unroll
                            for (int c = 0; c < BN / 64; ++c)
                                tma_load_3d(sB + stage * Cfg::kBBytes + c * kBChunkBytes, &tmB,
                                            &full[stage], tn * BN + c * 64, kb * kBK, u);
                            ++issued;
                            if (++stage == kStages) {
                                stage = 0;
                                phase ^= 1u;
                            }
                        }
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
            for (int t = blockIdx.x; t < num_tiles && ok; t += gridDim.x) {
                for (int L = 0; L < args.levels && ok; ++L) {
                    const int np = level_pairs(args, L);
                    const int kc = args.kc[L];
                    for (int kb0 = 0; kb0 < num_kb && ok; kb0 += kc, ++cnt) {
                        const int buf = static_cast<int>(cnt % kNBuf);
                        const uint32_t bph = static_cast<uint32_t>((cnt / kNBuf) & 1);
                        if (!mbar_wait(&tempty[buf], bph ^ 1u, ctl, limit, status)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t d = tmem_base + static_cast<uint32_t>(buf * BN);
                        const int kb1 = min(num_kb, kb0 + kc);
                        bool first = true;
                        for (int kb = kb0; kb < kb1 && ok; ++kb) {
                            for (int q = 0; q < np; ++q) {
                                if (!mbar_wait(&full[stage], phase, ctl, limit, status)) {
                                    ok = false;
                                    break;
                                }
                                tc_fence_after();
                                const uint64_t adesc =
                                    smem_desc_sw128(smem_u32(sA + stage * kABytes), 16, 1024);
                                const uint64_t bdesc = smem_desc_sw128(
                                    smem_u32(sB + stage * Cfg::kBBytes), kBChunkBytes, 1024);
#pragma unroll
                                for (int k = 0; k < kBK / 16; ++k) {
                                    mma_f16(d, adesc + static_cast<uint64_t>((k * 32) >> 4),
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
        long cnt = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < num_tiles && ok; t += gridDim.x) {
            int tm, tn;
            split_tile_coords(t, args.tiles_m, args.tiles_n, args.group_m, tm, tn);
            const int64_t row = static_cast<int64_t>(tm) * kBM + q * 32 + lane;
            const int64_t col_base = static_cast<int64_t>(tn) * BN + h * kCols;
            const bool row_ok = row < args.m;
            // FP64 modes keep the tile's int64 fixed-point total T in C itself
            // (same 8 bytes per element as the final FP64 value).
            long long* trow = reinterpret_cast<long long*>(args.C) + row * args.p;
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
                const int kc = args.kc[L];
                int since_fold = 0;
                for (int kb0 = 0; kb0 < num_kb; kb0 += kc, ++cnt) {
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
                    } else {
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
                    const bool level_end = kb0 + kc >= num_kb;
                    if (F64 && (level_end || since_fold == 64)) {
                        // fold the level's exact sum into the int64 total:
                        // T += round(R * 2^(beta(S-1-L) - drop)); the last fold
                        // of the tile converts once to FP64 and scales by
                        // 2^(eA_i + eB_j - beta(S+1) + drop).
                        const int sh = kBeta * (args.S - 1 - L) - args.drop;
                        const bool last = level_end && L == args.levels - 1;
#pragma unroll
                        for (int b = 0; b < kCols / 16; ++b) {
                            uint32_t rv[16];
                            if constexpr (MODE == kModeF64Tmem) {
                                tmem_ld16(r_base + 16u * b, rv);
                                tmem_ld_wait();
                            } else {
#pragma unroll
                                for (int i = 0; i < 16; ++i) rv[i] = 0u;
                            }
                            if (row_ok) {
                                // 16 independent loads of T, so their latency overlaps
                                long long told[16];
#pragma unroll
                                for (int i = 0; i < 16; ++i) {
                                    const int64_t col = col_base + b * 16 + i;
                                    told[i] = (t_init && col < args.p) ? trow[col] : 0ll;
                                }
#pragma unroll
                                for (int i = 0; i < 16; ++i) {
                                    const int64_t col = col_base + b * 16 + i;
                                    if (col >= args.p) continue;
                                    long long v;
                                    if constexpr (MODE == kModeF64Tmem)
                                        v = static_cast<int>(rv[i]);
                                    else
                                        v = static_cast<int>(acc[(b * 16 + i) % kRegs]);
                                    if (sh >= 0)
                                        v = v * (1ll << sh);
                                    else
                                        v = (v + (1ll << (-sh - 1))) >> (-sh);
                                    const long long tot = told[i] + v;
                                    if (last) {
                                        const int ex =
                                            er + args.eB[col] - kBeta * (args.S + 1) + args.drop;
                                        reinterpret_cast<double*>(trow)[col] =
                                            ldexp(__ll2double_rn(tot), ex);
                                    } else {
                                        trow[col] = tot;
                                    }
                                }
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
            // ---------------- FP32 mode: store the tile
            if (!F64 && row_ok) {
                float* crow = static_cast<float*>(args.C) + row * args.p;
                if (args.vec_ok && col_base + 64 <= args.p) {
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
                        if (col_base + i < args.p) crow[col_base + i] = __uint_as_float(acc[i % kRegs]);
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
static int f32_split_chunk_kb() {
    static int kb = 0;
    if (kb == 0) {
        const char* env = std::getenv("MOA_F32_SPLIT_CHUNK_K");
        const long k = env ? std::strtol(env, nullptr, 10) : 256;
        kb = static_cast<int>(std::max<long>(1, (k + kBK - 1) / kBK));
    }
    return kb;
}

int split_slices(moa_dtype dt, int slices) {
    if (dt == MOA_F32_SPLIT) return (slices == 0 || slices == 3) ? 3 : -1;
    if (slices == 0) return kDefaultSlices;
    if (slices < kMinSlices || slices > kMaxSlices) return -1;
    return slices;
}

SplitLayout split_layout(int64_t m, int64_t n, int64_t p, moa_dtype dt, int S) {
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    SplitLayout L{};
    L.S = S;
    L.lda = round_up(n, 8);
    L.ldb = round_up(p, 8);
    size_t off = 0;
    L.a_off = off;
    off += al(static_cast<size_t>(S) * m * L.lda * 2);
    L.b_off = off;
    off += al(static_cast<size_t>(S) * n * L.ldb * 2);
    if (dt != MOA_F32_SPLIT) {
        L.ea_off = off;
        off += al(static_cast<size_t>(m) * 4);
        L.eb_off = off;
        off += al(static_cast<size_t>(p) * 4);
        L.cmax_off = off;
        off += al(static_cast<size_t>(p) * 8);
    }
    L.total = off;
    return L;
}

size_t split_workspace_bytes(int64_t m, int64_t n, int64_t p, moa_dtype dt, int slices) {
    const int S = split_slices(dt, slices);
    if (S < 0) return 0;
    return split_layout(m, n, p, dt, S).total;
}

template <int BN, int MODE>
static int launch_split_cfg(const SplitArgs& a, const CUtensorMap& tmA, const CUtensorMap& tmB,
                            cudaStream_t s, moa_stats* st) {
    using Cfg = SplitCfg<BN, MODE>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(split_gemm_kernel<BN, MODE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::kSmem);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(split_gemm)");
        attr_set = true;
    }
    const long tiles = static_cast<long>(a.tiles_m) * a.tiles_n;
    const int grid = static_cast<int>(std::min<long>(tiles, num_sms()));
    prof_begin(s);
    split_gemm_kernel<BN, MODE><<<grid, Cfg::kThreads, Cfg::kSmem, s>>>(tmA, tmB, a);
    cudaError_t e = cudaGetLastError();
    prof_end(s);
    if (e != cudaSuccess) return cuda_fail(e, "split_gemm_kernel launch");
    if (st) {
        st->block_m = kBM;
        st->block_n = BN;
        st->block_k = kBK;
        st->grid = grid;
        st->tiles = tiles;
    }
    return MOA_OK;
}

// Tile width of the slice GEMM: 256 when that still gives every SM a tile
// (fewest B re-reads per flop), else 128.  moa_set_block_n(128 | 192 | 256)
// forces it (192: FP64 accuracy only).
static int split_block_n(int64_t m, int64_t p, bool f64) {
    const int ov = tile_override();
    if (ov == 128 || ov == 256 || (ov == 192 && f64)) return ov;
    const long tiles = ceil_div(m, kBM) * ceil_div(p, 256);
    return tiles >= num_sms() ? 256 : 128;
}

int split_gemm(int64_t m, int64_t n, int64_t p, moa_dtype dt, const void* A, const void* B,
               void* C, int slices, void* ws, size_t ws_bytes, cudaStream_t s, moa_stats* st) {
    const int S = split_slices(dt, slices);
    if (S < 0) return fail(MOA_ERR_DTYPE, "slice count not supported for this mode");
    const SplitLayout L = split_layout(m, n, p, dt, S);
    if (ws_bytes < L.total) return fail(MOA_ERR_WORKSPACE, "workspace too small for split mode");
    int* status = launch_status_ptr();
    if (!status) return MOA_ERR_CUDA;
    uint8_t* base = static_cast<uint8_t*>(ws);
    __nv_bfloat16* a_sl = reinterpret_cast<__nv_bfloat16*>(base + L.a_off);
    __nv_bfloat16* b_sl = reinterpret_cast<__nv_bfloat16*>(base + L.b_off);
    const int64_t a_plane = m * L.lda, b_plane = n * L.ldb;
    int kernels = 0;

    SplitArgs a{};
    a.C = C;
    a.m = m;
    a.n = n;
    a.p = p;
    const int bn = split_block_n(m, p, dt != MOA_F32_SPLIT);
    a.tiles_m = static_cast<int>(ceil_div(m, kBM));
    a.tiles_n = static_cast<int>(ceil_div(p, bn));
    a.num_kb = static_cast<int>(ceil_div(n, kBK));
    a.group_m = raster_group();
    a.S = S;
    a.wait_limit_ns = wait_limit_ns();
    a.status = status;
    a.vec_ok = (p % 4 == 0) && (reinterpret_cast<uintptr_t>(C) % 16 == 0);

    if (dt == MOA_F32_SPLIT) {
        const int va = (n % 4 == 0) && (reinterpret_cast<uintptr_t>(A) % 16 == 0);
        const int vb = (p % 4 == 0) && (reinterpret_cast<uintptr_t>(B) % 16 == 0);
        split3_kernel<<<grid_for(a_plane / 8, 256), 256, 0, s>>>(
            static_cast<const float*>(A), m, n, L.lda, a_sl, a_plane, va, status);
        split3_kernel<<<grid_for(b_plane / 8, 256), 256, 0, s>>>(
            static_cast<const float*>(B), n, p, L.ldb, b_sl, b_plane, vb, status);
        kernels += 2;
        a.f64 = 0;
        a.levels = 1;
        // Flush the FP32 TMEM accumulator into the epilogue's FP32 running sum
        // every kc K blocks: shorter chunks bound the accumulation error of
        // the tensor core's FP32 adds (MOA_F32_SPLIT_CHUNK_K, default 256).
        a.kc[0] = f32_split_chunk_kb();
        a.drop = 0;
    } else {
        int* eA = reinterpret_cast<int*>(base + L.ea_off);
        int* eB = reinterpret_cast<int*>(base + L.eb_off);
        void* cmax = base + L.cmax_off;
        const bool in64 = dt == MOA_F64_SPLIT_F64IN;
        cudaError_t e = cudaMemsetAsync(cmax, 0, static_cast<size_t>(p) * 8, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(colmax)");
        const int rows_per_block = 8;   // 8 warps of 32 threads
        const int64_t rblocks = std::min<int64_t>(ceil_div(m, rows_per_block), 16L * num_sms());
        const int64_t chunk = 256;
        dim3 cgrid(static_cast<unsigned>(ceil_div(p, 256)), static_cast<unsigned>(ceil_div(n, chunk)));
        if (cgrid.y > 65535) return fail(MOA_ERR_ARG, "n too large for the column-max grid");
        if (in64) {
            const double* Ad = static_cast<const double*>(A);
            const double* Bd = static_cast<const double*>(B);
            row_exp_kernel<double><<<static_cast<int>(rblocks), 256, 0, s>>>(Ad, m, n, eA, status);
            col_max_kernel<double><<<cgrid, 256, 0, s>>>(Bd, n, p, chunk,
                                                         static_cast<unsigned long long*>(cmax));
            col_exp_kernel<double><<<static_cast<int>(ceil_div(p, 256)), 256, 0, s>>>(
                static_cast<const unsigned long long*>(cmax), p, eB, status);
            digits_kernel<double><<<grid_for(a_plane / 8, 256), 256, 0, s>>>(Ad, m, n, L.lda, eA, 0, S,
                                                                          a_sl, a_plane);
            digits_kernel<double><<<grid_for(b_plane / 8, 256), 256, 0, s>>>(Bd, n, p, L.ldb, eB, 1, S,
                                                                          b_sl, b_plane);
        } else {
            const float* Af = static_cast<const float*>(A);
            const float* Bf = static_cast<const float*>(B);
            row_exp_kernel<float><<<static_cast<int>(rblocks), 256, 0, s>>>(Af, m, n, eA, status);
            col_max_kernel<float><<<cgrid, 256, 0, s>>>(Bf, n, p, chunk,
                                                        static_cast<unsigned int*>(cmax));
            col_exp_kernel<float><<<static_cast<int>(ceil_div(p, 256)), 256, 0, s>>>(
                static_cast<const unsigned int*>(cmax), p, eB, status);
            digits_kernel<float><<<grid_for(a_plane / 8, 256), 256, 0, s>>>(Af, m, n, L.lda, eA, 0, S,
                                                                        a_sl, a_plane);
            digits_kernel<float><<<grid_for(b_plane / 8, 256), 256, 0, s>>>(Bf, n, p, L.ldb, eB, 1, S,
                                                                        b_sl, b_plane);
        }
        kernels += 6;
        a.f64 = 1;
        a.levels = S;
        a.eA = eA;
        a.eB = eB;
        // Chunk lengths: every FP32 partial sum of a level must stay an
        // integer of magnitude <= 2^24.  With |d_0| <= 2^beta and
        // |d_s| <= 2^(beta-1), per k level 0 adds at most 2^(2 beta) and
        // level L >= 1 at most 2 * 2^(2 beta - 1) + (L - 1) * 2^(2 beta - 2)
        // = (L + 3) * 2^(2 beta - 2).
        for (int lev = 0; lev < S; ++lev) {
            const long long per_k = lev == 0 ? (1ll << (2 * kBeta))
                                             : static_cast<long long>(lev + 3) << (2 * kBeta - 2);
            const long long kmax = (1ll << 24) / per_k;
            a.kc[lev] = static_cast<int>(std::max(1ll, kmax / kBK));
        }
        // int64 total: |T| <= n * 2^(beta(S+1)) * 1.02 in units of the finest
        // level before dropping `drop` bits; keep it below 2^62.
        int nbits = 0;
        while ((1ll << nbits) < n) ++nbits;
        a.drop = std::max(0, nbits + kBeta * (S + 1) + 1 - 62);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "split pre-pass launch");

    CUtensorMap tmA, tmB;
    int rc = make_tmap_3d(&tmA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, a_sl, static_cast<uint64_t>(n),
                          static_cast<uint64_t>(m), static_cast<uint64_t>(S),
                          static_cast<uint64_t>(L.lda) * 2, static_cast<uint64_t>(a_plane) * 2, 64,
                          kBM);
    if (rc != MOA_OK) return rc;
    rc = make_tmap_3d(&tmB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, b_sl, static_cast<uint64_t>(p),
                      static_cast<uint64_t>(n), static_cast<uint64_t>(S),
                      static_cast<uint64_t>(L.ldb) * 2, static_cast<uint64_t>(b_plane) * 2, 64, kBK);
    if (rc != MOA_OK) return rc;
    if (a.f64)
        rc = bn == 256   ? launch_split_cfg<256, kModeF64Tmem>(a, tmA, tmB, s, st)
             : bn == 192 ? launch_split_cfg<192, kModeF64Reg>(a, tmA, tmB, s, st)
                         : launch_split_cfg<128, kModeF64Reg>(a, tmA, tmB, s, st);
    else
        rc = bn == 256 ? launch_split_cfg<256, kModeF32>(a, tmA, tmB, s, st)
                       : launch_split_cfg<128, kModeF32>(a, tmA, tmB, s, st);
    if (st) {
        st->slices = S;
        st->products = dt == MOA_F32_SPLIT ? 6 : S * (S + 1) / 2;
        st->kernels = kernels + 1;
    }
    return rc;
}

}  // namespace moa
