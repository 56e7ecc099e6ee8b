// split.h -- the split-precision modes (MOA_F32_SPLIT, MOA_F64_SPLIT_*),
// internal to libmoa.so.
#pragma once
#include "internal.h"

namespace moa {

inline bool is_e4m3_split(moa_dtype dt) {
    return dt == MOA_F64_SPLIT_F32IN_E4M3 || dt == MOA_F64_SPLIT_F64IN_E4M3;
}
inline bool is_split(moa_dtype dt) {
    return dt == MOA_F32_SPLIT || dt == MOA_F64_SPLIT_F32IN || dt == MOA_F64_SPLIT_F64IN ||
           is_e4m3_split(dt);
}

// Digit radix 2^kBeta of the FP64-accuracy mode and its slice-count limits.
// Base 128 (not 256): each digit product is 4x smaller, so the exact FP32
// accumulation chunks are 4x longer and their flushes hide behind the MMAs;
// 7 digits (28 slice products) keep 48 bits per operand with one headroom
// bit: the group exponent is one above the maximum's, so the top digit is at
// most 64 in magnitude like the others, every per-k product of a level is
// bounded by (L + 1) 2^12, and the exact chunks are 1.25-4x longer than
// without it (60 instead of 90 chunk flushes per 128 x 256 tile at n = 8192;
// each flush converts 32768 FP32 sums to integers).
constexpr int kBeta = 7;
constexpr int kHeadroomBF16 = 1;
constexpr int kMinSlices = 3;
constexpr int kMaxSlices = 8;
constexpr int kDefaultSlices = 7;

// The same method with FP8 E4M3 digit planes (kind::f8f6f4, twice the BF16
// MMA rate): radix 2^5 and one headroom bit, so every digit, the top one
// included, lies in [-16, 16] -- integers E4M3 holds exactly (3 stored
// mantissa bits).  10 digits span 5 * 10 - 1 = 49 bits per operand, as 7
// BF16 digits do, and keep the relative error of the slice product near
// 1e-13 (the dropped part of the triangle is larger than with radix 2^7);
// the triangle has 55 products instead of 28, each at twice the rate, and
// every per-k digit product is at most 2^8, so the exact FP32 chunks are 16x
// longer than with radix 2^7.
constexpr int kBetaE4M3 = 5;
constexpr int kHeadroomE4M3 = 1;
constexpr int kMinSlicesE4M3 = 4;
constexpr int kMaxSlicesE4M3 = 12;
constexpr int kDefaultSlicesE4M3 = 10;

// Resolves the `slices` argument (0 = default); -1 if not allowed for dt.
int split_slices(moa_dtype dt, int slices);

size_t split_workspace_bytes(int64_t m, int64_t n, int64_t p, moa_dtype dt, int slices);

int split_gemm(int64_t m, int64_t n, int64_t p, moa_dtype dt, const void* A, const void* B,
               void* C, int slices, void* ws, size_t ws_bytes, cudaStream_t s, moa_stats* st);

// Workspace layout of a split call (byte offsets from the workspace base).
struct SplitLayout {
    int S;                 // slices per operand
    int esize;             // bytes per slice element: 2 (BF16) or 1 (E4M3)
    bool b_trans;          // E4M3: B's planes hold B^T (p x ldb, K-major)
    int64_t lda, ldb;      // padded row pitches of the slice planes (elements)
    size_t a_off, b_off;   // slice planes: S x m x lda and S x n x ldb (S x p x ldb
                           // when b_trans)
    size_t ea_off, eb_off; // FP64-accuracy: per-row / per-column exponents (int32)
    size_t cmax_off;       // FP64-accuracy: per-column max |B| bit patterns (uint64)
    size_t cnt_off;        // FP64-accuracy, split K: finished-unit counters (int32,
    size_t cnt_bytes;      // one per tile and epilogue warp), then, at fine_off, the
    size_t fine_off;       // m x p int64 sums of the levels finer than the total's
    size_t fine_bytes;     // grid; both 0 when the shape cannot take split K
    // FP32-accuracy split K: at most f32_ks K slices; their FP32 partial tiles
    // (f32_ks x m x p) at part_off, summed in slice order by the last unit
    int f32_ks;
    size_t part_off, part_bytes;
    size_t total;
};
SplitLayout split_layout(int64_t m, int64_t n, int64_t p, moa_dtype dt, int S);

// Grouped calls (moa_gemm_grouped): FP32-accuracy split problems that the
// lone call would run without split K share one slice pre-pass launch and
// one persistent GEMM launch (per-problem TMA descriptors and tile widths);
// each result equals its lone call's bit for bit.  status_of (may be NULL):
// a device status word per descriptor for non-finite inputs.
bool split_grouped_ok(const moa_gemm_desc& d);
size_t split_grouped_workspace(int count, const moa_gemm_desc* d);
int split_grouped_launch(int count, const moa_gemm_desc* d, void* ws, size_t ws_bytes,
                         cudaStream_t s, int* const* status_of = nullptr);

}  // namespace moa
