// internal.h -- declarations shared by the translation units of libmoa.so
// (not part of the public ABI; see include/moa.h for that).
#pragma once
#include <atomic>
#include <cstddef>
#include <cstdint>
#include <string>

#include <cuda.h>
#include <cuda_runtime.h>

#include "moa.h"

namespace moa {

// ------------------------------------------------------------------ modes
inline bool valid_dtype(int dt) { return dt >= MOA_F64 && dt <= MOA_F64_CRT_F64IN; }
// Bytes per element of A and B, and of C, for each mode.
inline int dtype_in_bytes(moa_dtype dt) {
    return (dt == MOA_F64 || dt == MOA_F64_SPLIT_F64IN || dt == MOA_F64_SPLIT_F64IN_E4M3 ||
            dt == MOA_F64_CRT_F64IN)
               ? 8
               : (dt == MOA_BF16 ? 2 : 4);
}
inline int dtype_out_bytes(moa_dtype dt) {
    return (dt == MOA_F64 || dt == MOA_F64_SPLIT_F32IN || dt == MOA_F64_SPLIT_F64IN ||
            dt == MOA_F64_SPLIT_F32IN_E4M3 || dt == MOA_F64_SPLIT_F64IN_E4M3 ||
            dt == MOA_F64_CRT_F32IN || dt == MOA_F64_CRT_F64IN)
               ? 8
               : 4;
}

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);
int fail(int status, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

// ------------------------------------------------------------------ logging / tracing
// MOA_LOG=0..3 (default 0): 1 = errors (every fail / cuda_fail message),
// 2 = the plan of every launch (kernel, tile, grid), 3 = more.  Lines go to
// stderr prefixed "[moa] ".
int log_level();
void log_msg(int level, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
// MOA_DEBUG_CANARY=1: every call with at least kCanaryBytes of workspace past
// what it needs fills those bytes with a pattern before its kernels and checks
// them after (a one-block kernel that records kDevCanary in the status word,
// reported by moa_sync_status), catching writes past the used workspace.
constexpr size_t kCanaryBytes = 256;
bool canary_enabled();
int canary_arm(void* guard, cudaStream_t s);
int canary_check(const void* guard, cudaStream_t s);
// NVTX ranges (no cost unless a profiler tool is attached).
void trace_push(const char* name);
void trace_pop();
struct TraceRange {
    explicit TraceRange(const char* name) { trace_push(name); }
    ~TraceRange() { trace_pop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

// Optional per-thread profiling events (moa_profile_events): recorded on the
// call's stream immediately before and after the main GEMM kernel.
void prof_begin(cudaStream_t s);
void prof_end(cudaStream_t s);

// Per-device status word (device address), created on first use.
int* device_status_ptr();
// Status word the kernels launched by this thread record into: the
// per-device word, unless a caller (the serving loop) set a per-request
// slot with set_status_override (nullptr restores the default).
int* launch_status_ptr();
void set_status_override(int* p);
uint64_t wait_limit_ns();
int num_sms();
// Raises `func`'s dynamic shared-memory limit to `bytes` on the current
// device, once per device (the attribute belongs to the device context, so
// a process that launches on several GPUs needs it on each).  `done` is the
// caller's per-kernel record (bit d: device d set); devices numbered 64 and
// above are set on every call.
int smem_attr_once(const void* func, int bytes, std::atomic<uint64_t>& done, const char* what);

// ------------------------------------------------------------------ TMA maps
// 2-D tiled map over a row-major matrix of `outer` rows x `inner` columns with
// a row pitch of `pitch_bytes`; box = box_outer rows x box_inner columns,
// 128-byte swizzle, zero fill out of bounds.
int make_tmap_2d(CUtensorMap* map, CUtensorMapDataType dt, const void* base, uint64_t inner,
                 uint64_t outer, uint64_t pitch_bytes, uint32_t box_inner, uint32_t box_outer);
// 3-D variant: `depth` matrices of outer x inner, matrix pitch `plane_bytes`.
int make_tmap_3d(CUtensorMap* map, CUtensorMapDataType dt, const void* base, uint64_t inner,
                 uint64_t outer, uint64_t depth, uint64_t pitch_bytes, uint64_t plane_bytes,
                 uint32_t box_inner, uint32_t box_outer, int swizzle_bytes = 128);

// ------------------------------------------------------------------ kernels
// Dense tcgen05 GEMM, A (m x n, row pitch lda elements), C (m x p, FP32,
// pitch p).  in_bf16: BF16 operands, B given as n x p (pitch ldb).  Else FP32
// operands on the TF32 kind, B given TRANSPOSED as p x n (pitch ldb).
struct TileChoice {
    int block_n;     // 64, 128 or 256
};
int dense_tc_launch(bool in_bf16, int64_t m, int64_t n, int64_t p, const void* A, int64_t lda,
                    const void* B, int64_t ldb, float* C, cudaStream_t s, moa_stats* st);

// Tile-width choice of the dense kernels (tuner.cu): per-thread override
// (0 = none) and the measured width for a shape bucket (0 = none).
int tile_override();
// Tile-height override of the modular-slice GEMM (0 = none, 128 = one CTA a
// tile, 256 = a CTA pair a tile).
int tile_m_override();
// Tile rows per raster group of the persistent kernels (the L2-level lift):
// MOA_RASTER_GROUP, default 16.
int raster_group();
// The same for the slice GEMM, whose tiles each sweep the K range once per
// slice product: MOA_RASTER_GROUP, default 16, or 8 once n > 12288 (measured
// on the B300 at n = 16384: 4-7 % faster than 16; 16 best at n = 8192).
int split_raster_group(int64_t n);
int tuned_block_n(moa_dtype dt, int64_t m, int64_t n, int64_t p);

// SIMT kernels (no tensor cores).
int simt_f64_launch(int64_t m, int64_t n, int64_t p, const double* A, const double* B, double* C,
                    cudaStream_t s);
int simt_f32_launch(int64_t m, int64_t n, int64_t p, const float* A, const float* B, float* C,
                    cudaStream_t s);

// Bt (cols x ld, row-major) := transpose of X (rows x cols), zero-filling
// Bt[:, rows:ld].  FP32.
int transpose_pad_launch(const float* X, int64_t rows, int64_t cols, float* Xt, int64_t ld,
                         cudaStream_t s);

// Copy a rows x cols row-major matrix into a buffer with row pitch ld >= cols
// (elements), zero-filling the padding columns.
int pad_copy_launch(const void* src, void* dst, int64_t rows, int64_t cols, int64_t ld,
                    int esize, cudaStream_t s);

// Pinned host staging for per-call device tables (a small ring per host
// thread): get() returns a buffer of at least n bytes whose previous copy has
// finished; release() records, on the stream of the copy that reads it, when
// it may be reused.
void* staging_get(size_t n, int* slot);
void staging_release(int slot, cudaStream_t s);

inline int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }
inline int64_t ceil_div(int64_t x, int64_t a) { return (x + a - 1) / a; }

}  // namespace moa
