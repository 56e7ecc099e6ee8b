/*
 * moa.h -- C ABI of the B300-native MoA ONF GEMM library (libmoa.so).
 *
 * The operation (Mullin, "From array algebra to energy efficiency on GPUs",
 * Sec. 2, Eq. (eq:dnf) and its address form):
 *
 *     C[(i*p) + j] := sum_{k=0}^{n-1} A[(i*n) + k] * B[(k*p) + j]
 *     0 <= i < m,  0 <= j < p,  0 <= k < n          (Eqs. (eq:shapes), (eq:indices))
 *
 * Layout: A is m x n, B is n x p and C is m x p, each a dense row-major array
 * starting at the given pointer (the gamma_row layout of the Appendix); there
 * are no leading-dimension arguments.  C is assigned, not accumulated into:
 * callers need not clear it.
 *
 * Memory: A, B, C, workspaces and the serving arena are DEVICE pointers owned
 * by the caller (allocate them with cudaMalloc or PyTorch).  The library
 * allocates device memory in one place only, moa_gemm()'s internal workspace
 * (documented below); it also holds pinned host staging buffers for grouped
 * calls and serving status slots.  Streams are passed as
 * `void*` holding a cudaStream_t (NULL = the legacy default stream).
 *
 * Errors: every entry point returns a moa_status.  Argument errors are
 * detected on the host before anything is launched and leave C untouched;
 * moa_last_error() then gives a message (thread-local).  Launches are
 * asynchronous on the given stream; a device-side failure (a pipeline wait
 * that ran past its time limit) is recorded in a per-device status word and
 * reported by moa_sync_status().
 *
 * Precision modes (moa_dtype): see the enum.  Tolerances the test suite
 * holds each mode to, as relative Frobenius error against the FP64 oracle:
 * MOA_F64 1e-12, MOA_F64_SPLIT_* (both digit formats) and MOA_F64_CRT_* 1e-12 (the
 * latter also bit-exact against the oracle's exact integer product of the
 * scaled operands), MOA_F32_SPLIT 1e-5, MOA_F32_TF32
 * 5e-3, MOA_BF16 1e-2 (and bit-exact on integer-valued inputs in {-8..8}
 * for every mode).
 */
#ifndef MOA_H_
#define MOA_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MOA_OK = 0,
    MOA_ERR_ARG = -1,         /* negative size, NULL pointer with nonzero size, bad count */
    MOA_ERR_DTYPE = -2,       /* unknown moa_dtype or unsupported slice count */
    MOA_ERR_ALIGN = -3,       /* pointer not aligned to its element size */
    MOA_ERR_WORKSPACE = -4,   /* workspace NULL or smaller than the *_workspace_size query */
    MOA_ERR_NONFINITE = -5,   /* split modes: an input is NaN or +-Inf (seen by the pre-pass) */
    MOA_ERR_CUDA = -6,        /* a CUDA runtime/driver call failed (see moa_last_error) */
    MOA_ERR_TIMEOUT = -7,     /* a device pipeline wait ran past its limit; results invalid */
    MOA_ERR_BUDGET = -8,      /* serving: the request alone exceeds the arena */
    MOA_ERR_REJECTED = -9,    /* serving: rejected by the admission policy */
    MOA_ERR_BUSY = -10,       /* serving: queue full */
    MOA_ERR_UNSUPPORTED = -11 /* device is not sm_103 / sm_100 class */
} moa_status;

typedef enum {
    MOA_F64 = 0,              /* A,B,C FP64.  Native FP64 arithmetic (DFMA).                  */
    MOA_F32_TF32 = 1,         /* A,B,C FP32.  tcgen05 kind::tf32, FP32 accumulation.         */
    MOA_F32_SIMT = 2,         /* A,B,C FP32.  Plain FP32 FFMA (comparison path).             */
    MOA_BF16 = 3,             /* A,B BF16, C FP32.  tcgen05 kind::f16, FP32 accumulation.    */
    MOA_F32_SPLIT = 4,        /* A,B,C FP32.  3 BF16 slices each, 6 slice products, FP32 acc.*/
    MOA_F64_SPLIT_F32IN = 5,  /* A,B FP32, C FP64.  Integer-digit BF16 slices, exact         */
                              /*   chunked accumulation, FP64 recombination.                 */
    MOA_F64_SPLIT_F64IN = 6,  /* A,B,C FP64.  As above with FP64 inputs.                     */
    MOA_F64_SPLIT_F32IN_E4M3 = 7, /* A,B FP32, C FP64.  As MOA_F64_SPLIT_F32IN with FP8 E4M3 */
                              /*   digit slices (radix 2^5, one headroom bit: every digit in */
                              /*   [-16, 16], exact in E4M3) on tcgen05 kind::f8f6f4.        */
                              /*   slices: 4..12, default 10 (a 49-bit span per operand);   */
                              /*   55 slice products at twice the BF16 rate.                 */
    MOA_F64_SPLIT_F64IN_E4M3 = 8, /* A,B,C FP64.  As above with FP64 inputs.                 */
    MOA_F64_CRT_F32IN = 9,    /* A,B FP32, C FP64.  Modular slices: rows of A and columns of  */
                              /*   B scaled to t-bit integers, their residues modulo M        */
                              /*   pairwise-coprime moduli <= 256 as BF16 planes, one exact    */
                              /*   tensor-core GEMM per modulus, the exact integer product    */
                              /*   recovered by the Chinese remainder theorem and rounded     */
                              /*   once to FP64.  slices = M: 8..16, default 14 (15 once      */
                              /*   n > 36639), t the largest with n 2^(2t+1) < prod(moduli).  */
    MOA_F64_CRT_F64IN = 10    /* A,B,C FP64.  As above with FP64 inputs.                     */
} moa_dtype;

/* Optional per-call report (may be NULL). */
typedef struct {
    int32_t block_m, block_n, block_k;   /* tile chosen by the planner */
    int32_t slices;                      /* slices per operand (split modes), else 1 */
    int32_t products;                    /* slice products issued per K block, else 1 */
    int32_t grid;                        /* CTAs launched for the main kernel */
    int64_t tiles;                       /* output tiles */
    int32_t kernels;                     /* kernel launches made by this call (memsets not counted) */
    int32_t padded;                      /* 1 if operands were copied to padded pitches */
} moa_stats;

/* ---------------------------------------------------------------------- */
/* Single GEMM                                                             */
/* ---------------------------------------------------------------------- */

/* C := A . B on the legacy default stream, using a library-owned workspace
 * that grows on demand (cudaMalloc) and is freed by moa_shutdown().  This is
 * the one entry point that allocates device memory.  Split modes use their
 * default slice count.  Asynchronous: synchronise (or moa_sync_status) before
 * reading C on the host.
 * m == 0 or p == 0: MOA_OK, nothing launched.  n == 0: C := 0. */
int moa_gemm(int64_t m, int64_t n, int64_t p, moa_dtype dt,
             const void* A, const void* B, void* C);

/* Bytes of workspace moa_gemm_ex needs for this problem (0 if none).
 * slices: split modes only (0 = default); ignored otherwise.  Allowed slice
 * counts: MOA_F32_SPLIT 3; MOA_F64_SPLIT_F32IN / _F64IN 3..8 (default 7);
 * the _E4M3 forms 4..12 (default 10); MOA_F64_CRT_* 8..16 moduli (default 14,
 * 15 once n > 36639).  Returns 0 for a count not allowed. */
size_t moa_gemm_workspace_size(int64_t m, int64_t n, int64_t p, moa_dtype dt, int slices);

/* C := A . B on `stream` with a caller-provided device workspace of at least
 * moa_gemm_workspace_size(...) bytes (ws may be NULL when that size is 0).
 * Allocates nothing.  stats may be NULL.
 * CUDA graphs: once a call of the same mode has run on the device (it sets up
 * kernel attributes and the device status word), a call records only kernel
 * launches and memsets on `stream`, so it can be captured into a CUDA graph
 * and replayed; each replay reads the current contents of A, B and ws. */
int moa_gemm_ex(int64_t m, int64_t n, int64_t p, moa_dtype dt,
                const void* A, const void* B, void* C, int slices,
                void* ws, size_t ws_bytes, void* stream, moa_stats* stats);

/* C := A . B with A, B and C in HOST memory (row-major, contiguous), the
 * call a user without device buffers makes.  On `stream`, in order: A and B
 * are copied to device buffers inside `ws`, the GEMM runs there exactly as
 * moa_gemm_ex would run it (same kernels, same bits), and C is copied back to
 * hC.  ws: a device buffer of at least moa_gemm_host_workspace_size(...)
 * bytes, 256-byte aligned, owned by the caller (the call allocates nothing);
 * it must not be in use by another call until this one's stream work is
 * done.  Asynchronous like moa_gemm_ex: hC holds the result once `stream` has
 * been synchronised (moa_sync_status(stream) also reports the device
 * status).  The copies overlap other streams' work only from page-locked
 * host memory (cudaHostAlloc / cudaHostRegister); from pageable memory they
 * are staged by the driver and the call may return only after them.
 * Independent calls on different streams with different workspaces overlap
 * one call's copies with another's GEMM.  stats may be NULL.  Errors as
 * moa_gemm_ex, plus MOA_ERR_WORKSPACE / MOA_ERR_ALIGN for the workspace;
 * host pointers need only their element alignment.
 * m == 0 or p == 0: MOA_OK, nothing enqueued.  n == 0: hC := 0. */
int moa_gemm_host(int64_t m, int64_t n, int64_t p, moa_dtype dt,
                  const void* hA, const void* hB, void* hC, int slices,
                  void* ws, size_t ws_bytes, void* stream, moa_stats* stats);

/* Bytes of device workspace moa_gemm_host needs: device copies of A, B and C
 * (each rounded up to 256 bytes) plus moa_gemm_workspace_size(...).  0 for
 * an unknown mode or a negative dimension. */
size_t moa_gemm_host_workspace_size(int64_t m, int64_t n, int64_t p, moa_dtype dt, int slices);

/* ---------------------------------------------------------------------- */
/* Grouped GEMM: `count` independent problems of any shapes in one          */
/* persistent launch (the batching pattern).                                */
/* ---------------------------------------------------------------------- */

typedef struct {
    int64_t m, n, p;
    moa_dtype dt;             /* any mode; BF16 problems take the persistent path */
    const void* A;
    const void* B;
    void* C;
} moa_gemm_desc;

/* Workspace bytes for moa_gemm_grouped with these descriptors (device tables
 * of the persistent launch, plus scratch for problems it does not take). */
size_t moa_gemm_grouped_workspace_size(int count, const moa_gemm_desc* descs);

/* Every C_g := A_g . B_g of `descs` (Eq. eq:dnf per problem) on `stream`.
 * BF16 problems with 16-byte row pitches and 16-byte aligned A, B run in ONE
 * persistent tcgen05 launch: each problem gets a tile width from a shape cost
 * model, all output tiles are dealt to the SMs longest-first, and per-problem
 * TMA descriptors live in `ws`.  Modular-slice problems (MOA_F64_CRT_*, with
 * 16-byte aligned A and B) run as one grouped sequence: one exponent and one
 * residue launch per input type over all of them, ONE persistent residue-GEMM
 * launch over every (problem, modulus, tile) unit (longest K first), one
 * reconstruction launch; each result is bit-identical to the problem run
 * alone.  FP32-accuracy split problems (MOA_F32_SPLIT, 16-byte aligned A and
 * B) that a lone call would run without split K (enough tiles for the SMs)
 * share one slice pre-pass launch and ONE persistent slice-GEMM launch over
 * all their tiles (longest K first, each problem at its lone call's tile
 * width), bit-identical to the lone calls.  Other problems (other dtypes,
 * unaligned pitches, few-tile long-K FP32-accuracy problems) run one by one on
 * the same stream.  A call that repeats the
 * previous call of the same thread (identical descriptors, same `ws`, same
 * device) reuses the tables already in `ws`, so callers must not modify `ws`
 * between such calls.  Host-side tables are staged in pinned host memory
 * owned by the library (per thread).  Errors: MOA_ERR_ARG / MOA_ERR_DTYPE for a
 * bad descriptor (nothing launched), MOA_ERR_WORKSPACE if ws is too small. */
int moa_gemm_grouped(int count, const moa_gemm_desc* descs,
                     void* ws, size_t ws_bytes, void* stream);

/* The path a problem takes in moa_gemm_grouped (and in the server's grouped
 * calls): MOA_GROUPED_BF16 (the persistent BF16 launch), MOA_GROUPED_CRT (the
 * grouped modular-slice launches), MOA_GROUPED_F32_SPLIT (the grouped
 * FP32-accuracy split launches) or MOA_GROUPED_ALONE (its own launches on the
 * same stream).  Host-side only.  MOA_ERR_ARG for a NULL descriptor. */
enum { MOA_GROUPED_ALONE = 0, MOA_GROUPED_BF16 = 1, MOA_GROUPED_CRT = 2,
       MOA_GROUPED_F32_SPLIT = 3 };
int moa_grouped_path(const moa_gemm_desc* d);

/* ---------------------------------------------------------------------- */
/* The inner/outer-product family as one algorithm (paper's Appendix)       */
/* ---------------------------------------------------------------------- */

/* With the outer product T[i,j,k,l] = A[i,j] * B[k,l] (A is m x n, B is
 * p x q, row-major), the Hadamard, Kronecker and matrix products are one
 * index map over the output C (R x Q, row-major):
 *     C[r, c] = sum_{s < S} A[r / ra, c / ca + s] * B[r % rb + s, c % cb]
 *   MOA_PRODUCT_HADAMARD   C[i,j] = T[i,j,i,j]       m = p, n = q; R x Q = m x n, S = 1
 *   MOA_PRODUCT_KRONECKER  C[(i*p)+k, (j*q)+l] = T[i,j,k,l]; R x Q = mp x nq, S = 1
 *   MOA_PRODUCT_MATMUL     C[i,l] = sum_j T[i,j,j,l]  n = p; R x Q = m x q, S = n */
typedef enum {
    MOA_PRODUCT_HADAMARD = 0,
    MOA_PRODUCT_KRONECKER = 1,
    MOA_PRODUCT_MATMUL = 2
} moa_product_kind;

/* C := the product `kind` of A and B by the single outer-product kernel:
 * each output element is its sum of S products, each product rounded and the
 * sums added in s order (no fused multiply-add), so MOA_PRODUCT_MATMUL in
 * FP64 follows the oracle's i-k-j order element for element.  dt: MOA_F64
 * (FP64 in/out), MOA_F32_TF32 or MOA_F32_SIMT (FP32 in/out, FP32
 * arithmetic), MOA_BF16 (BF16 in, FP32 out).  The matrix product here is the
 * algebra's reference form on CUDA cores; moa_gemm_ex is its tensor-core
 * specialisation.  Asynchronous on `stream`; MOA_ERR_ARG for mismatched
 * shapes, MOA_ERR_DTYPE for other modes. */
int moa_product(moa_product_kind kind, int64_t m, int64_t n, int64_t p, int64_t q, moa_dtype dt,
                const void* A, const void* B, void* C, void* stream);


/* Kronecker product C := A (x) B: A is m x n, B is p x q, C is (m*p) x (n*q),
 * all row-major, C[(i*p)+k, (j*q)+l] = A[i,j] * B[k,l] (one rounding per
 * element); moa_product(MOA_PRODUCT_KRONECKER, ...).  dt: MOA_F64 (FP64
 * in/out), MOA_F32_TF32 or MOA_F32_SIMT (FP32 in/out, plain FP32 products),
 * MOA_BF16 (BF16 in, FP32 out, exact).  Asynchronous on `stream`.
 * MOA_ERR_DTYPE for other modes. */
int moa_kronecker(int64_t m, int64_t n, int64_t p, int64_t q, moa_dtype dt, const void* A,
                  const void* B, void* C, void* stream);

/* Hadamard product C := A o B of two m x n arrays: C[i,j] = A[i,j] * B[i,j]
 * (moa_product(MOA_PRODUCT_HADAMARD, m, n, m, n, ...)); dtypes as for
 * moa_kronecker.  Asynchronous on `stream`. */
int moa_hadamard(int64_t m, int64_t n, moa_dtype dt, const void* A, const void* B, void* C,
                 void* stream);

/* ---------------------------------------------------------------------- */
/* Batched (3-D) contraction                                                */
/* ---------------------------------------------------------------------- */

/* C[b] := A[b] . B[b] for 0 <= b < batch: the contraction
 *     C[b, i, j] = sum_k A[b, i, k] * B[b, k, j]
 * the higher-dimensional extension of the inner product of Eq. (eq:dnf)
 * (the paper's Appendix).  Entry b of each operand starts stride_x ELEMENTS
 * after entry b - 1 (stride 0 broadcasts one A or B to every entry; C's
 * stride must be >= m * p).  Each entry is row-major m x n, n x p, m x p in
 * mode dt.  BF16 batches with 16-byte row pitches run as one persistent
 * grouped launch; other modes one launch per entry.  Workspace as returned
 * by moa_gemm_batched_workspace_size. */
size_t moa_gemm_batched_workspace_size(int batch, int64_t m, int64_t n, int64_t p, moa_dtype dt,
                                       int64_t stride_a, int64_t stride_b, int64_t stride_c);
int moa_gemm_batched(int batch, int64_t m, int64_t n, int64_t p, moa_dtype dt, const void* A,
                     int64_t stride_a, const void* B, int64_t stride_b, void* C, int64_t stride_c,
                     void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------- */
/* Tile widths of the dense tensor-core GEMMs (MOA_BF16, MOA_F32_TF32)       */
/* ---------------------------------------------------------------------- */

/* The tile is 128 rows x block_n columns; the planner picks block_n from the
 * shape (Sec. 3.4 of the paper: block sizes from the static shapes and types).
 * moa_set_block_n forces block_n for the calling thread's later calls: the
 * dense modes take 64, 128 or 256, the split modes 128, 192 (FP64 accuracy)
 * or 256 (FP32 accuracy); other values leave that mode to its planner.  0
 * restores the planners.  MOA_ERR_ARG for values outside {0,64,128,192,256}. */
int moa_set_block_n(int block_n);

/* Tile height: 128-row tiles on one SM, or 256 x 256 tiles on a pair of SMs
 * (a cluster of two CTAs whose tensor-core MMAs span both: each SM stages
 * half of the operands).  Modular-slice modes (MOA_F64_CRT_*): the planner
 * picks one by a wave-count cost model while the operand planes fit in the
 * L2.  Dense modes (MOA_BF16, MOA_F32_TF32): the planner chooses among
 * 128-row tiles and 256 x 256 tiles on one SM; pair tiles (each SM with a
 * double-buffered accumulator) are available but measured no faster.
 * moa_set_block_m(128 | 256) forces 128-row tiles or pair tiles for the
 * calling thread's later calls (256 implies block_n 256; a forced block_n of
 * 128 implies 128 rows), 0 restores the planners.  Results are identical
 * either way.  MOA_ERR_ARG for values outside {0, 128, 256}. */
int moa_set_block_m(int block_m);

/* Measured refinement of the planner: times C := A . B with every block_n on
 * the caller's buffers (1 warm-up + 3 timed calls each, CUDA events on
 * `stream`, synchronous), records the fastest for the shape bucket of
 * (m, n, p, dt) -- half-octaves of each dimension -- and returns it in
 * *best_block_n (and its time in *best_ms; either may be NULL).  Later calls
 * in the bucket use it.  Leaves C holding the product.  Workspace as for
 * moa_gemm_ex.  MOA_ERR_DTYPE for modes without tile widths. */
int moa_tune_dense(int64_t m, int64_t n, int64_t p, moa_dtype dt, const void* A, const void* B,
                   void* C, void* ws, size_t ws_bytes, void* stream, int* best_block_n,
                   float* best_ms);

/* The tile width (64, 128 or 256) the grouped persistent launch gives a BF16
 * problem of this shape: the width moa_tune_dense recorded for its shape
 * bucket when there is one (or a width forced by moa_set_block_n), else the
 * shape cost model's.  0 for empty shapes. */
int moa_grouped_block_n(int64_t m, int64_t n, int64_t p);

/* Writes / reads / clears the measured table (text: "dt m n p block_n" per
 * line, dimensions as half-octave buckets).  The file named by the
 * MOA_TUNE_CACHE environment variable is loaded on first use. */
int moa_tune_save(const char* path);
int moa_tune_load(const char* path);
int moa_tune_clear(void);

/* ---------------------------------------------------------------------- */
/* Serving: a continuous-batching GEMM server (the serving pattern).        */
/* ---------------------------------------------------------------------- */

typedef struct moa_server moa_server;

typedef struct {
    void* arena;              /* caller-owned device memory for request workspaces */
    size_t arena_bytes;       /* the HBM budget: admitted workspaces never exceed it */
    int max_inflight;         /* most requests on the GPU at once (> 0) */
    int n_streams;            /* CUDA streams the server launches on (1..64) */
    int queue_capacity;       /* most queued requests; submit returns MOA_ERR_BUSY beyond (0 = 65536) */
    double queue_deadline_s;  /* a request queued longer is rejected (0 = never) */
} moa_serve_config;

typedef struct {
    uint64_t ticket;
    int status;               /* MOA_OK, MOA_ERR_REJECTED (deadline) or a launch error */
    moa_dtype dt;
    int64_t m, n, p;
    double t_submit, t_start, t_done;   /* steady-clock seconds */
} moa_completion;

typedef struct {
    uint64_t submitted, admitted, completed, rejected, failed, batches;
    uint64_t queued, inflight;
    int inflight_peak;
    size_t arena_peak, arena_used;
    double p50_ms, p99_ms, max_ms, mean_ms;   /* submit -> done, completed requests */
} moa_serve_counters;

/* Starts a server on the current device: creates its streams, one completion
 * event per in-flight slot and a scheduler thread.  The scheduler polls the
 * completion events without sleeping while requests are queued or in flight
 * (and for 2 ms after the last activity), so a busy server keeps one host
 * core busy; an idle one sleeps until moa_serve_submit wakes it.  The arena
 * (256-byte aligned) stays owned by the caller and must outlive the server;
 * its first 256-byte granules (4 bytes per in-flight slot) hold the slots'
 * device status words, the rest is the request workspace pool.
 * MOA_ERR_ARG / MOA_ERR_ALIGN on a bad config, MOA_ERR_BUDGET if the arena
 * cannot hold the status words. */
int moa_serve_create(const moa_serve_config* cfg, moa_server** out);

/* Queues C := A . B (any moa_dtype; operands and C are device memory that
 * stays resident and valid until the ticket completes).  Non-blocking.  A
 * scheduler thread admits queued requests in FIFO order while fewer than
 * max_inflight run and the request's workspace fits in the free arena; the
 * requests admitted in one pass form a batch (its BF16 requests and its
 * modular-slice and FP32-accuracy split requests of at most 2 GFLOP share one
 * grouped call) spread over the server's streams, so requests
 * arriving while others run overlap with them on the device.  Returns MOA_OK
 * (queued), MOA_ERR_BUDGET (the workspace alone exceeds the arena),
 * MOA_ERR_BUSY (queue full), MOA_ERR_ARG / MOA_ERR_DTYPE (bad descriptor).
 * Every queued ticket completes exactly once. */
int moa_serve_submit(moa_server* s, const moa_gemm_desc* d, uint64_t* ticket);

/* Moves up to `max` completions into `out`; *n_out = how many. */
int moa_serve_poll(moa_server* s, moa_completion* out, int max, int* n_out);

/* Counters, arena use and latency percentiles of the completed requests. */
int moa_serve_stats(moa_server* s, moa_serve_counters* out);

/* Stops accepting, drains every queued and in-flight request, joins the
 * scheduler, destroys the streams and frees the server (not the arena). */
int moa_serve_destroy(moa_server* s);

/* ---------------------------------------------------------------------- */
/* Allocation-free variant                                                  */
/* ---------------------------------------------------------------------- */

/* C := A . B in the FP32-accuracy split mode (as moa_gemm_ex with
 * MOA_F32_SPLIT), for callers that may not allocate device memory at all:
 * real-time or safety-certified hosts whose device memory is fixed at
 * start-up (a run-time cudaMalloc can block, synchronise the device or fail
 * late), plugins inside another runtime's memory pool that are handed no
 * allocator, and deployments with a static memory plan.  The paper has no
 * counterpart; this is a deployment convenience of this library.
 *
 * A (m x n), B (n x p) and C (m x p) are FP32 row-major device arrays owned by
 * the caller, A and B 16-byte aligned.  The scratch (three BF16 slice planes
 * of A and of B; for few-tile problems also split-K counters and FP32 partial
 * tiles) lives in one static device array of 32 MiB that every GPU loading
 * this library holds until exit; problems whose scratch does not fit
 * (moa_gemm_workspace_size(m, n, p, MOA_F32_SPLIT, 0) > 32 MiB) are rejected
 * with MOA_ERR_WORKSPACE and nothing is launched.  No cudaMalloc, cudaFree or
 * allocating library routine is called.
 *
 * The first call on each device (with that device current) looks up the
 * array's device address with cudaGetSymbolAddress; make that first call
 * before any stream capture begins.  All calls share the array and find the
 * previous call's contents there; each call clears what must start at zero
 * (the split-K counters) on its own stream.  Calls whose work overlaps on the
 * GPU (other streams, unordered host threads) race on the array, so
 * serialise them.  Asynchronous on `stream` like moa_gemm_ex. */
int moa_gemm_f32split_noalloc(int64_t m, int64_t n, int64_t p, const float* A, const float* B,
                              float* C, void* stream);

/* ---------------------------------------------------------------------- */
/* Status and housekeeping                                                 */
/* ---------------------------------------------------------------------- */

/* Synchronises `stream`, then returns and clears the current device's
 * status word: MOA_OK, MOA_ERR_TIMEOUT (a kernel gave up on a pipeline
 * wait), MOA_ERR_NONFINITE (a split pre-pass saw NaN/Inf) or MOA_ERR_CUDA
 * (the synchronisation itself failed, or, with MOA_DEBUG_CANARY=1 set in
 * the environment, a call wrote into the guard bytes past its workspace). */
int moa_sync_status(void* stream);

/* Thread-local message describing the last non-OK status of this thread. */
const char* moa_last_error(void);

/* Per-wait time limit of device pipeline waits, in nanoseconds
 * (default 2e9; also read from the MOA_WAIT_LIMIT_NS environment variable).
 * Returns the previous value. */
uint64_t moa_set_wait_limit_ns(uint64_t ns);

/* Profiling hook for the calling thread: when both are non-NULL cudaEvent_t
 * handles, every later GEMM call of this thread records `start_event`
 * immediately before its main kernel (the tensor-core or CUDA-core GEMM, not
 * the pre-passes) and `stop_event` immediately after it, on the call's stream.
 * Pass NULL, NULL to stop.  The events stay owned by the caller.  Returns MOA_OK. */
int moa_profile_events(void* start_event, void* stop_event);

/* Failure-detection self-test: launches one CTA whose pipeline wait (the
 * bounded mbarrier wait every tensor-core kernel uses) waits for an arrival
 * that never comes; after `limit_ns` (0 < limit_ns <= 10 s) the kernel records
 * the timeout in the device status word and returns, leaving the context
 * usable.  A following moa_sync_status(stream) returns MOA_ERR_TIMEOUT.
 * Diagnostic only; the paper has no counterpart. */
int moa_selftest_wait_timeout(uint64_t limit_ns, void* stream);

/* Measured FP64 rate of this device (the roofline denominator of the native
 * FP64 mode): kind 0 = independent fused multiply-adds on the CUDA cores,
 * kind 1 = independent warp-level FP64 MMAs (mma.sync m16n8k4, the FP64
 * tensor path).  Runs a short warm-up launch and five launches of about
 * 1.5e10 flops (a GEMM kernel's length) on `stream`, each timed with CUDA
 * events (synchronous: returns after them), and writes the best rate in
 * TFLOP/s to *tflops.  Allocates nothing.  MOA_ERR_ARG for another kind or a
 * NULL tflops.  Diagnostic only. */
int moa_measure_fp64_rate(int kind, void* stream, double* tflops);

/* Library version string. */
const char* moa_version(void);

/* Frees moa_gemm()'s internal workspace on every device that has one. */
void moa_shutdown(void);

#ifdef __cplusplus
}
#endif

#endif /* MOA_H_ */
