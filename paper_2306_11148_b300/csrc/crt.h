// crt.h -- the FP64-accuracy modular-slice modes (MOA_F64_CRT_F32IN,
// MOA_F64_CRT_F64IN), internal to libmoa.so.
#pragma once
#include "internal.h"

namespace moa {

inline bool is_crt(moa_dtype dt) { return dt == MOA_F64_CRT_F32IN || dt == MOA_F64_CRT_F64IN; }

// Modulus counts: 8..16 accepted (the product of the moduli stays below
// 2^128); by default the fewest from 14 that keep t >= 47 bits per operand
// (14 up to n = 36639, 15 up to n = 7218057, 16 beyond).
constexpr int kCrtMinModuli = 8;
constexpr int kCrtMaxModuli = 16;
constexpr int kCrtDefaultModuli = 14;

// Modulus count for a call (slices = 0: the default for this n); -1 if the
// count is not allowed.
int crt_moduli_for(moa_dtype dt, int64_t n, int slices);
// Largest t <= 62 with n * 2^(2t+1) < P (P the product of the first M moduli);
// -1 if none.
int crt_bits(int64_t n, int M);

size_t crt_workspace_bytes(int64_t m, int64_t n, int64_t p, moa_dtype dt, int slices);

int crt_gemm(int64_t m, int64_t n, int64_t p, moa_dtype dt, const void* A, const void* B, void* C,
             int slices, void* ws, size_t ws_bytes, cudaStream_t s, moa_stats* st);

// moa_gemm_host for the modular-slice modes (m, n, p > 0): host A, B, C;
// device copies dA, dB, dC; ws / ws_bytes as for crt_gemm.  B is uploaded
// and its passes run once; then A's rows go through in bands of about 2048
// rows, each band's upload, passes + GEMM + reconstruction and download on
// their own streams, so that they overlap; `s` ends after all of it (a
// problem of one band runs in order on `s` alone).  The result equals
// crt_gemm's bit for bit.
int crt_gemm_host(int64_t m, int64_t n, int64_t p, moa_dtype dt, const void* hA, const void* hB,
                  void* hC, int slices, void* dA, void* dB, void* dC, void* ws, size_t ws_bytes,
                  cudaStream_t s, moa_stats* st);

// Grouped calls (moa_gemm_grouped): the modular-slice problems of a call that
// this path takes (positive sizes, 16-byte aligned A and B, 8-byte aligned C)
// run as one exponent and one residue launch per input type, ONE persistent
// residue GEMM launch over every (problem, modulus, tile) unit and one
// reconstruction launch.  Each problem's result is bit-identical to the same
// problem run alone.
bool crt_grouped_ok(const moa_gemm_desc& d);
size_t crt_grouped_workspace(int count, const moa_gemm_desc* d);
// Runs the problems of d[] that crt_grouped_ok takes; `ws` must hold
// crt_grouped_workspace(count, d) bytes.  status (may be NULL): a device
// status word per descriptor, where that problem's non-finite inputs are
// recorded (pipeline timeouts, which belong to the shared launch, go to the
// launch's word).
int crt_grouped_launch(int count, const moa_gemm_desc* d, void* ws, size_t ws_bytes,
                       cudaStream_t s, int* const* status = nullptr);

// Workspace layout of a modular-slice call (byte offsets from the base).
struct CrtLayout {
    int M;                  // moduli
    int ks_max;             // most K slices per tile the residue planes hold
    int64_t lda, ldb, ldr;  // row pitches: A / B residue planes (BF16 elements),
                            // output residue planes (bytes)
    size_t a_off, b_off;    // M x m x lda and M x n x ldb BF16 residues of A' and B'
    size_t ea_off, eb_off;  // per-row / per-column exponents (int32)
    size_t cmax_off;        // per-column max |B| bit patterns (8 bytes each)
    size_t r_off;           // residues of the product: (M * ks_max) x m x ldr bytes
    size_t total;
};
CrtLayout crt_layout(int64_t m, int64_t n, int64_t p, int M);

}  // namespace moa
