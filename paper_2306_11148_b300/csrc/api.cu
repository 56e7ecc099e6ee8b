// api.cu -- the C ABI entry points of libmoa.so for single GEMMs (include/moa.h):
// argument validation, workspace sizing, the padding of row pitches that TMA
// cannot address, and dispatch to the kernels of each precision mode.
//
// The operation is Eq. (eq:dnf) of Sec. 2 over the row-major shapes of
// Eqs. (eq:shapes)/(eq:indices); C is assigned (callers need not clear it).
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>
#include <string>

#include "crt.h"
#include "internal.h"
#include "split.h"

namespace moa {
namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

int in_size(moa_dtype dt) { return dtype_in_bytes(dt); }
int out_size(moa_dtype dt) { return dtype_out_bytes(dt); }

bool is_tc_dense(moa_dtype dt) { return dt == MOA_BF16 || dt == MOA_F32_TF32; }

// Elements per 16 bytes: TMA needs row pitches that are multiples of 16 bytes.
int64_t tma_pitch(int64_t cols, int esize) { return round_up(cols, 16 / esize); }

struct DenseWs {
    bool pad_a, pad_b, trans_b;
    int64_t lda, ldb;
    size_t a_bytes, b_bytes, total;
};

// BF16: A and B are read in place unless a row pitch is not a multiple of 16
// bytes (then copied to a padded pitch).  TF32: B is always transposed into
// the workspace (p x round_up(n, 4)), because the TF32 MMA reads K-major B only.
DenseWs dense_ws(int64_t m, int64_t n, int64_t p, moa_dtype dt) {
    DenseWs w{};
    const int es = in_size(dt);
    w.lda = tma_pitch(n, es);
    w.pad_a = w.lda != n;
    w.a_bytes = w.pad_a ? align_up(static_cast<size_t>(m) * w.lda * es) : 0;
    if (!w.pad_a) w.lda = n;
    if (dt == MOA_F32_TF32) {
        w.trans_b = true;
        w.ldb = tma_pitch(n, es);
        w.b_bytes = align_up(static_cast<size_t>(p) * w.ldb * es);
    } else {
        w.ldb = tma_pitch(p, es);
        w.pad_b = w.ldb != p;
        w.b_bytes = w.pad_b ? align_up(static_cast<size_t>(n) * w.ldb * es) : 0;
        if (!w.pad_b) w.ldb = p;
    }
    w.total = w.a_bytes + w.b_bytes;
    return w;
}

int validate(int64_t m, int64_t n, int64_t p, int dt, const void* A, const void* B, const void* C) {
    if (!valid_dtype(dt)) return fail(MOA_ERR_DTYPE, "unknown moa_dtype");
    if (m < 0 || n < 0 || p < 0) return fail(MOA_ERR_ARG, "negative dimension");
    if (m > (int64_t(1) << 31) || n > (int64_t(1) << 31) || p > (int64_t(1) << 31))
        return fail(MOA_ERR_ARG, "dimension above 2^31");
    const moa_dtype d = static_cast<moa_dtype>(dt);
    if (m > 0 && p > 0 && C == nullptr) return fail(MOA_ERR_ARG, "C is NULL");
    if (m > 0 && p > 0 && n > 0 && (A == nullptr || B == nullptr))
        return fail(MOA_ERR_ARG, "A or B is NULL");
    const uintptr_t ia = reinterpret_cast<uintptr_t>(A), ib = reinterpret_cast<uintptr_t>(B),
                    ic = reinterpret_cast<uintptr_t>(C);
    if (ia % in_size(d) || ib % in_size(d) || ic % out_size(d))
        return fail(MOA_ERR_ALIGN, "pointer not aligned to its element size");
    if ((is_tc_dense(d) || is_split(d) || is_crt(d)) && m > 0 && n > 0 && p > 0 &&
        (ia % 16 || ib % 16))
        return fail(MOA_ERR_ALIGN, "tensor-core modes need 16-byte aligned A and B");
    return MOA_OK;
}

// Library-owned workspace of moa_gemm(), one per device.
std::mutex g_ws_mu;
constexpr int kMaxDev = 64;
void* g_ws[kMaxDev] = {nullptr};
size_t g_ws_bytes[kMaxDev] = {0};

}  // namespace

// The host-side argument checks of moa_gemm_ex (mode, sizes, pointers,
// alignment), for entry points that size their scratch before dispatching.
int validate_gemm_args(int64_t m, int64_t n, int64_t p, int dt, const void* A, const void* B,
                       const void* C) {
    return validate(m, n, p, dt, A, B, C);
}

size_t workspace_bytes(int64_t m, int64_t n, int64_t p, moa_dtype dt, int slices) {
    if (m <= 0 || p <= 0 || n <= 0) return 0;
    if (is_tc_dense(dt)) return dense_ws(m, n, p, dt).total;
    if (is_split(dt)) return split_workspace_bytes(m, n, p, dt, slices);
    if (is_crt(dt)) return crt_workspace_bytes(m, n, p, dt, slices);
    return 0;
}

int gemm_ex_impl(int64_t m, int64_t n, int64_t p, moa_dtype dt, const void* A, const void* B,
                 void* C, int slices, void* ws, size_t ws_bytes, cudaStream_t s, moa_stats* st);

int gemm_ex(int64_t m, int64_t n, int64_t p, moa_dtype dt, const void* A, const void* B, void* C,
            int slices, void* ws, size_t ws_bytes, cudaStream_t s, moa_stats* st) {
    if (canary_enabled() && ws && m > 0 && n > 0 && p > 0) {
        const size_t need = (workspace_bytes(m, n, p, dt, slices) + kAlign - 1) / kAlign * kAlign;
        if (ws_bytes >= need + kCanaryBytes) {
            void* guard = static_cast<uint8_t*>(ws) + need;
            int rc = canary_arm(guard, s);
            if (rc != MOA_OK) return rc;
            rc = gemm_ex_impl(m, n, p, dt, A, B, C, slices, ws, need, s, st);
            const int rc2 = canary_check(guard, s);
            return rc != MOA_OK ? rc : rc2;
        }
    }
    return gemm_ex_impl(m, n, p, dt, A, B, C, slices, ws, ws_bytes, s, st);
}

int gemm_ex_impl(int64_t m, int64_t n, int64_t p, moa_dtype dt, const void* A, const void* B,
                 void* C, int slices, void* ws, size_t ws_bytes, cudaStream_t s, moa_stats* st) {
    int rc = validate(m, n, p, dt, A, B, C);
    if (rc != MOA_OK) return rc;
    if (st) {
        *st = moa_stats{};
        st->slices = 1;
        st->products = 1;
    }
    if (m == 0 || p == 0) return MOA_OK;
    if (n == 0) {
        cudaError_t e = cudaMemsetAsync(C, 0, static_cast<size_t>(m) * p * out_size(dt), s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(C)");
        if (st) st->kernels = 0;   // a memset of C, no kernel
        return MOA_OK;
    }
    const size_t need = workspace_bytes(m, n, p, dt, slices);
    if (need > 0 && (ws == nullptr || ws_bytes < need)) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "workspace of %zu bytes needed, %zu given", need,
                      ws ? ws_bytes : size_t(0));
        return fail(MOA_ERR_WORKSPACE, buf);
    }
    if (ws && reinterpret_cast<uintptr_t>(ws) % kAlign)
        return fail(MOA_ERR_ALIGN, "workspace must be 256-byte aligned");
    switch (dt) {
        case MOA_F64:
            if (st) st->kernels = 1;
            return simt_f64_launch(m, n, p, static_cast<const double*>(A),
                                   static_cast<const double*>(B), static_cast<double*>(C), s);
        case MOA_F32_SIMT:
            if (st) st->kernels = 1;
            return simt_f32_launch(m, n, p, static_cast<const float*>(A),
                                   static_cast<const float*>(B), static_cast<float*>(C), s);
        case MOA_BF16:
        case MOA_F32_TF32: {
            const DenseWs w = dense_ws(m, n, p, dt);
            const int es = in_size(dt);
            const void* a = A;
            const void* b = B;
            uint8_t* base = static_cast<uint8_t*>(ws);
            int kernels = 0;
            if (w.pad_a) {
                rc = pad_copy_launch(A, base, m, n, w.lda, es, s);
                if (rc != MOA_OK) return rc;
                a = base;
                ++kernels;
            }
            if (w.trans_b) {
                rc = transpose_pad_launch(static_cast<const float*>(B), n, p,
                                          reinterpret_cast<float*>(base + w.a_bytes), w.ldb, s);
                if (rc != MOA_OK) return rc;
                b = base + w.a_bytes;
                ++kernels;
            } else if (w.pad_b) {
                rc = pad_copy_launch(B, base + w.a_bytes, n, p, w.ldb, es, s);
                if (rc != MOA_OK) return rc;
                b = base + w.a_bytes;
                ++kernels;
            }
            rc = dense_tc_launch(dt == MOA_BF16, m, n, p, a, w.lda, b, w.ldb,
                                 static_cast<float*>(C), s, st);
            if (st) {
                st->kernels += kernels;
                st->padded = (w.pad_a || w.pad_b) ? 1 : 0;
            }
            return rc;
        }
        case MOA_F64_CRT_F32IN:
        case MOA_F64_CRT_F64IN:
            return crt_gemm(m, n, p, dt, A, B, C, slices, ws, ws_bytes, s, st);
        default:
            return split_gemm(m, n, p, dt, A, B, C, slices, ws, ws_bytes, s, st);
    }
}

}  // namespace moa

extern "C" {

size_t moa_gemm_workspace_size(int64_t m, int64_t n, int64_t p, moa_dtype dt, int slices) {
    if (!moa::valid_dtype(dt) || m < 0 || n < 0 || p < 0) return 0;
    return moa::workspace_bytes(m, n, p, dt, slices);
}

int moa_gemm_ex(int64_t m, int64_t n, int64_t p, moa_dtype dt, const void* A, const void* B,
                void* C, int slices, void* ws, size_t ws_bytes, void* stream, moa_stats* stats) {
    moa::TraceRange tr("moa_gemm_ex");
    return moa::gemm_ex(m, n, p, dt, A, B, C, slices, ws, ws_bytes,
                        static_cast<cudaStream_t>(stream), stats);
}

}  // extern "C"

// ---------------------------------------------------------------- host buffers
// Workspace of moa_gemm_host: device copies of A, B and C, then the mode's
// own workspace (each region 256-byte aligned).
namespace moa {
namespace {
struct HostLayout {
    size_t a_bytes, b_bytes, c_bytes;
    size_t a_off, b_off, c_off, g_off, total;
};
HostLayout host_layout(int64_t m, int64_t n, int64_t p, moa_dtype dt, int slices) {
    auto al = [](size_t x) { return (x + kAlign - 1) / kAlign * kAlign; };
    HostLayout L{};
    L.a_bytes = static_cast<size_t>(m) * n * in_size(dt);
    L.b_bytes = static_cast<size_t>(n) * p * in_size(dt);
    L.c_bytes = static_cast<size_t>(m) * p * out_size(dt);
    L.a_off = 0;
    L.b_off = al(L.a_bytes);
    L.c_off = L.b_off + al(L.b_bytes);
    L.g_off = L.c_off + al(L.c_bytes);
    L.total = L.g_off + workspace_bytes(m, n, p, dt, slices);
    return L;
}
}  // namespace
}  // namespace moa

extern "C" {

size_t moa_gemm_host_workspace_size(int64_t m, int64_t n, int64_t p, moa_dtype dt, int slices) {
    if (!moa::valid_dtype(dt) || m < 0 || n < 0 || p < 0) return 0;
    if (m > (int64_t(1) << 31) || n > (int64_t(1) << 31) || p > (int64_t(1) << 31)) return 0;
    return moa::host_layout(m, n, p, dt, slices).total;
}

int moa_gemm_host(int64_t m, int64_t n, int64_t p, moa_dtype dt, const void* hA, const void* hB,
                  void* hC, int slices, void* ws, size_t ws_bytes, void* stream,
                  moa_stats* stats) {
    moa::TraceRange tr("moa_gemm_host");
    if (!moa::valid_dtype(dt)) return moa::fail(MOA_ERR_DTYPE, "unknown moa_dtype");
    if (m < 0 || n < 0 || p < 0) return moa::fail(MOA_ERR_ARG, "negative dimension");
    if (m > (int64_t(1) << 31) || n > (int64_t(1) << 31) || p > (int64_t(1) << 31))
        return moa::fail(MOA_ERR_ARG, "dimension above 2^31");
    if (m > 0 && p > 0 && hC == nullptr) return moa::fail(MOA_ERR_ARG, "C is NULL");
    if (m > 0 && p > 0 && n > 0 && (hA == nullptr || hB == nullptr))
        return moa::fail(MOA_ERR_ARG, "A or B is NULL");
    if (stats) *stats = moa_stats{};
    if (m == 0 || p == 0) return MOA_OK;
    const moa::HostLayout L = moa::host_layout(m, n, p, dt, slices);
    if (ws_bytes < L.total || ws == nullptr)
        return moa::fail(MOA_ERR_WORKSPACE, "workspace smaller than moa_gemm_host_workspace_size");
    if (reinterpret_cast<uintptr_t>(ws) % moa::kAlign)
        return moa::fail(MOA_ERR_ALIGN, "workspace not 256-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint8_t* base = static_cast<uint8_t*>(ws);
    void* dA = base + L.a_off;
    void* dB = base + L.b_off;
    void* dC = base + L.c_off;
    // modular slices: B once, then A in bands whose uploads, GEMMs and
    // downloads overlap
    if (moa::is_crt(dt) && n > 0)
        return moa::crt_gemm_host(m, n, p, dt, hA, hB, hC, slices, dA, dB, dC, base + L.g_off,
                                  ws_bytes - L.g_off, s, stats);
    cudaError_t e = cudaSuccess;
    if (L.a_bytes) e = cudaMemcpyAsync(dA, hA, L.a_bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && L.b_bytes) e = cudaMemcpyAsync(dB, hB, L.b_bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return moa::cuda_fail(e, "cudaMemcpyAsync(A, B to the device)");
    const int rc = moa::gemm_ex(m, n, p, dt, n ? dA : nullptr, n ? dB : nullptr, dC, slices,
                                base + L.g_off, ws_bytes - L.g_off, s, stats);
    if (rc != MOA_OK) return rc;
    e = cudaMemcpyAsync(hC, dC, L.c_bytes, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return moa::cuda_fail(e, "cudaMemcpyAsync(C to the host)");
    return MOA_OK;
}

int moa_gemm(int64_t m, int64_t n, int64_t p, moa_dtype dt, const void* A, const void* B, void* C) {
    moa::TraceRange tr("moa_gemm");
    int rc = moa::validate(m, n, p, dt, A, B, C);
    if (rc != MOA_OK) return rc;
    size_t need = moa::workspace_bytes(m, n, p, dt, 0);
    // room for the guard bytes of MOA_DEBUG_CANARY
    if (need > 0 && moa::canary_enabled())
        need = (need + moa::kAlign - 1) / moa::kAlign * moa::kAlign + moa::kCanaryBytes;
    void* ws = nullptr;
    if (need > 0) {
        int d = 0;
        cudaError_t e = cudaGetDevice(&d);
        if (e != cudaSuccess) return moa::cuda_fail(e, "cudaGetDevice");
        if (d < 0 || d >= moa::kMaxDev) return moa::fail(MOA_ERR_CUDA, "device index out of range");
        std::lock_guard<std::mutex> lk(moa::g_ws_mu);
        if (moa::g_ws_bytes[d] < need) {
            if (moa::g_ws[d]) {
                // The legacy default stream orders this after earlier work.
                cudaStreamSynchronize(nullptr);
                cudaFree(moa::g_ws[d]);
                moa::g_ws[d] = nullptr;
                moa::g_ws_bytes[d] = 0;
            }
            e = cudaMalloc(&moa::g_ws[d], need);
            if (e != cudaSuccess) return moa::cuda_fail(e, "cudaMalloc(moa_gemm workspace)");
            moa::g_ws_bytes[d] = need;
        }
        ws = moa::g_ws[d];
        return moa::gemm_ex(m, n, p, dt, A, B, C, 0, ws, moa::g_ws_bytes[d], nullptr, nullptr);
    }
    return moa::gemm_ex(m, n, p, dt, A, B, C, 0, nullptr, 0, nullptr, nullptr);
}

void moa_shutdown(void) {
    std::lock_guard<std::mutex> lk(moa::g_ws_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (int d = 0; d < moa::kMaxDev; ++d) {
        if (moa::g_ws[d]) {
            cudaSetDevice(d);
            cudaDeviceSynchronize();
            cudaFree(moa::g_ws[d]);
            moa::g_ws[d] = nullptr;
            moa::g_ws_bytes[d] = 0;
        }
    }
    cudaSetDevice(cur);
}

}  // extern "C"
