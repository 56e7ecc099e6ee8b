// grouped.cu -- moa_gemm_grouped: `count` independent ONF GEMMs of arbitrary
// shapes (Eq. (eq:dnf) per problem).  This first version validates every
// descriptor and issues the problems one after another on the stream.
#include <cuda_runtime.h>

#include "internal.h"

namespace moa {
int gemm_ex(int64_t m, int64_t n, int64_t p, moa_dtype dt, const void* A, const void* B, void* C,
            int slices, void* ws, size_t ws_bytes, cudaStream_t s, moa_stats* st);
size_t workspace_bytes(int64_t m, int64_t n, int64_t p, moa_dtype dt, int slices);
}  // namespace moa

extern "C" {

size_t moa_gemm_grouped_workspace_size(int count, const moa_gemm_desc* d) {
    if (count <= 0 || d == nullptr) return 0;
    size_t mx = 0;
    for (int g = 0; g < count; ++g) {
        const size_t w = moa::workspace_bytes(d[g].m, d[g].n, d[g].p, d[g].dt, 0);
        if (w > mx) mx = w;
    }
    return mx;
}

int moa_gemm_grouped(int count, const moa_gemm_desc* d, void* ws, size_t ws_bytes, void* stream) {
    if (count < 0) return moa::fail(MOA_ERR_ARG, "negative count");
    if (count == 0) return MOA_OK;
    if (d == nullptr) return moa::fail(MOA_ERR_ARG, "descriptor array is NULL");
    for (int g = 0; g < count; ++g) {
        const int rc = moa::gemm_ex(d[g].m, d[g].n, d[g].p, d[g].dt, d[g].A, d[g].B, d[g].C, 0, ws,
                                    ws_bytes, static_cast<cudaStream_t>(stream), nullptr);
        if (rc != MOA_OK) return rc;
    }
    return MOA_OK;
}

}  // extern "C"
