// fastdiv.cuh -- n / d and n % d for 32-bit n < 2^31 by a precomputed
// reciprocal, for index arithmetic in memory-bound kernels (a 32- or 64-bit
// integer division costs tens of instructions).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace moa {

// m = floor(2^32 / d) (2^32 - 1 for d = 1) gives floor(n m / 2^32) in
// {q - 1, q} for n < 2^31, and one correction step makes it exact.
struct FastDiv {
    uint32_t d, m;
};
inline FastDiv make_fastdiv(uint32_t d) {
    return FastDiv{d, d <= 1 ? 0xFFFFFFFFu : static_cast<uint32_t>((uint64_t(1) << 32) / d)};
}
__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f, uint32_t& rem) {
    uint32_t q = __umulhi(n, f.m);
    uint32_t r = n - q * f.d;
    if (r >= f.d) {
        ++q;
        r -= f.d;
    }
    rem = r;
    return q;
}

}  // namespace moa
