// fpbits.cuh -- bit-level views of FP32 / FP64 values shared by the
// pre-passes of the FP64-accuracy modes: magnitude bit patterns (whose
// integer order is the order of the magnitudes), frexp exponents from them,
// and the round-half-even scaling of an FP64 value to an integer.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace moa {

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
};

}  // namespace moa
