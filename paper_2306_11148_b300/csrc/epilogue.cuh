// epilogue.cuh -- coalesced stores of FP32 accumulator blocks read from TMEM.
//
// A tcgen05.ld 32x32b load leaves one ROW of a 32 x 32 block in each lane
// (lane = TMEM lane = output row).  Storing straight from there makes every
// warp store touch 32 rows x 16 bytes.  store_block32 passes the block
// through a 4 KB shared-memory tile instead (16-byte chunks XOR-swizzled by
// row, so that both the row-wise writes and the column-wise reads run at the
// minimum number of shared-memory wavefronts) and writes it back so that each
// warp store covers 4 rows x 128 contiguous bytes of the row-major C
// (C[(i*p)+j], Eq. (eq:dnf)).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace moa {

// stage: this warp's 4 KB staging tile (16-byte aligned, not shared with other
// warps).  r: the lane's row of the block (32 FP32 bit patterns).  The block's
// top-left element is C[row0, col0] of a row-major C with pitch ld; rows_left /
// cols_left: rows and columns of the block that lie inside C.  vec: ld is a
// multiple of 4 and C is 16-byte aligned (col0 is a multiple of 32).
__device__ __forceinline__ void store_block32(uint8_t* stage, const uint32_t (&r)[32], float* C,
                                              int64_t ld, int64_t row0, int rows_left,
                                              int64_t col0, int64_t cols_left, bool vec) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int v = 0; v < 8; ++v)
        *reinterpret_cast<uint4*>(stage + lane * 128 + ((v ^ (lane & 7)) << 4)) =
            make_uint4(r[4 * v], r[4 * v + 1], r[4 * v + 2], r[4 * v + 3]);
    __syncwarp();
    const int v = lane & 7;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int rr = 4 * i + (lane >> 3);
        const uint4 x = *reinterpret_cast<const uint4*>(stage + rr * 128 + ((v ^ (rr & 7)) << 4));
        if (rr < rows_left) {
            float* dst = C + (row0 + rr) * ld + col0 + 4 * v;
            const int64_t cl = cols_left - 4 * v;
            if (vec && cl >= 4) {
                *reinterpret_cast<uint4*>(dst) = x;
            } else {
                if (cl > 0) dst[0] = __uint_as_float(x.x);
                if (cl > 1) dst[1] = __uint_as_float(x.y);
                if (cl > 2) dst[2] = __uint_as_float(x.z);
                if (cl > 3) dst[3] = __uint_as_float(x.w);
            }
        }
    }
    __syncwarp();   // the staging tile is free for the next block
}

}  // namespace moa
