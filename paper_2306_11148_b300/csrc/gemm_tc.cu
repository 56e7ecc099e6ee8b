// gemm_tc.cu -- dense ONF GEMM on the 5th-generation tensor cores (tcgen05).
//
// C[(i*p)+j] := sum_k A[(i*n)+k] * B[(k*p)+j]   (Eq. (eq:dnf), Sec. 2)
//
// Dimension lifting (Sec. 3.1) mapped onto the B300:
//   * the i loop is split into 128- or 256-row tiles (128 rows per TMEM lane
//     set; a 256-row tile runs two M = 128 MMAs per K step on one staged B
//     tile), the j loop into BLOCK_N-column tiles (the MMA N extent), so that
//     each output tile is an independent block product (Fig. fig:omega);
//   * the sigma (k) loop is split into K blocks of 128 bytes of operand each,
//     summed into the same TMEM accumulator (the "extra summation loop" that
//     closes Sec. 3.1);
//   * output tiles are dealt round-robin to persistent CTAs, one per SM, in a
//     grouped raster order so that neighbouring CTAs share A rows and B
//     columns in L2 (the L2-level lift of Sec. 3.4);
//   * the tile shape is chosen per problem by a wave-count cost model (the
//     block-size model of Sec. 3.4).
// Both operands are read exactly as the ONF lays them out: A row strips are
// K-major (contiguous in k), B row strips are MN-major (contiguous in j, the
// "row of B" of Fig. fig:mm).  TMA stages them into 128-byte-swizzled shared
// memory; one thread issues tcgen05.mma; the epilogue warps (one or two per
// TMEM lane quadrant) drain the accumulator (double-buffered for 128-row
// tiles, so the next tile's MMAs overlap the stores) and write C through a
// shared-memory staging tile in coalesced row segments.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>

#include "epilogue.cuh"
#include "internal.h"
#include "ptx.cuh"

namespace moa {
namespace {

struct DenseArgs {
    float* C;
    int64_t m, n, p;
    int tiles_m, tiles_n, num_kb;
    int group_m;
    int vec_ok;
    uint64_t wait_limit_ns;
    int* status;
};

__device__ __forceinline__ void tile_coords(int t, int tiles_m, int tiles_n, int group_m, int& tm,
                                            int& tn) {
    const int per_group = group_m * tiles_n;
    const int g = t / per_group;
    const int first_m = g * group_m;
    const int gsize = min(tiles_m - first_m, group_m);
    const int r = t - g * per_group;
    tm = first_m + r % gsize;
    tn = r / gsize;
}

// MT: 128-row halves per CTA tile.  MT = 1: 128 x BLOCK_N tiles with a
// double-buffered TMEM accumulator (the next tile's MMAs overlap the
// stores).  MT = 2: 256 x BLOCK_N tiles, two M = 128 MMAs per K step sharing
// each staged B tile (a third fewer operand bytes per flop, so the same
// shared memory buffers more MMA time), single-buffered accumulators (all
// 512 TMEM columns) drained by eight epilogue warps.
template <int ESIZE, int BLOCK_N, int STAGES, int BKM, int MT = 1>
struct DenseCfg {
    static constexpr int BLOCK_M = 128 * MT;
    static constexpr int BK = 128 / ESIZE;          // K elements per stage (128 bytes)
    static constexpr int MMA_K = 32 / ESIZE;        // K per tcgen05.mma (32 bytes)
    static constexpr int CHUNK_N = 128 / ESIZE;     // B columns per 128-byte swizzle row
    static constexpr int CHUNK_BYTES = BK * 128;    // one B column chunk: BK rows x 128 B
    static constexpr int A_BYTES = BLOCK_M * 128;
    static constexpr int B_BYTES = BLOCK_N * BK * ESIZE;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int NBUF = MT == 1 ? 2 : 1;   // accumulator buffers
    static constexpr int TMEM_COLS = 2 * BLOCK_N <= 32 ? 32 : (2 * BLOCK_N <= 64 ? 64 : (2 * BLOCK_N <= 128 ? 128 : (2 * BLOCK_N <= 256 ? 256 : 512)));
    static constexpr int EPI_WARPS = 4 * MT;
    static constexpr int THREADS = 64 + 32 * EPI_WARPS;
    static constexpr int OUT_STAGE = EPI_WARPS * 4096;   // 4 KB store staging per epilogue warp
    static constexpr int SMEM = 1024 + STAGES * STAGE_BYTES + OUT_STAGE + 256;
    static constexpr uint32_t IDESC =
        make_idesc(ESIZE == 2 ? 1u : 2u, 128, BLOCK_N, 0u, BKM ? 0u : 1u);
};

// BKM = 0: B staged MN-major (row-major n x p, contiguous in j).
// BKM = 1: B staged K-major from its transpose (p x n), for the TF32 kind,
//          whose MMA does not read MN-major operands.
template <int ESIZE, int BLOCK_N, int STAGES, int BKM, int MT>
__global__ void __launch_bounds__(DenseCfg<ESIZE, BLOCK_N, STAGES, BKM, MT>::THREADS, 1)
    dense_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    const DenseArgs args) {
    using Cfg = DenseCfg<ESIZE, BLOCK_N, STAGES, BKM, MT>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                               ~static_cast<uintptr_t>(1023));
    uint8_t* sA = smem;
    uint8_t* sB = smem + STAGES * Cfg::A_BYTES;
    uint8_t* out_stage = sB + STAGES * Cfg::B_BYTES;
    uint64_t* bars = reinterpret_cast<uint64_t*>(out_stage + Cfg::OUT_STAGE);
    uint64_t* full = bars;
    uint64_t* empty = bars + STAGES;
    uint64_t* tfull = bars + 2 * STAGES;
    uint64_t* tempty = tfull + 2;
    uint64_t* drain = tempty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    CtaCtl* ctl = reinterpret_cast<CtaCtl*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint64_t limit = args.wait_limit_ns;
    int* status = args.status;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], Cfg::EPI_WARPS);
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
        tmem_alloc(tmem_slot, Cfg::TMEM_COLS);
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
            // ---------------- TMA producer
            int stage = 0;
            uint32_t phase = 0;
            long issued = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < num_tiles && ok; t += gridDim.x) {
                int tm, tn;
                tile_coords(t, args.tiles_m, args.tiles_n, args.group_m, tm, tn);
                for (int kb = 0; kb < num_kb; ++kb) {
                    if (!mbar_wait(&empty[stage], phase ^ 1u, ctl, limit, status)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[stage], Cfg::STAGE_BYTES);
                    tma_load_2d(sA + stage * Cfg::A_BYTES, &tmA, &full[stage], kb * Cfg::BK,
                                tm * Cfg::BLOCK_M);
                    if constexpr (BKM) {
                        tma_load_2d(sB + stage * Cfg::B_BYTES, &tmB, &full[stage], kb * Cfg::BK,
                                    tn * BLOCK_N);
                    } else {
#pragma unroll
                        for (int c = 0; c < BLOCK_N / Cfg::CHUNK_N; ++c)
                            tma_load_2d(sB + stage * Cfg::B_BYTES + c * Cfg::CHUNK_BYTES, &tmB,
                                        &full[stage], tn * BLOCK_N + c * Cfg::CHUNK_N, kb * Cfg::BK);
                    }
                    ++issued;
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) {
                // Let the loads already in flight land before the CTA exits.
                CtaCtl local{0};
                const long outstanding = issued < STAGES ? issued : STAGES;
                for (long q = 1; q <= outstanding; ++q) {
                    const long idx = issued - q;
                    mbar_wait(&full[idx % STAGES], static_cast<uint32_t>((idx / STAGES) & 1), &local,
                              limit, status);
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer
            int stage = 0;
            uint32_t phase = 0;
            int local_t = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < num_tiles && ok; t += gridDim.x, ++local_t) {
                const int acc = Cfg::NBUF == 2 ? (local_t & 1) : 0;
                const uint32_t acc_phase =
                    static_cast<uint32_t>(Cfg::NBUF == 2 ? (local_t >> 1) : local_t) & 1u;
                if (!mbar_wait(&tempty[acc], acc_phase ^ 1u, ctl, limit, status)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem_base + static_cast<uint32_t>(acc * BLOCK_N);
                for (int kb = 0; kb < num_kb; ++kb) {
                    if (!mbar_wait(&full[stage], phase, ctl, limit, status)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t adesc =
                        smem_desc_sw128(smem_u32(sA + stage * Cfg::A_BYTES), 16, 1024);
                    const uint64_t bdesc = smem_desc_sw128(smem_u32(sB + stage * Cfg::B_BYTES),
                                                           BKM ? 16 : Cfg::CHUNK_BYTES, 1024);
#pragma unroll
                    for (int k = 0; k < Cfg::BK / Cfg::MMA_K; ++k) {
                        const uint64_t a_off = static_cast<uint64_t>((k * 32) >> 4);
                        const uint64_t b_off = BKM ? a_off
                                                   : static_cast<uint64_t>((k * Cfg::MMA_K * 128) >> 4);
#pragma unroll
                        for (int h = 0; h < MT; ++h) {
                            // half h: A rows 128h.. (16 KB further in the stage),
                            // accumulator columns h * BLOCK_N
                            const uint32_t dh = d + static_cast<uint32_t>(h * BLOCK_N);
                            const uint64_t ah = adesc + a_off + static_cast<uint64_t>((h * 128 * 128) >> 4);
                            if constexpr (ESIZE == 2)
                                mma_f16(dh, ah, bdesc + b_off, Cfg::IDESC, (kb | k) != 0);
                            else
                                mma_tf32(dh, ah, bdesc + b_off, Cfg::IDESC, (kb | k) != 0);
                        }
                    }
                    mma_commit(&empty[stage]);
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) break;
                mma_commit(&tfull[acc]);
            }
            // Every MMA issued above must finish before TMEM is released.
            mma_commit(drain);
            CtaCtl local{0};
            mbar_wait(drain, 0, &local, limit, status);
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: TMEM lane quadrant q = warp % 4; with MT = 2
        // warps 2..5 drain the upper half (rows 0..127), warps 6..9 the lower
        const int q = warp & 3;
        const int h = (warp - 2) >> 2;
        int local_t = 0;
        for (int t = blockIdx.x; t < num_tiles; t += gridDim.x, ++local_t) {
            const int acc = Cfg::NBUF == 2 ? (local_t & 1) : 0;
            const uint32_t acc_phase =
                static_cast<uint32_t>(Cfg::NBUF == 2 ? (local_t >> 1) : local_t) & 1u;
            bool ok = mbar_wait(&tfull[acc], acc_phase, ctl, limit, status);
            if (!__all_sync(0xffffffffu, ok)) break;
            tc_fence_after();
            int tm, tn;
            tile_coords(t, args.tiles_m, args.tiles_n, args.group_m, tm, tn);
            const int64_t row0 = static_cast<int64_t>(tm) * Cfg::BLOCK_M + h * 128 + q * 32;
            const int64_t rl = args.m - row0;
            const int rows_left = rl <= 0 ? 0 : (rl >= 32 ? 32 : static_cast<int>(rl));
            uint8_t* stage_w = out_stage + (warp - 2) * 4096;
#pragma unroll 1
            for (int c = 0; c < BLOCK_N / 32; ++c) {
                uint32_t r[32];
                tmem_ld32(tmem_base + (static_cast<uint32_t>(q * 32) << 16) +
                              static_cast<uint32_t>((acc + h) * BLOCK_N + c * 32),
                          r);
                tmem_ld_wait();
                const int64_t col0 = static_cast<int64_t>(tn) * BLOCK_N + c * 32;
                if (rows_left > 0 && col0 < args.p)
                    store_block32(stage_w, r, args.C, args.p, row0, rows_left, col0,
                                  args.p - col0, args.vec_ok != 0);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[acc]);
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, Cfg::TMEM_COLS);
    }
}

// ---------------------------------------------------------------- CTA pairs
// 256 x 256 output tiles, each computed by a cluster of two CTAs with
// cta_group::2 MMAs (M = 256, N = 256): CTA r holds rows 128 r .. 128 r + 127
// of the tile's A rows and columns 128 r .. 128 r + 127 of its B (32 KB a K
// block, six stages), and accumulates its 128 x 256 half of the tile in TMEM,
// double-buffered (all 512 columns) so that the next tile's MMAs overlap the
// stores -- which the one-CTA 256 x 256 tiles, whose single accumulator fills
// TMEM, cannot.  Both CTAs' loads complete on the even CTA's `full` barrier;
// the even CTA issues the MMAs and its commits release both CTAs' stages and
// hand both accumulators to the epilogues; both epilogues report the drain to
// the even CTA.  Every wait is bounded; a cluster barrier precedes the TMEM
// release and the exit.
template <int ESIZE, int BKM>
struct DensePairCfg {
    static constexpr int BK = 128 / ESIZE;            // K elements per stage (128 bytes)
    static constexpr int MMA_K = 32 / ESIZE;          // K per tcgen05.mma (32 bytes)
    static constexpr int CHUNK_N = 128 / ESIZE;       // B columns per 128-byte swizzle row
    static constexpr int CHUNK_BYTES = BK * 128;      // one MN-major B column chunk
    static constexpr int A_BYTES = 128 * 128;         // this CTA's 128 rows x 128 B
    static constexpr int B_BYTES = 128 * BK * ESIZE;  // this CTA's 128 columns of B
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int STAGES = 6;
    static constexpr int EPI_WARPS = 4;               // one per TMEM lane quadrant
    static constexpr int THREADS = 64 + 32 * EPI_WARPS;
    static constexpr int OUT_STAGE = EPI_WARPS * 4096;
    static constexpr int SMEM = 1024 + STAGES * STAGE_BYTES + OUT_STAGE + 256;
    static_assert(SMEM <= 227 * 1024, "dense pair kernel shared memory");
    static constexpr int TMEM_COLS = 512;             // two 256-column accumulators
    static constexpr uint32_t IDESC = make_idesc(ESIZE == 2 ? 1u : 2u, 256, 256, 0u, BKM ? 0u : 1u);
};

template <int ESIZE, int BKM>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(DensePairCfg<ESIZE, BKM>::THREADS, 1)
    dense_pair_kernel(const __grid_constant__ CUtensorMap tmA,
                      const __grid_constant__ CUtensorMap tmB, const DenseArgs args) {
    using Cfg = DensePairCfg<ESIZE, BKM>;
    constexpr int STAGES = Cfg::STAGES;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                               ~static_cast<uintptr_t>(1023));
    uint8_t* sA = smem;
    uint8_t* sB = smem + STAGES * Cfg::A_BYTES;
    uint8_t* out_stage = sB + STAGES * Cfg::B_BYTES;
    uint64_t* bars = reinterpret_cast<uint64_t*>(out_stage + Cfg::OUT_STAGE);
    uint64_t* full = bars;                  // (even CTA) both CTAs' stage has landed
    uint64_t* empty = bars + STAGES;        // the pair's MMAs are done with the stage
    uint64_t* tfull = bars + 2 * STAGES;    // an accumulator holds a finished tile
    uint64_t* tempty = tfull + 2;           // (even CTA) both epilogues drained it
    uint64_t* drain = tempty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    CtaCtl* ctl = reinterpret_cast<CtaCtl*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint32_t rank = cluster_ctarank();
    const uint64_t limit = args.wait_limit_ns;
    int* status = args.status;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], 2 * Cfg::EPI_WARPS);
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
        tmem_alloc_pair(tmem_slot, Cfg::TMEM_COLS);
        tmem_relinquish_pair();
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();   // both CTAs' barriers exist before any arrival crosses over
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const int cid = static_cast<int>(blockIdx.x) >> 1;
    const int ncl = static_cast<int>(gridDim.x) >> 1;
    const int num_tiles = args.tiles_m * args.tiles_n;
    const int num_kb = args.num_kb;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer: this CTA's rows of A, columns of B
            const uint32_t full0 = mapa_shared(smem_u32(full), 0);
            int stage = 0;
            uint32_t phase = 0;
            long issued = 0;
            bool ok = true;
            for (int t = cid; t < num_tiles && ok; t += ncl) {
                int tm, tn;
                tile_coords(t, args.tiles_m, args.tiles_n, args.group_m, tm, tn);
                const int row0 = tm * 256 + static_cast<int>(rank) * 128;
                const int col0 = tn * 256 + static_cast<int>(rank) * 128;
                for (int kb = 0; kb < num_kb; ++kb) {
                    if (!mbar_wait(&empty[stage], phase ^ 1u, ctl, limit, status)) {
                        ok = false;
                        break;
                    }
                    if (rank == 0) mbar_arrive_expect_tx(&full[stage], 2 * Cfg::STAGE_BYTES);
                    const uint32_t fb = full0 + 8u * static_cast<uint32_t>(stage);
                    tma_load_2d_pair(sA + stage * Cfg::A_BYTES, &tmA, fb, kb * Cfg::BK, row0);
                    if constexpr (BKM) {
                        tma_load_2d_pair(sB + stage * Cfg::B_BYTES, &tmB, fb, kb * Cfg::BK, col0);
                    } else {
#pragma unroll
                        for (int c = 0; c < 128 / Cfg::CHUNK_N; ++c)
                            tma_load_2d_pair(sB + stage * Cfg::B_BYTES + c * Cfg::CHUNK_BYTES, &tmB,
                                             fb, col0 + c * Cfg::CHUNK_N, kb * Cfg::BK);
                    }
                    ++issued;
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) {
                // Let the loads already in flight land before the CTA exits:
                // the even CTA waits on its full barriers (which count both
                // CTAs' loads); the odd CTA gives its own at most STAGES loads
                // a millisecond.
                CtaCtl local{0};
                if (rank == 0) {
                    const long outstanding = issued < STAGES ? issued : STAGES;
                    for (long q = 1; q <= outstanding; ++q) {
                        const long idx = issued - q;
                        mbar_wait(&full[idx % STAGES], static_cast<uint32_t>((idx / STAGES) & 1),
                                  &local, limit, status);
                    }
                } else {
                    const uint64_t t0 = global_timer_ns();
                    while (global_timer_ns() - t0 < 1000000ull) {
                    }
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0 && rank == 0) {
            // ---------------- even CTA: MMA issuer for the pair
            int stage = 0;
            uint32_t phase = 0;
            int local_t = 0;
            bool ok = true;
            for (int t = cid; t < num_tiles && ok; t += ncl, ++local_t) {
                const int acc = local_t & 1;
                const uint32_t acc_phase = static_cast<uint32_t>(local_t >> 1) & 1u;
                if (!mbar_wait(&tempty[acc], acc_phase ^ 1u, ctl, limit, status)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem_base + static_cast<uint32_t>(acc * 256);
                for (int kb = 0; kb < num_kb; ++kb) {
                    if (!mbar_wait(&full[stage], phase, ctl, limit, status)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t adesc =
                        smem_desc_sw128(smem_u32(sA + stage * Cfg::A_BYTES), 16, 1024);
                    const uint64_t bdesc = smem_desc_sw128(smem_u32(sB + stage * Cfg::B_BYTES),
                                                           BKM ? 16 : Cfg::CHUNK_BYTES, 1024);
#pragma unroll
                    for (int k = 0; k < Cfg::BK / Cfg::MMA_K; ++k) {
                        const uint64_t a_off = static_cast<uint64_t>((k * 32) >> 4);
                        const uint64_t b_off = BKM ? a_off
                                                   : static_cast<uint64_t>((k * Cfg::MMA_K * 128) >> 4);
                        if constexpr (ESIZE == 2)
                            mma_f16_pair(d, adesc + a_off, bdesc + b_off, Cfg::IDESC, (kb | k) != 0);
                        else
                            mma_tf32_pair(d, adesc + a_off, bdesc + b_off, Cfg::IDESC, (kb | k) != 0);
                    }
                    mma_commit_pair_mc(&empty[stage], 0x3);
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) break;
                mma_commit_pair_mc(&tfull[acc], 0x3);
            }
            // Every MMA issued above must finish before either CTA releases
            // TMEM or exits.
            mma_commit_pair(drain);
            CtaCtl local{0};
            mbar_wait(drain, 0, &local, limit, status);
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: TMEM lane quadrant q = warp % 4, all 256 columns
        const int q = warp & 3;
        const uint32_t tempty0 = rank == 0 ? 0u : mapa_shared(smem_u32(tempty), 0);
        uint8_t* stage_w = out_stage + (warp - 2) * 4096;
        int local_t = 0;
        for (int t = cid; t < num_tiles; t += ncl, ++local_t) {
            const int acc = local_t & 1;
            const uint32_t acc_phase = static_cast<uint32_t>(local_t >> 1) & 1u;
            bool ok = mbar_wait(&tfull[acc], acc_phase, ctl, limit, status);
            if (!__all_sync(0xffffffffu, ok)) break;
            tc_fence_after();
            int tm, tn;
            tile_coords(t, args.tiles_m, args.tiles_n, args.group_m, tm, tn);
            const int64_t row0 = static_cast<int64_t>(tm) * 256 + rank * 128 + q * 32;
            const int64_t rl = args.m - row0;
            const int rows_left = rl <= 0 ? 0 : (rl >= 32 ? 32 : static_cast<int>(rl));
#pragma unroll 1
            for (int c = 0; c < 256 / 32; ++c) {
                uint32_t r[32];
                tmem_ld32(tmem_base + (static_cast<uint32_t>(q * 32) << 16) +
                              static_cast<uint32_t>(acc * 256 + c * 32),
                          r);
                tmem_ld_wait();
                const int64_t col0 = static_cast<int64_t>(tn) * 256 + c * 32;
                if (rows_left > 0 && col0 < args.p)
                    store_block32(stage_w, r, args.C, args.p, row0, rows_left, col0,
                                  args.p - col0, args.vec_ok != 0);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                if (rank == 0)
                    mbar_arrive(&tempty[acc]);
                else
                    mbar_arrive_remote(tempty0 + 8u * static_cast<uint32_t>(acc));
            }
        }
    }
    __syncthreads();
    cluster_sync_all();   // the pair's MMAs and cross-CTA arrivals are over
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc_pair(tmem_base, Cfg::TMEM_COLS);
    }
}

template <int ESIZE, int BLOCK_N, int STAGES, int BKM, int MT>
int launch_cfg(int64_t m, int64_t n, int64_t p, const void* A, int64_t lda, const void* B,
               int64_t ldb, float* C, cudaStream_t s, moa_stats* st) {
    using Cfg = DenseCfg<ESIZE, BLOCK_N, STAGES, BKM, MT>;
    const CUtensorMapDataType dt =
        ESIZE == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    CUtensorMap tmA, tmB;
    int rc = make_tmap_2d(&tmA, dt, A, static_cast<uint64_t>(n), static_cast<uint64_t>(m),
                          static_cast<uint64_t>(lda) * ESIZE, Cfg::BK, Cfg::BLOCK_M);
    if (rc != MOA_OK) return rc;
    if (BKM)   // B^T: p rows of n (pitch ldb), box = BLOCK_N rows x 128 bytes
        rc = make_tmap_2d(&tmB, dt, B, static_cast<uint64_t>(n), static_cast<uint64_t>(p),
                          static_cast<uint64_t>(ldb) * ESIZE, Cfg::BK, BLOCK_N);
    else
        rc = make_tmap_2d(&tmB, dt, B, static_cast<uint64_t>(p), static_cast<uint64_t>(n),
                          static_cast<uint64_t>(ldb) * ESIZE, Cfg::CHUNK_N, Cfg::BK);
    if (rc != MOA_OK) return rc;

    DenseArgs args;
    args.C = C;
    args.m = m;
    args.n = n;
    args.p = p;
    args.tiles_m = static_cast<int>(ceil_div(m, Cfg::BLOCK_M));
    args.tiles_n = static_cast<int>(ceil_div(p, BLOCK_N));
    args.num_kb = static_cast<int>(ceil_div(n, Cfg::BK));
    args.group_m = raster_group();
    args.vec_ok = (p % 4 == 0) && (reinterpret_cast<uintptr_t>(C) % 16 == 0);
    args.wait_limit_ns = wait_limit_ns();
    args.status = launch_status_ptr();
    if (!args.status) return MOA_ERR_CUDA;

    auto kern = dense_tc_kernel<ESIZE, BLOCK_N, STAGES, BKM, MT>;
    static std::atomic<uint64_t> attr_done{0};   // per instantiation, per device
    {
        const int rc = smem_attr_once(reinterpret_cast<const void*>(kern), Cfg::SMEM, attr_done,
                                      "cudaFuncSetAttribute(dense_tc)");
        if (rc != MOA_OK) return rc;
    }
    const long tiles = static_cast<long>(args.tiles_m) * args.tiles_n;
    const int grid = static_cast<int>(std::min<long>(tiles, num_sms()));
    prof_begin(s);
    kern<<<grid, Cfg::THREADS, Cfg::SMEM, s>>>(tmA, tmB, args);
    cudaError_t e = cudaGetLastError();
    prof_end(s);
    if (e != cudaSuccess) return cuda_fail(e, "dense_tc_kernel launch");
    log_msg(2, "dense %s m=%lld n=%lld p=%lld tile %dx%d stages %d grid %d tiles %ld",
            ESIZE == 2 ? "bf16" : "tf32", static_cast<long long>(m), static_cast<long long>(n),
            static_cast<long long>(p), Cfg::BLOCK_M, BLOCK_N, STAGES, grid, tiles);
    if (st) {
        st->block_m = Cfg::BLOCK_M;
        st->block_n = BLOCK_N;
        st->block_k = Cfg::BK;
        st->grid = grid;
        st->tiles = tiles;
        st->kernels += 1;
    }
    return MOA_OK;
}

// 256 x 256 tiles for the 256-wide case: on unless MOA_DENSE_TALL=0.
bool dense_tall_tiles() {
    static int on = -1;
    if (on < 0) {
        const char* env = std::getenv("MOA_DENSE_TALL");
        on = (env && env[0] == '0') ? 0 : 1;
    }
    return on == 1;
}

}  // namespace

// Clusters of dense_pair_kernel<ESIZE, BKM> that fit on the device at once
// (cached per device; 0 when the query fails: no pair tiles).
template <int ESIZE, int BKM>
long dense_pair_clusters() {
    using Cfg = DensePairCfg<ESIZE, BKM>;
    static std::atomic<long> cache[64];
    int d = -1;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= 64) return 0;
    const long have = cache[d].load(std::memory_order_acquire);
    if (have != 0) return have;
    static std::atomic<uint64_t> attr_done{0};
    if (smem_attr_once(reinterpret_cast<const void*>(dense_pair_kernel<ESIZE, BKM>), Cfg::SMEM,
                       attr_done, "cudaFuncSetAttribute(dense_pair)") != MOA_OK)
        return 0;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(2 * static_cast<unsigned>(num_sms()), 1, 1);
    cfg.blockDim = dim3(Cfg::THREADS, 1, 1);
    cfg.dynamicSmemBytes = Cfg::SMEM;
    int nc = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&nc, dense_pair_kernel<ESIZE, BKM>, &cfg);
    if (e != cudaSuccess || nc < 1) {
        cudaGetLastError();
        log_msg(1, "dense pair kernel: cluster occupancy query failed; one-SM tiles only");
        return 0;
    }
    cache[d].store(nc, std::memory_order_release);
    return nc;
}

template <int ESIZE, int BKM>
int launch_pair(int64_t m, int64_t n, int64_t p, const void* A, int64_t lda, const void* B,
                int64_t ldb, float* C, long clusters, cudaStream_t s, moa_stats* st) {
    using Cfg = DensePairCfg<ESIZE, BKM>;
    const CUtensorMapDataType dt =
        ESIZE == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    CUtensorMap tmA, tmB;
    int rc = make_tmap_2d(&tmA, dt, A, static_cast<uint64_t>(n), static_cast<uint64_t>(m),
                          static_cast<uint64_t>(lda) * ESIZE, Cfg::BK, 128);
    if (rc != MOA_OK) return rc;
    if (BKM)   // B^T: p rows of n (pitch ldb), box = this CTA's 128 rows x 128 bytes
        rc = make_tmap_2d(&tmB, dt, B, static_cast<uint64_t>(n), static_cast<uint64_t>(p),
                          static_cast<uint64_t>(ldb) * ESIZE, Cfg::BK, 128);
    else
        rc = make_tmap_2d(&tmB, dt, B, static_cast<uint64_t>(p), static_cast<uint64_t>(n),
                          static_cast<uint64_t>(ldb) * ESIZE, Cfg::CHUNK_N, Cfg::BK);
    if (rc != MOA_OK) return rc;
    DenseArgs args;
    args.C = C;
    args.m = m;
    args.n = n;
    args.p = p;
    args.tiles_m = static_cast<int>(ceil_div(m, 256));
    args.tiles_n = static_cast<int>(ceil_div(p, 256));
    args.num_kb = static_cast<int>(ceil_div(n, Cfg::BK));
    args.group_m = std::max(1, raster_group() / 2);   // the same rows a raster group
    args.vec_ok = (p % 4 == 0) && (reinterpret_cast<uintptr_t>(C) % 16 == 0);
    args.wait_limit_ns = wait_limit_ns();
    args.status = launch_status_ptr();
    if (!args.status) return MOA_ERR_CUDA;
    const long tiles = static_cast<long>(args.tiles_m) * args.tiles_n;
    const int grid = 2 * static_cast<int>(std::min<long>(tiles, clusters));
    prof_begin(s);
    dense_pair_kernel<ESIZE, BKM><<<grid, Cfg::THREADS, Cfg::SMEM, s>>>(tmA, tmB, args);
    cudaError_t e = cudaGetLastError();
    prof_end(s);
    if (e != cudaSuccess) return cuda_fail(e, "dense_pair_kernel launch");
    log_msg(2, "dense %s m=%lld n=%lld p=%lld tile 256x256 (CTA pairs) grid %d tiles %ld",
            ESIZE == 2 ? "bf16" : "tf32", static_cast<long long>(m), static_cast<long long>(n),
            static_cast<long long>(p), grid, tiles);
    if (st) {
        st->block_m = 256;
        st->block_n = 256;
        st->block_k = Cfg::BK;
        st->grid = grid;
        st->tiles = tiles;
        st->kernels += 1;
    }
    return MOA_OK;
}

int dense_tc_launch(bool in_bf16, int64_t m, int64_t n, int64_t p, const void* A, int64_t lda,
                    const void* B, int64_t ldb, float* C, cudaStream_t s, moa_stats* st) {
    // moa_set_block_m(256): 256 x 256 tiles on CTA pairs
    if (tile_m_override() == 256) {
        const long cl = in_bf16 ? dense_pair_clusters<2, 0>() : dense_pair_clusters<4, 1>();
        if (cl > 0)
            return in_bf16 ? launch_pair<2, 0>(m, n, p, A, lda, B, ldb, C, cl, s, st)
                           : launch_pair<4, 1>(m, n, p, A, lda, B, ldb, C, cl, s, st);
    }
    // Tile planner (the block-size model of Sec. 3.4 on this machine): the
    // candidate tiles are 256 x 256, 128 x 256, 128 x 128 and 128 x 64; each
    // costs ceil(tiles / SMs) waves of (tile area / its relative MMA
    // efficiency), the efficiencies measured on the B300 (1.0, 0.9, 0.7, 0.39:
    // narrower tiles re-read their operands more often per flop).  The
    // cheapest wins, the larger tile on a tie.  A per-thread override
    // (moa_set_block_n) or a measured choice for this shape bucket
    // (moa_tune_dense) fixes the width; the 256 x 256 / 128 x 256 choice for
    // width 256 stays with the model (MOA_DENSE_TALL=0 rules out 256 x 256).
    const int sms = num_sms();
    auto cost = [&](int bm, int bn_, double eff) {
        const long tiles = ceil_div(m, bm) * ceil_div(p, bn_);
        return static_cast<double>((tiles + sms - 1) / sms) * (bm * bn_) / eff;
    };
    // moa_set_block_m(128): 128-row tiles only
    const double c_tall =
        (dense_tall_tiles() && tile_m_override() != 128) ? cost(256, 256, 1.0) : 1e300;
    const double c256 = cost(128, 256, 0.9), c128 = cost(128, 128, 0.7), c64 = cost(128, 64, 0.39);
    int bn = 256;
    double best = std::min(c_tall, c256);
    if (c128 < best) {
        bn = 128;
        best = c128;
    }
    if (c64 < best) bn = 64;
    const int tuned = tuned_block_n(in_bf16 ? MOA_BF16 : MOA_F32_TF32, m, n, p);
    if (tuned) bn = tuned;
    if (tile_override() == 64 || tile_override() == 128 || tile_override() == 256)
        bn = tile_override();
    const bool tall = bn == 256 && c_tall <= c256;
    if (in_bf16) {
        if (bn == 256)
            return tall ? launch_cfg<2, 256, 3, 0, 2>(m, n, p, A, lda, B, ldb, C, s, st)
                        : launch_cfg<2, 256, 4, 0, 1>(m, n, p, A, lda, B, ldb, C, s, st);
        if (bn == 128) return launch_cfg<2, 128, 6, 0, 1>(m, n, p, A, lda, B, ldb, C, s, st);
        return launch_cfg<2, 64, 8, 0, 1>(m, n, p, A, lda, B, ldb, C, s, st);
    }
    // TF32: B is passed transposed (p x n, row pitch ldb), K-major.
    if (bn == 256)
        return tall ? launch_cfg<4, 256, 3, 1, 2>(m, n, p, A, lda, B, ldb, C, s, st)
                    : launch_cfg<4, 256, 4, 1, 1>(m, n, p, A, lda, B, ldb, C, s, st);
    if (bn == 128) return launch_cfg<4, 128, 6, 1, 1>(m, n, p, A, lda, B, ldb, C, s, st);
    return launch_cfg<4, 64, 8, 1, 1>(m, n, p, A, lda, B, ldb, C, s, st);
}

}  // namespace moa
