// grouped.cu -- moa_gemm_grouped: `count` independent ONF GEMMs of arbitrary
// shapes (Eq. (eq:dnf) per problem) in ONE persistent tcgen05 launch.
//
// Batching pattern: every problem g gets its own tile width BN_g in {64, 128,
// 256} from a shape-driven cost model (the paper's block sizes chosen from
// "the static information of types and shapes", Sec. 3.4).  Its output tiles
// (128 x BN_g) enter one work list; the host deals the list to the persistent
// CTAs longest-processing-time first (each tile to the least-loaded CTA), so
// heavy-tailed size mixes stay balanced.  Per-problem TMA descriptors live in
// the workspace (global memory); the MMA N extent is a runtime field of the
// instruction descriptor, so one kernel binary serves every tile width.
//
// The persistent path takes BF16 problems whose rows are 16-byte multiples
// (n % 8 == 0, p % 8 == 0) and 16-byte aligned A and B.  Other problems of the
// call (other dtypes, unaligned pitches) are issued one by one through the
// single-GEMM path on the same stream, with the workspace tail as scratch.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <functional>
#include <queue>
#include <vector>

#include "crt.h"
#include "split.h"
#include "epilogue.cuh"
#include "internal.h"
#include "ptx.cuh"

namespace moa {
int gemm_ex(int64_t m, int64_t n, int64_t p, moa_dtype dt, const void* A, const void* B, void* C,
            int slices, void* ws, size_t ws_bytes, cudaStream_t s, moa_stats* st);
size_t workspace_bytes(int64_t m, int64_t n, int64_t p, moa_dtype dt, int slices);

namespace {

constexpr int kGBM = 128, kGBK = 64, kGStages = 4;
constexpr int kGABytes = kGBM * 128;                    // 128 rows x 64 BF16
constexpr int kGBChunk = kGBK * 128;                    // 64 rows x 64 BF16 columns
constexpr int kGStageBytes = kGABytes + 4 * kGBChunk;   // room for BN = 256
// Epilogue: two warps per TMEM lane quadrant (alternate 32-column blocks),
// each with a 4 KB staging tile for coalesced stores.
constexpr int kGEpiWarps = 8;
constexpr int kGThreads = 64 + 32 * kGEpiWarps;
constexpr int kGStageOut = kGEpiWarps * 4096;
constexpr int kGSmem = 1024 + kGStages * kGStageBytes + kGStageOut + 256;

struct GroupDev {
    float* C;
    int m, n, p;
    int bn;        // tile width: 64, 128 or 256
    int tiles_n;
    int num_kb;
    int vec_ok;
    int pad;
};

struct GroupedArgs {
    const CUtensorMap* maps;   // 2 per problem: A, B (64-byte aligned, global memory)
    const GroupDev* groups;
    const int4* tiles;         // (group, tm, tn, 0) per tile, grouped by CTA
    const int* cta_begin;      // grid + 1 offsets into tiles
    uint64_t wait_limit_ns;
    int* status;
};

// A role's walk over its CTA's work list.  The tile record of tile t + 2 and
// the problem record of tile t + 1 are requested while tile t is processed,
// so the dependent global-memory lookups (tile -> problem) never stall the
// role between tiles.
struct TileWalk {
    int4 tl;        // current tile (problem, tm, tn, 0)
    GroupDev g;     // its problem
    int4 tl_next;   // the next tile
    __device__ void start(const GroupedArgs& a, int t0, int t1) {
        if (t0 < t1) {
            tl = a.tiles[t0];
            g = a.groups[tl.x];
        }
        tl_next = (t0 + 1 < t1) ? a.tiles[t0 + 1] : tl;
    }
};

__global__ void __launch_bounds__(kGThreads, 1) grouped_tc_kernel(const GroupedArgs args) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                               ~static_cast<uintptr_t>(1023));
    uint8_t* out_stage = smem + kGStages * kGStageBytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(out_stage + kGStageOut);
    uint64_t* full = bars;
    uint64_t* empty = bars + kGStages;
    uint64_t* tfull = bars + 2 * kGStages;
    uint64_t* tempty = tfull + 2;
    uint64_t* drain = tempty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    CtaCtl* ctl = reinterpret_cast<CtaCtl*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint64_t limit = args.wait_limit_ns;
    int* status = args.status;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kGStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], kGEpiWarps);
        }
        mbar_init(drain, 1);
        ctl->abort = 0;
        fence_barrier_init();
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const int t0 = args.cta_begin[blockIdx.x];
    const int t1 = args.cta_begin[blockIdx.x + 1];

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer
            int stage = 0;
            uint32_t phase = 0;
            long issued = 0;
            bool ok = true;
            TileWalk w;
            w.start(args, t0, t1);
            for (int t = t0; t < t1 && ok; ++t) {
                const int4 tl_nn = (t + 2 < t1) ? args.tiles[t + 2] : w.tl_next;
                const GroupDev g_n = (t + 1 < t1) ? args.groups[w.tl_next.x] : w.g;
                if (t + 1 < t1) {   // the next problem's TMA descriptors
                    prefetch_tmap(args.maps + 2 * w.tl_next.x);
                    prefetch_tmap(args.maps + 2 * w.tl_next.x + 1);
                }
                const int4 tl = w.tl;
                const GroupDev g = w.g;
                const CUtensorMap* mA = args.maps + 2 * tl.x;
                const CUtensorMap* mB = mA + 1;
                const uint32_t bytes = kGABytes + static_cast<uint32_t>(g.bn) * kGBK * 2;
                for (int kb = 0; kb < g.num_kb; ++kb) {
                    if (!mbar_wait(&empty[stage], phase ^ 1u, ctl, limit, status)) {
                        ok = false;
                        break;
                    }
                    uint8_t* sa = smem + stage * kGStageBytes;
                    mbar_arrive_expect_tx(&full[stage], bytes);
                    tma_load_2d(sa, mA, &full[stage], kb * kGBK, tl.y * kGBM);
                    for (int c = 0; c < g.bn / 64; ++c)
                        tma_load_2d(sa + kGABytes + c * kGBChunk, mB, &full[stage],
                                    tl.z * g.bn + c * 64, kb * kGBK);
                    ++issued;
                    if (++stage == kGStages) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                w.tl = w.tl_next;
                w.g = g_n;
                w.tl_next = tl_nn;
            }
            if (!ok) {
                // Let the loads already in flight land before the CTA exits.
                CtaCtl local{0};
                const long outstanding = issued < kGStages ? issued : kGStages;
                for (long q = 1; q <= outstanding; ++q) {
                    const long idx = issued - q;
                    mbar_wait(&full[idx % kGStages], static_cast<uint32_t>((idx / kGStages) & 1),
                              &local, limit, status);
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer, runtime N per tile
            int stage = 0;
            uint32_t phase = 0;
            int local_t = 0;
            bool ok = true;
            TileWalk w;
            w.start(args, t0, t1);
            for (int t = t0; t < t1 && ok; ++t, ++local_t) {
                const int4 tl_nn = (t + 2 < t1) ? args.tiles[t + 2] : w.tl_next;
                const GroupDev g_n = (t + 1 < t1) ? args.groups[w.tl_next.x] : w.g;
                const int bn = w.g.bn;
                const int num_kb = w.g.num_kb;
                w.tl = w.tl_next;
                w.g = g_n;
                w.tl_next = tl_nn;
                const uint32_t idesc = make_idesc(1u, kGBM, static_cast<uint32_t>(bn), 0u, 1u);
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
                    uint8_t* sa = smem + stage * kGStageBytes;
                    const uint64_t adesc = smem_desc_sw128(smem_u32(sa), 16, 1024);
                    const uint64_t bdesc = smem_desc_sw128(smem_u32(sa + kGABytes), kGBChunk, 1024);
#pragma unroll
                    for (int k = 0; k < kGBK / 16; ++k)
                        mma_f16(d, adesc + static_cast<uint64_t>((k * 32) >> 4),
                                bdesc + static_cast<uint64_t>((k * 16 * 128) >> 4), idesc,
                                (kb | k) != 0);
                    mma_commit(&empty[stage]);
                    if (++stage == kGStages) {
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
        // ---------------- epilogue: warps 2..9; TMEM lane quadrant q = warp % 4,
        // column blocks h, h + 2, ... of 32 (h = 0 for warps 2..5, 1 for 6..9)
        const int q = warp & 3;
        const int h = (warp - 2) >> 2;
        uint8_t* stage_w = out_stage + (warp - 2) * 4096;
        int local_t = 0;
        TileWalk w;
        w.start(args, t0, t1);
        for (int t = t0; t < t1; ++t, ++local_t) {
            const int4 tl_nn = (t + 2 < t1) ? args.tiles[t + 2] : w.tl_next;
            const GroupDev g_n = (t + 1 < t1) ? args.groups[w.tl_next.x] : w.g;
            const int4 tl = w.tl;
            const GroupDev g = w.g;
            w.tl = w.tl_next;
            w.g = g_n;
            w.tl_next = tl_nn;
            const int acc = local_t & 1;
            const uint32_t acc_phase = static_cast<uint32_t>(local_t >> 1) & 1u;
            bool ok = mbar_wait(&tfull[acc], acc_phase, ctl, limit, status);
            if (!__all_sync(0xffffffffu, ok)) break;
            tc_fence_after();
            const int64_t row0 = static_cast<int64_t>(tl.y) * kGBM + q * 32;
            const int64_t rl = g.m - row0;
            const int rows_left = rl <= 0 ? 0 : (rl >= 32 ? 32 : static_cast<int>(rl));
            for (int c = h; c < g.bn / 32; c += 2) {
                uint32_t r[32];
                tmem_ld32(tmem_base + (static_cast<uint32_t>(q * 32) << 16) +
                              static_cast<uint32_t>(acc * 256 + c * 32),
                          r);
                tmem_ld_wait();
                const int64_t col0 = static_cast<int64_t>(tl.z) * g.bn + c * 32;
                if (rows_left > 0 && col0 < g.p)
                    store_block32(stage_w, r, g.C, g.p, row0, rows_left, col0, g.p - col0,
                                  g.vec_ok != 0);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[acc]);
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, 512);
    }
}

// ------------------------------------------------------------------ planning
// Cost of one output tile in units of "one K block of a 128 x 256 tile at full
// tensor rate" (512 SM cycles): the larger of its MMA work (bn/256 per K block,
// divided by the width's MMA efficiency: narrow tiles re-read A from shared
// memory for fewer columns and are shared-memory bound) and its memory time
// (A strip + B strip + C tile bytes at one SM's share of HBM bandwidth,
// about 12 KB per unit), plus a fixed share per tile for the TMEM drain, the
// stores and the pipeline fill.  Small-K tiles of a mixed batch are memory
// bound; costing them by MMA work alone let the dealing overload some SMs.
constexpr double kTileOverheadKb = 3.0;

double mma_eff(int bn) { return bn >= 256 ? 1.0 : (bn >= 128 ? 0.9 : 0.67); }

double tile_cost(int64_t n, int bn) {
    const double compute = static_cast<double>(ceil_div(n, kGBK)) * (bn / 256.0) / mma_eff(bn);
    const double bytes = 2.0 * kGBM * n + 2.0 * n * bn + 4.0 * kGBM * bn;
    const double memory = bytes / (12.0 * 1024.0);
    return (compute > memory ? compute : memory) + kTileOverheadKb;
}

bool persistent_ok(const moa_gemm_desc& d) {
    return d.dt == MOA_BF16 && d.m > 0 && d.p > 0 && d.n > 0 && d.n % 8 == 0 && d.p % 8 == 0 &&
           reinterpret_cast<uintptr_t>(d.A) % 16 == 0 && reinterpret_cast<uintptr_t>(d.B) % 16 == 0 &&
           reinterpret_cast<uintptr_t>(d.C) % 4 == 0 && d.m < (int64_t(1) << 31) &&
           d.n < (int64_t(1) << 31) && d.p < (int64_t(1) << 31);
}

// Tile width of one problem (the block size chosen from the static shapes,
// Sec. 3.4): the width recorded by the measured autotuner for the problem's
// shape bucket (moa_tune_dense / moa_tune_load) when there is one, else the
// width with the least total tile cost.  The balance of all tiles over the
// SMs is left to the LPT dealing of the work list.  (A per-thread
// moa_set_block_n of 64, 128 or 256 forces the width here too.)
int plan_bn(const moa_gemm_desc& d) {
    const int ov = tile_override();
    if (ov == 64 || ov == 128 || ov == 256) return ov;
    const int tuned = tuned_block_n(MOA_BF16, d.m, d.n, d.p);
    if (tuned == 64 || tuned == 128 || tuned == 256) return tuned;
    const int64_t tiles_m = ceil_div(d.m, kGBM);
    int best = 256;
    double best_cost = 1e300;
    for (int bn : {256, 128, 64}) {
        const double cost = static_cast<double>(tiles_m * ceil_div(d.p, bn)) * tile_cost(d.n, bn);
        if (cost < best_cost * 0.999) {
            best_cost = cost;
            best = bn;
        }
    }
    return best;
}

struct Layout {
    size_t maps_off, groups_off, tiles_off, begin_off, total;
};

Layout layout_for(int G, long T, int grid) {
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    Layout L{};
    size_t off = 0;
    L.maps_off = off;
    off += al(static_cast<size_t>(2) * G * sizeof(CUtensorMap));
    L.groups_off = off;
    off += al(static_cast<size_t>(G) * sizeof(GroupDev));
    L.tiles_off = off;
    off += al(static_cast<size_t>(T) * sizeof(int4));
    L.begin_off = off;
    off += al(static_cast<size_t>(grid + 1) * sizeof(int));
    L.total = off;
    return L;
}

// Pinned host staging for the per-call tables: a ring of buffers per thread,
// each guarded by an event recorded after the copy that reads it, so a call
// only waits when it laps a copy that has not finished.
struct Staging {
    static constexpr int kRing = 4;
    void* p[kRing] = {nullptr};
    size_t bytes[kRing] = {0};
    cudaEvent_t ev[kRing] = {nullptr};
    int next = 0;
    ~Staging() {
        for (int i = 0; i < kRing; ++i) {
            if (ev[i]) {
                cudaEventSynchronize(ev[i]);
                cudaEventDestroy(ev[i]);
            }
            if (p[i]) cudaFreeHost(p[i]);
        }
    }
    void* get(size_t n, int* slot) {
        const int i = next;
        next = (next + 1) % kRing;
        if (ev[i]) {
            cudaEventSynchronize(ev[i]);
        } else if (cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) != cudaSuccess) {
            return nullptr;
        }
        if (n > bytes[i]) {
            if (p[i]) cudaFreeHost(p[i]);
            p[i] = nullptr;
            bytes[i] = 0;
            if (cudaHostAlloc(&p[i], n, cudaHostAllocDefault) != cudaSuccess) return nullptr;
            bytes[i] = n;
        }
        *slot = i;
        return p[i];
    }
    void release(int slot, cudaStream_t s) { cudaEventRecord(ev[slot], s); }
};
thread_local Staging t_staging;

// The last persistent plan of this thread: when a call repeats it (same
// descriptors, same workspace, same device) the device tables written by that
// call are still in the workspace and the launch reuses them.
struct PlanCache {
    std::vector<moa_gemm_desc> descs;
    void* ws = nullptr;
    int device = -1;
    int grid = 0;
    bool valid = false;
};
thread_local PlanCache t_plan;

bool same_descs(const std::vector<moa_gemm_desc>& a, int count, const moa_gemm_desc* d) {
    if (static_cast<int>(a.size()) != count) return false;
    return std::memcmp(a.data(), d, sizeof(moa_gemm_desc) * count) == 0;
}

int launch_kernel(uint8_t* dev, const Layout& L, int grid, cudaStream_t s) {
    GroupedArgs a;
    a.maps = reinterpret_cast<const CUtensorMap*>(dev + L.maps_off);
    a.groups = reinterpret_cast<const GroupDev*>(dev + L.groups_off);
    a.tiles = reinterpret_cast<const int4*>(dev + L.tiles_off);
    a.cta_begin = reinterpret_cast<const int*>(dev + L.begin_off);
    a.wait_limit_ns = wait_limit_ns();
    a.status = launch_status_ptr();
    if (!a.status) return MOA_ERR_CUDA;
    static std::atomic<uint64_t> attr_done{0};   // per device
    {
        const int rc = smem_attr_once(reinterpret_cast<const void*>(grouped_tc_kernel), kGSmem,
                                      attr_done, "cudaFuncSetAttribute(grouped)");
        if (rc != MOA_OK) return rc;
    }
    prof_begin(s);
    grouped_tc_kernel<<<grid, kGThreads, kGSmem, s>>>(a);
    cudaError_t e = cudaGetLastError();
    prof_end(s);
    if (e != cudaSuccess) return cuda_fail(e, "grouped_tc_kernel launch");
    log_msg(2, "grouped persistent launch: grid %d", grid);
    return MOA_OK;
}

}  // namespace

void* staging_get(size_t n, int* slot) { return t_staging.get(n, slot); }
void staging_release(int slot, cudaStream_t s) { t_staging.release(slot, s); }

int grouped_plan_bn(int64_t m, int64_t n, int64_t p) {
    moa_gemm_desc d{};
    d.m = m;
    d.n = n;
    d.p = p;
    d.dt = MOA_BF16;
    return plan_bn(d);
}

// Workspace of a grouped call: the persistent BF16 tables, then the grouped
// modular-slice region, then scratch for the problems run one by one.
size_t grouped_main_bytes(int count, const moa_gemm_desc* d) {
    int G = 0;
    long T = 0;
    for (int g = 0; g < count; ++g)
        if (persistent_ok(d[g])) {
            ++G;
            T += ceil_div(d[g].m, kGBM) * ceil_div(d[g].p, plan_bn(d[g]));
        }
    return G > 0 ? layout_for(G, T, static_cast<int>(std::min<long>(T, num_sms()))).total : 0;
}

size_t grouped_workspace(int count, const moa_gemm_desc* d) {
    size_t side = 0;
    for (int g = 0; g < count; ++g)
        if (!persistent_ok(d[g]) && !crt_grouped_ok(d[g]) && !split_grouped_ok(d[g]) &&
            d[g].m >= 0 && d[g].n >= 0 && d[g].p >= 0)
            side = std::max(side, workspace_bytes(d[g].m, d[g].n, d[g].p, d[g].dt, 0));
    const size_t crt = crt_grouped_workspace(count, d);
    const size_t spl = split_grouped_workspace(count, d);
    return grouped_main_bytes(count, d) + (crt + 255) / 256 * 256 + (spl + 255) / 256 * 256 + side;
}

int grouped_launch(int count, const moa_gemm_desc* d, void* ws, size_t ws_bytes, cudaStream_t s,
                   bool allow_cache, int* const* status_of) {
    const int sms = num_sms();
    std::vector<int> idx;
    std::vector<int> bn;
    long T = 0;
    for (int g = 0; g < count; ++g) {
        const moa_gemm_desc& x = d[g];
        if (!valid_dtype(x.dt)) return fail(MOA_ERR_DTYPE, "unknown dtype in descriptor");
        if (x.m < 0 || x.n < 0 || x.p < 0) return fail(MOA_ERR_ARG, "negative dimension in descriptor");
        if (x.m > 0 && x.p > 0 && x.C == nullptr) return fail(MOA_ERR_ARG, "descriptor C is NULL");
        if (x.m > 0 && x.p > 0 && x.n > 0 && (x.A == nullptr || x.B == nullptr))
            return fail(MOA_ERR_ARG, "descriptor A or B is NULL");
        if (persistent_ok(x)) {
            idx.push_back(g);
            bn.push_back(plan_bn(x));
            T += ceil_div(x.m, kGBM) * ceil_div(x.p, bn.back());
        }
    }
    const size_t need = grouped_workspace(count, d);
    if (need > 0 && (ws == nullptr || ws_bytes < need))
        return fail(MOA_ERR_WORKSPACE, "grouped workspace too small");
    if (ws && reinterpret_cast<uintptr_t>(ws) % 256)
        return fail(MOA_ERR_ALIGN, "workspace must be 256-byte aligned");
    if (T > (1L << 30)) return fail(MOA_ERR_ARG, "too many tiles in one grouped call");
    size_t main_bytes = 0;
    int device = -1;
    cudaGetDevice(&device);
    if (!idx.empty()) {
        const int G = static_cast<int>(idx.size());
        const int grid = static_cast<int>(std::min<long>(T, sms));
        const Layout L = layout_for(G, T, grid);
        main_bytes = L.total;
        uint8_t* dev = static_cast<uint8_t*>(ws);
        if (allow_cache && t_plan.valid && t_plan.ws == ws && t_plan.device == device &&
            t_plan.grid == grid && same_descs(t_plan.descs, count, d)) {
            const int rc = launch_kernel(dev, L, grid, s);
            if (rc != MOA_OK) return rc;
        } else {
            t_plan.valid = false;
            int slot = 0;
            uint8_t* host = static_cast<uint8_t*>(t_staging.get(L.total, &slot));
            if (!host) return fail(MOA_ERR_CUDA, "pinned staging buffer unavailable");
            CUtensorMap* maps = reinterpret_cast<CUtensorMap*>(host + L.maps_off);
            GroupDev* groups = reinterpret_cast<GroupDev*>(host + L.groups_off);
            int4* tiles = reinterpret_cast<int4*>(host + L.tiles_off);
            int* begin = reinterpret_cast<int*>(host + L.begin_off);
            struct Tile {
                double cost;
                int g, tm, tn;
            };
            std::vector<Tile> all;
            all.reserve(static_cast<size_t>(T));
            for (int i = 0; i < G; ++i) {
                const moa_gemm_desc& x = d[idx[i]];
                GroupDev& gd = groups[i];
                gd.C = static_cast<float*>(x.C);
                gd.m = static_cast<int>(x.m);
                gd.n = static_cast<int>(x.n);
                gd.p = static_cast<int>(x.p);
                gd.bn = bn[i];
                gd.tiles_n = static_cast<int>(ceil_div(x.p, gd.bn));
                gd.num_kb = static_cast<int>(ceil_div(x.n, kGBK));
                gd.vec_ok = (x.p % 4 == 0) && (reinterpret_cast<uintptr_t>(x.C) % 16 == 0);
                gd.pad = 0;
                int rc = make_tmap_2d(&maps[2 * i], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, x.A,
                                      static_cast<uint64_t>(x.n), static_cast<uint64_t>(x.m),
                                      static_cast<uint64_t>(x.n) * 2, kGBK, kGBM);
                if (rc != MOA_OK) return rc;
                rc = make_tmap_2d(&maps[2 * i + 1], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, x.B,
                                  static_cast<uint64_t>(x.p), static_cast<uint64_t>(x.n),
                                  static_cast<uint64_t>(x.p) * 2, 64, kGBK);
                if (rc != MOA_OK) return rc;
                const double cost = tile_cost(x.n, gd.bn);
                const int tm_n = static_cast<int>(ceil_div(x.m, kGBM));
                for (int tm = 0; tm < tm_n; ++tm)
                    for (int tn = 0; tn < gd.tiles_n; ++tn) all.push_back({cost, i, tm, tn});
            }
            // longest processing time first, each tile onto the least-loaded CTA
            std::stable_sort(all.begin(), all.end(),
                             [](const Tile& a, const Tile& b) { return a.cost > b.cost; });
            using Load = std::pair<double, int>;
            std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
            for (int c = 0; c < grid; ++c) heap.push({0.0, c});
            std::vector<std::vector<int>> per_cta(grid);
            for (size_t t = 0; t < all.size(); ++t) {
                Load l = heap.top();
                heap.pop();
                per_cta[l.second].push_back(static_cast<int>(t));
                l.first += all[t].cost;
                heap.push(l);
            }
            int pos = 0;
            for (int c = 0; c < grid; ++c) {
                begin[c] = pos;
                for (int t : per_cta[c]) tiles[pos++] = make_int4(all[t].g, all[t].tm, all[t].tn, 0);
            }
            begin[grid] = pos;
            cudaError_t e = cudaMemcpyAsync(dev, host, L.total, cudaMemcpyHostToDevice, s);
            t_staging.release(slot, s);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(grouped tables)");
            const int rc = launch_kernel(dev, L, grid, s);
            if (rc != MOA_OK) return rc;
            if (allow_cache) {
                t_plan.descs.assign(d, d + count);
                t_plan.ws = ws;
                t_plan.device = device;
                t_plan.grid = grid;
                t_plan.valid = true;
            }
        }
    }
    // modular-slice problems: one grouped sequence of launches
    const size_t crt_bytes = (crt_grouped_workspace(count, d) + 255) / 256 * 256;
    if (crt_bytes > 0) {
        const int rc = crt_grouped_launch(count, d, static_cast<uint8_t*>(ws) + main_bytes,
                                          crt_bytes, s, status_of);
        if (rc != MOA_OK) return rc;
    }
    // FP32-accuracy split problems: one pre-pass launch and one persistent GEMM
    const size_t spl_bytes = (split_grouped_workspace(count, d) + 255) / 256 * 256;
    if (spl_bytes > 0) {
        const int rc = split_grouped_launch(count, d,
                                            static_cast<uint8_t*>(ws) + main_bytes + crt_bytes,
                                            spl_bytes, s, status_of);
        if (rc != MOA_OK) return rc;
    }
    // problems outside the persistent paths, one by one on the same stream
    uint8_t* side = static_cast<uint8_t*>(ws) + main_bytes + crt_bytes + spl_bytes;
    const size_t side_bytes = ws ? ws_bytes - main_bytes - crt_bytes - spl_bytes : 0;
    for (int g = 0; g < count; ++g) {
        if (persistent_ok(d[g]) || crt_grouped_ok(d[g]) || split_grouped_ok(d[g])) continue;
        const int rc = gemm_ex(d[g].m, d[g].n, d[g].p, d[g].dt, d[g].A, d[g].B, d[g].C, 0,
                               side_bytes ? side : nullptr, side_bytes, s, nullptr);
        if (rc != MOA_OK) return rc;
    }
    return MOA_OK;
}

}  // namespace moa

extern "C" {

int moa_grouped_block_n(int64_t m, int64_t n, int64_t p) {
    if (m <= 0 || n <= 0 || p <= 0) return 0;
    return moa::grouped_plan_bn(m, n, p);
}

int moa_grouped_path(const moa_gemm_desc* d) {
    if (d == nullptr) return moa::fail(MOA_ERR_ARG, "descriptor is NULL");
    if (moa::persistent_ok(*d)) return MOA_GROUPED_BF16;
    if (moa::crt_grouped_ok(*d)) return MOA_GROUPED_CRT;
    if (moa::split_grouped_ok(*d)) return MOA_GROUPED_F32_SPLIT;
    return MOA_GROUPED_ALONE;
}

size_t moa_gemm_grouped_workspace_size(int count, const moa_gemm_desc* d) {
    if (count <= 0 || d == nullptr) return 0;
    return moa::grouped_workspace(count, d);
}

int moa_gemm_grouped(int count, const moa_gemm_desc* d, void* ws, size_t ws_bytes, void* stream) {
    moa::TraceRange tr("moa_gemm_grouped");
    if (count < 0) return moa::fail(MOA_ERR_ARG, "negative count");
    if (count == 0) return MOA_OK;
    if (d == nullptr) return moa::fail(MOA_ERR_ARG, "descriptor array is NULL");
    return moa::grouped_launch(count, d, ws, ws_bytes, static_cast<cudaStream_t>(stream), true,
                               nullptr);
}

}  // extern "C"

// ------------------------------------------------------------------ batched
// moa_gemm_batched: C[b] := A[b] . B[b] for b < batch, the 3-D contraction
// C[b, i, j] = sum_k A[b, i, k] B[b, k, j] (the Appendix's higher-dimensional
// extension of the inner product), with element strides between the batch
// entries (stride 0 broadcasts one operand).  Built on the grouped path: BF16
// batches are one persistent launch, other modes one launch per entry.
namespace moa {
namespace {
int batched_descs(int batch, int64_t m, int64_t n, int64_t p, moa_dtype dt, const void* A,
                  int64_t sa, const void* B, int64_t sb, void* C, int64_t sc,
                  std::vector<moa_gemm_desc>& d) {
    if (batch < 0) return fail(MOA_ERR_ARG, "negative batch");
    if (sa < 0 || sb < 0 || sc < 0) return fail(MOA_ERR_ARG, "negative stride");
    if (!valid_dtype(dt)) return fail(MOA_ERR_DTYPE, "unknown dtype");
    if (batch > 1 && m > 0 && p > 0 && sc < m * p)
        return fail(MOA_ERR_ARG, "C stride smaller than m * p would overlap outputs");
    const int ies = dtype_in_bytes(dt);
    const int oes = dtype_out_bytes(dt);
    d.resize(static_cast<size_t>(batch));
    for (int b = 0; b < batch; ++b) {
        d[b].m = m;
        d[b].n = n;
        d[b].p = p;
        d[b].dt = dt;
        d[b].A = static_cast<const uint8_t*>(A) + static_cast<int64_t>(b) * sa * ies;
        d[b].B = static_cast<const uint8_t*>(B) + static_cast<int64_t>(b) * sb * ies;
        d[b].C = static_cast<uint8_t*>(C) + static_cast<int64_t>(b) * sc * oes;
    }
    return MOA_OK;
}
}  // namespace
}  // namespace moa

extern "C" {

size_t moa_gemm_batched_workspace_size(int batch, int64_t m, int64_t n, int64_t p, moa_dtype dt,
                                       int64_t stride_a, int64_t stride_b, int64_t stride_c) {
    std::vector<moa_gemm_desc> d;
    // only the shapes and alignments matter for the size: use aligned stand-in pointers
    if (moa::batched_descs(batch, m, n, p, dt, reinterpret_cast<void*>(256), stride_a,
                           reinterpret_cast<void*>(256), stride_b, reinterpret_cast<void*>(256),
                           stride_c, d) != MOA_OK || batch == 0)
        return 0;
    return moa::grouped_workspace(batch, d.data());
}

int moa_gemm_batched(int batch, int64_t m, int64_t n, int64_t p, moa_dtype dt, const void* A,
                     int64_t stride_a, const void* B, int64_t stride_b, void* C, int64_t stride_c,
                     void* ws, size_t ws_bytes, void* stream) {
    moa::TraceRange tr("moa_gemm_batched");
    std::vector<moa_gemm_desc> d;
    const int rc = moa::batched_descs(batch, m, n, p, dt, A, stride_a, B, stride_b, C, stride_c, d);
    if (rc != MOA_OK) return rc;
    if (batch == 0) return MOA_OK;
    return moa::grouped_launch(batch, d.data(), ws, ws_bytes, static_cast<cudaStream_t>(stream),
                               true, nullptr);
}

}  // extern "C"
