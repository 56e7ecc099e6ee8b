// serve.cu -- moa_serve_*: a continuous-batching GEMM server.
//
// Requests (moa_gemm_desc: shapes, precision mode, device pointers to
// operands that stay resident on the GPU, and the output) are submitted from
// any host thread and queue in FIFO order.  A scheduler thread admits queued
// requests while both hold: fewer than `max_inflight` are on the GPU, and the
// request's workspace fits in the free part of the caller's HBM arena (a
// first-fit allocator over [arena, arena + arena_bytes)).  Requests that
// arrive while others run are admitted as soon as slots and memory free up
// (continuous batching, not a static queue): every pass of the scheduler
// forms a batch of all requests it can admit; the BF16 requests of a batch go
// into one grouped persistent launch, the others are launched one by one;
// launches rotate over `n_streams` CUDA streams so that their work overlaps on
// the device.  Each request's last stream operation records a CUDA event; the
// scheduler polls the oldest unfinished event of every stream (streams run in
// order), timestamps each completion when it sees it, frees the request's
// arena block and publishes the completion to moa_serve_poll.  Latency =
// completion - submission.  While requests are queued or in flight, and for
// a short grace period after the last activity, the scheduler thread polls
// without sleeping (one host core busy) so that neither admission nor
// completion waits for a thread wake-up; an idle server sleeps on a
// condition variable that moa_serve_submit signals.
// Every in-flight slot also has its own device status word (at the start of
// the arena): a request's kernels record a pipeline timeout or a non-finite
// split input there instead of in the per-device word; a one-thread kernel
// after them stores the word into mapped pinned host memory and clears it for
// the slot's next request, so the request completes with MOA_ERR_TIMEOUT /
// MOA_ERR_NONFINITE accordingly without a copy-engine transfer.
//
// Each GEMM is Eq. (eq:dnf) of Sec. 2, computed by the same kernels as a
// moa_gemm_ex call with the same arguments, so a result does not depend on
// what else is in flight.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "crt.h"
#include "split.h"
#include "internal.h"
#include "ptx.cuh"

namespace moa {
int gemm_ex(int64_t m, int64_t n, int64_t p, moa_dtype dt, const void* A, const void* B, void* C,
            int slices, void* ws, size_t ws_bytes, cudaStream_t s, moa_stats* st);
size_t workspace_bytes(int64_t m, int64_t n, int64_t p, moa_dtype dt, int slices);
size_t grouped_workspace(int count, const moa_gemm_desc* d);
int grouped_launch(int count, const moa_gemm_desc* d, void* ws, size_t ws_bytes, cudaStream_t s,
                   bool allow_cache, int* const* status_of);

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

// First-fit allocator over a caller-owned device range (256-byte granules).
class Arena {
  public:
    void init(uintptr_t base, size_t bytes) {
        base_ = base;
        bytes_ = bytes / 256 * 256;
        free_.clear();
        if (bytes_) free_[0] = bytes_;
        used_ = peak_ = 0;
    }
    static size_t granule(size_t n) { return n == 0 ? 256 : (n + 255) / 256 * 256; }
    // Offset of a free block of at least n bytes, or SIZE_MAX.
    size_t alloc(size_t n) {
        n = granule(n);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                const size_t off = it->first;
                const size_t rest = it->second - n;
                free_.erase(it);
                if (rest) free_[off + n] = rest;
                used_ += n;
                peak_ = std::max(peak_, used_);
                return off;
            }
        }
        return SIZE_MAX;
    }
    void release(size_t off, size_t n) {
        n = granule(n);
        used_ -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    void* ptr(size_t off) const { return reinterpret_cast<void*>(base_ + off); }
    size_t bytes() const { return bytes_; }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }

  private:
    uintptr_t base_ = 0;
    size_t bytes_ = 0;
    std::map<size_t, size_t> free_;
    size_t used_ = 0, peak_ = 0;
};

struct Request {
    uint64_t ticket = 0;
    moa_gemm_desc d{};
    size_t ws_bytes = 0, ws_off = 0;   // block = workspace + one 256-byte status slot
    int hidx = -1;                     // pinned host status index
    size_t extra_bytes = 0, extra_off = 0;   // grouped tables of a batch (lead request only)
    double t_submit = 0, t_start = 0, t_done = 0;
    int status = MOA_OK;
    int stream = 0;
};

}  // namespace
}  // namespace moa

struct moa_server {
    moa_serve_config cfg{};
    int device = 0;
    std::vector<cudaStream_t> streams;
    moa::Arena arena;

    std::mutex mu;
    std::condition_variable cv;
    std::deque<moa::Request> queue;               // submitted, not admitted
    std::map<uint64_t, moa::Request> inflight;    // admitted, on the GPU
    std::deque<moa_completion> done;              // completed, not yet polled
    std::vector<uint64_t> finished;               // tickets that failed to launch
    std::vector<std::deque<uint64_t>> launched;   // per stream: tickets in launch order
    std::vector<cudaEvent_t> done_ev;             // per status index: completion event
    std::vector<double> latencies_ms;
    uint64_t next_ticket = 1;
    uint64_t n_submitted = 0, n_admitted = 0, n_completed = 0, n_rejected = 0, n_failed = 0,
             n_batches = 0;
    int inflight_peak = 0;
    int next_stream = 0;
    int* host_status = nullptr;        // mapped pinned host memory, one int per in-flight slot
    int* host_status_dev = nullptr;    // the same memory as the device sees it
    int* dev_status = nullptr;         // device status words (arena start), one per slot
    std::vector<int> free_hidx;
    bool stop = false;
    std::thread sched;
};

namespace moa {
namespace {

// Largest modular-slice request (algorithmic flops) that joins a batch's
// grouped call: about 2 GFLOP, a few tens of microseconds of tensor work.
constexpr double kServeGroupFlops = 2.0e9;

moa_completion completion_of(const Request& r, int status, double t_done) {
    moa_completion c{};
    c.ticket = r.ticket;
    c.status = status;
    c.dt = r.d.dt;
    c.m = r.d.m;
    c.n = r.d.n;
    c.p = r.d.p;
    c.t_submit = r.t_submit;
    c.t_start = r.t_start;
    c.t_done = t_done;
    return c;
}

size_t block_bytes(size_t ws) { return Arena::granule(ws); }

// Publishes a request's status to the host (mapped pinned memory): its own
// device word if that records a failure, else the word of the launch it ran
// in (`shared`; the same word for a request launched alone).  reset_own /
// reset_shared clear the words for the slots' next requests.
__global__ void publish_status_kernel(int* own, int* shared, int* host_word, int reset_own,
                                      int reset_shared) {
    const int o = *reinterpret_cast<volatile int*>(own);
    const int v = o != kDevOk ? o : *reinterpret_cast<volatile int*>(shared);
    *reinterpret_cast<volatile int*>(host_word) = v;
    if (reset_own) *own = kDevOk;
    if (reset_shared) *shared = kDevOk;
}

int publish_status(moa_server* s, int own_slot, int shared_slot, int host_slot, bool reset_own,
                   bool reset_shared, cudaStream_t st) {
    publish_status_kernel<<<1, 1, 0, st>>>(s->dev_status + own_slot, s->dev_status + shared_slot,
                                           s->host_status_dev + host_slot, reset_own ? 1 : 0,
                                           reset_shared ? 1 : 0);
    return cudaGetLastError() == cudaSuccess ? MOA_OK : MOA_ERR_CUDA;
}

int status_of(int launch_rc, int dev) {
    if (launch_rc != MOA_OK) return launch_rc;
    if (dev == kDevTimeout) return MOA_ERR_TIMEOUT;
    if (dev == kDevNonFinite) return MOA_ERR_NONFINITE;
    return dev == kDevOk ? MOA_OK : MOA_ERR_CUDA;
}

int take_stream(moa_server* s) {
    const int si = s->next_stream;
    s->next_stream = (s->next_stream + 1) % static_cast<int>(s->streams.size());
    return si;
}

// Moves the tickets whose completion events have fired (the oldest first on
// every stream) to s->finished, with their completion times.
void collect_completions(moa_server* s) {
    for (auto& fifo : s->launched) {
        while (!fifo.empty()) {
            auto it = s->inflight.find(fifo.front());
            if (it == s->inflight.end()) {
                fifo.pop_front();
                continue;
            }
            const cudaError_t e = cudaEventQuery(s->done_ev[it->second.hidx]);
            if (e == cudaErrorNotReady) break;
            if (e != cudaSuccess && it->second.status == MOA_OK) it->second.status = MOA_ERR_CUDA;
            it->second.t_done = now_s();
            s->finished.push_back(fifo.front());
            fifo.pop_front();
        }
    }
}

void scheduler(moa_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    double last_activity = now_s();
    constexpr double kSpinGrace = 2e-3;   // seconds of polling after the last activity
    while (true) {
        // 1. retire requests the device has finished
        collect_completions(s);
        if (!s->finished.empty()) last_activity = now_s();
        for (uint64_t t : s->finished) {
            auto it = s->inflight.find(t);
            if (it == s->inflight.end()) continue;
            Request& r = it->second;
            s->arena.release(r.ws_off, block_bytes(r.ws_bytes));
            if (r.extra_bytes) s->arena.release(r.extra_off, block_bytes(r.extra_bytes));
            r.status = status_of(
                r.status,
                r.hidx >= 0 ? *reinterpret_cast<volatile int*>(s->host_status + r.hidx) : kDevOk);
            if (r.hidx >= 0) s->free_hidx.push_back(r.hidx);
            const double td = r.t_done > 0 ? r.t_done : now_s();
            s->done.push_back(completion_of(r, r.status, td));
            if (r.status == MOA_OK) {
                ++s->n_completed;
                s->latencies_ms.push_back((td - r.t_submit) * 1e3);
            } else {
                ++s->n_failed;
            }
            s->inflight.erase(it);
        }
        s->finished.clear();
        if (s->stop && s->queue.empty() && s->inflight.empty()) break;

        // 2. admit a batch: FIFO, while slots and arena memory allow
        std::vector<Request> batch;
        const double tnow = now_s();
        while (!s->queue.empty() &&
               static_cast<int>(s->inflight.size() + batch.size()) < s->cfg.max_inflight) {
            Request& r = s->queue.front();
            if (s->cfg.queue_deadline_s > 0 && tnow - r.t_submit > s->cfg.queue_deadline_s) {
                ++s->n_rejected;
                s->done.push_back(completion_of(r, MOA_ERR_REJECTED, tnow));
                s->queue.pop_front();
                continue;
            }
            const size_t off = s->arena.alloc(block_bytes(r.ws_bytes));
            if (off == SIZE_MAX) break;   // wait until memory frees up
            r.ws_off = off;
            r.hidx = s->free_hidx.back();
            s->free_hidx.pop_back();
            s->host_status[r.hidx] = kDevOk;
            r.t_start = tnow;
            batch.push_back(r);
            s->queue.pop_front();
        }
        if (batch.empty()) {
            if (!s->queue.empty() || !s->inflight.empty() ||
                now_s() - last_activity < kSpinGrace) {
                // poll: let submitters take the lock, then look again
                lk.unlock();
                std::this_thread::yield();
                lk.lock();
            } else {
                s->cv.wait_for(lk, std::chrono::microseconds(200));
                last_activity = now_s();   // a wake-up (submit or timeout) starts a new grace
            }
            continue;
        }
        last_activity = now_s();
        ++s->n_batches;
        s->n_admitted += batch.size();

        // BF16, modular-slice and FP32-accuracy split requests of the batch
        // share one grouped call (one persistent launch per kind); its
        // workspace gets its own arena block, released with the lead request
        // (all of them finish with the same kernels).
        // Only small split-precision requests join the group: a request grouped
        // with a large one would complete only when the large one does.
        auto groupable = [](const moa_gemm_desc& d) {
            return d.dt == MOA_BF16 ||
                   ((crt_grouped_ok(d) || split_grouped_ok(d)) &&
                    2.0 * d.m * d.n * d.p <= kServeGroupFlops);
        };
        std::vector<moa_gemm_desc> bf;
        std::vector<size_t> bf_idx;
        for (size_t i = 0; i < batch.size(); ++i)
            if (groupable(batch[i].d)) {
                bf.push_back(batch[i].d);
                bf_idx.push_back(i);
            }
        size_t toff = SIZE_MAX, tbytes = 0;
        if (bf.size() > 1) {
            tbytes = grouped_workspace(static_cast<int>(bf.size()), bf.data());
            toff = s->arena.alloc(block_bytes(tbytes));
            if (toff != SIZE_MAX) {
                batch[bf_idx[0]].extra_off = toff;
                batch[bf_idx[0]].extra_bytes = tbytes;
            }
        }
        const bool grouped = toff != SIZE_MAX;
        const int gstream = grouped ? take_stream(s) : 0;
        for (Request& r : batch) r.stream = (grouped && groupable(r.d)) ? gstream : take_stream(s);
        for (const Request& r : batch) s->inflight[r.ticket] = r;
        s->inflight_peak = std::max<int>(s->inflight_peak, static_cast<int>(s->inflight.size()));
        lk.unlock();

        TraceRange tr("moa_serve batch");
        log_msg(3, "serve batch of %zu requests, %zu in flight", batch.size(), s->inflight.size());
        std::vector<int> rcs(batch.size(), MOA_OK);
        if (grouped) {
            cudaStream_t gs = s->streams[gstream];
            // Failures of the shared launch (a pipeline timeout) go to the
            // lead's status word; a modular-slice request's non-finite inputs
            // go to its own word, so one bad request does not fail the rest.
            const int lead = batch[bf_idx[0]].hidx;
            std::vector<int*> own(bf.size());
            for (size_t k = 0; k < bf_idx.size(); ++k) own[k] = s->dev_status + batch[bf_idx[k]].hidx;
            set_status_override(s->dev_status + lead);
            const int rc = grouped_launch(static_cast<int>(bf.size()), bf.data(), s->arena.ptr(toff),
                                          tbytes, gs, false, own.data());
            set_status_override(nullptr);
            for (size_t k = 0; k < bf_idx.size(); ++k) {
                const size_t i = bf_idx[k];
                const bool last = k + 1 == bf_idx.size();
                const int prc = publish_status(s, batch[i].hidx, lead, batch[i].hidx,
                                               batch[i].hidx != lead, last, gs);
                rcs[i] = rc != MOA_OK ? rc : prc;
            }
        }
        std::vector<uint64_t> failed_now;
        for (size_t i = 0; i < batch.size(); ++i) {
            Request& r = batch[i];
            if (!(grouped && groupable(r.d))) {
                cudaStream_t rs = s->streams[r.stream];
                set_status_override(s->dev_status + r.hidx);
                rcs[i] = gemm_ex(r.d.m, r.d.n, r.d.p, r.d.dt, r.d.A, r.d.B, r.d.C, 0,
                                 r.ws_bytes ? s->arena.ptr(r.ws_off) : nullptr, r.ws_bytes, rs,
                                 nullptr);
                set_status_override(nullptr);
                const int prc = publish_status(s, r.hidx, r.hidx, r.hidx, true, true, rs);
                if (rcs[i] == MOA_OK) rcs[i] = prc;
            }
            if (cudaEventRecord(s->done_ev[r.hidx], s->streams[r.stream]) != cudaSuccess) {
                rcs[i] = MOA_ERR_CUDA;
                failed_now.push_back(r.ticket);
            }
        }
        lk.lock();
        {
            size_t f = 0;
            for (const Request& r : batch) {
                if (f < failed_now.size() && failed_now[f] == r.ticket) {
                    ++f;
                    continue;
                }
                s->launched[r.stream].push_back(r.ticket);
            }
        }
        for (size_t i = 0; i < batch.size(); ++i) {
            auto it = s->inflight.find(batch[i].ticket);
            if (it != s->inflight.end() && rcs[i] != MOA_OK) it->second.status = rcs[i];
        }
        for (uint64_t t : failed_now) s->finished.push_back(t);
    }
}

}  // namespace
}  // namespace moa

extern "C" {

int moa_serve_create(const moa_serve_config* cfg, moa_server** out) {
    if (!cfg || !out) return moa::fail(MOA_ERR_ARG, "NULL config or output");
    if (cfg->arena_bytes > 0 && cfg->arena == nullptr) return moa::fail(MOA_ERR_ARG, "arena is NULL");
    if (reinterpret_cast<uintptr_t>(cfg->arena) % 256)
        return moa::fail(MOA_ERR_ALIGN, "arena must be 256-byte aligned");
    if (cfg->max_inflight <= 0 || cfg->n_streams <= 0 || cfg->n_streams > 64)
        return moa::fail(MOA_ERR_ARG, "max_inflight must be > 0 and n_streams in 1..64");
    moa_server* s = new moa_server();
    s->cfg = *cfg;
    if (s->cfg.queue_capacity <= 0) s->cfg.queue_capacity = 65536;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e != cudaSuccess) {
        delete s;
        return moa::cuda_fail(e, "cudaGetDevice");
    }
    for (int i = 0; i < cfg->n_streams; ++i) {
        cudaStream_t st;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
            delete s;
            return moa::cuda_fail(e, "cudaStreamCreateWithFlags");
        }
        s->streams.push_back(st);
    }
    // the first bytes of the arena hold the per-slot device status words
    const size_t words = moa::Arena::granule(sizeof(int) * static_cast<size_t>(cfg->max_inflight));
    if (cfg->arena_bytes < words) {
        for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
        delete s;
        return moa::fail(MOA_ERR_BUDGET, "arena smaller than the status words of the slots");
    }
    s->dev_status = static_cast<int*>(cfg->arena);
    s->arena.init(reinterpret_cast<uintptr_t>(cfg->arena) + words, cfg->arena_bytes - words);
    e = cudaMemset(s->dev_status, 0, words);
    if (e == cudaSuccess)
        e = cudaHostAlloc(reinterpret_cast<void**>(&s->host_status),
                          sizeof(int) * static_cast<size_t>(cfg->max_inflight),
                          cudaHostAllocMapped);
    if (e == cudaSuccess)
        e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&s->host_status_dev), s->host_status, 0);
    if (e != cudaSuccess) {
        if (s->host_status) cudaFreeHost(s->host_status);
        for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
        delete s;
        return moa::cuda_fail(e, "status words");
    }
    for (int i = cfg->max_inflight - 1; i >= 0; --i) s->free_hidx.push_back(i);
    s->done_ev.assign(static_cast<size_t>(cfg->max_inflight), nullptr);
    for (cudaEvent_t& ev : s->done_ev) {
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            for (cudaEvent_t x : s->done_ev)
                if (x) cudaEventDestroy(x);
            for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
            cudaFreeHost(s->host_status);
            delete s;
            return moa::cuda_fail(e, "cudaEventCreateWithFlags");
        }
    }
    s->launched.resize(s->streams.size());
    s->sched = std::thread(moa::scheduler, s);
    *out = s;
    return MOA_OK;
}

int moa_serve_submit(moa_server* s, const moa_gemm_desc* d, uint64_t* ticket) {
    if (!s || !d || !ticket) return moa::fail(MOA_ERR_ARG, "NULL argument");
    const moa_gemm_desc& x = *d;
    if (!moa::valid_dtype(x.dt)) return moa::fail(MOA_ERR_DTYPE, "unknown dtype");
    if (x.m < 0 || x.n < 0 || x.p < 0) return moa::fail(MOA_ERR_ARG, "negative dimension");
    if (x.m > 0 && x.p > 0 && (!x.C || (x.n > 0 && (!x.A || !x.B))))
        return moa::fail(MOA_ERR_ARG, "NULL operand");
    moa::Request r;
    r.d = x;
    r.ws_bytes = moa::workspace_bytes(x.m, x.n, x.p, x.dt, 0);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return moa::fail(MOA_ERR_REJECTED, "server is shutting down");
        if (moa::block_bytes(r.ws_bytes) > s->arena.bytes()) {
            ++s->n_rejected;
            return moa::fail(MOA_ERR_BUDGET, "request workspace exceeds the arena");
        }
        if (static_cast<int>(s->queue.size()) >= s->cfg.queue_capacity) {
            ++s->n_rejected;
            return moa::fail(MOA_ERR_BUSY, "queue full");
        }
        r.ticket = s->next_ticket++;
        r.t_submit = moa::now_s();
        s->queue.push_back(r);
        ++s->n_submitted;
        *ticket = r.ticket;
    }
    s->cv.notify_all();
    return MOA_OK;
}

int moa_serve_poll(moa_server* s, moa_completion* out, int max, int* n_out) {
    if (!s || !n_out || (max > 0 && !out)) return moa::fail(MOA_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    int n = 0;
    while (n < max && !s->done.empty()) {
        out[n++] = s->done.front();
        s->done.pop_front();
    }
    *n_out = n;
    return MOA_OK;
}

int moa_serve_stats(moa_server* s, moa_serve_counters* st) {
    if (!s || !st) return moa::fail(MOA_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *st = moa_serve_counters{};
    st->submitted = s->n_submitted;
    st->admitted = s->n_admitted;
    st->completed = s->n_completed;
    st->rejected = s->n_rejected;
    st->failed = s->n_failed;
    st->batches = s->n_batches;
    st->queued = s->queue.size();
    st->inflight = s->inflight.size();
    st->inflight_peak = s->inflight_peak;
    st->arena_peak = s->arena.peak();
    st->arena_used = s->arena.used();
    std::vector<double> v = s->latencies_ms;
    if (!v.empty()) {
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) {
            const size_t i = std::min(v.size() - 1, static_cast<size_t>(q * (v.size() - 1) + 0.5));
            return v[i];
        };
        st->p50_ms = pct(0.50);
        st->p99_ms = pct(0.99);
        st->max_ms = v.back();
        double sum = 0;
        for (double x : v) sum += x;
        st->mean_ms = sum / v.size();
    }
    return MOA_OK;
}

int moa_serve_destroy(moa_server* s) {
    if (!s) return moa::fail(MOA_ERR_ARG, "NULL server");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->sched.joinable()) s->sched.join();
    int rc = MOA_OK;
    for (cudaStream_t st : s->streams) {
        if (cudaStreamSynchronize(st) != cudaSuccess) rc = MOA_ERR_CUDA;
        cudaStreamDestroy(st);
    }
    for (cudaEvent_t ev : s->done_ev)
        if (ev) cudaEventDestroy(ev);
    if (s->host_status) cudaFreeHost(s->host_status);
    delete s;
    return rc;
}

}  // extern "C"
