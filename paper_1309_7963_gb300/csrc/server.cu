// Serving loop (host code): continuous batching of interaction requests from a transport
// driver. Requests are queued on submit; a scheduler thread admits them in order whenever a
// stream is free and both the device output arena and the pinned host arena have room for
// the request (memory-based admission). Every admitted request is one persistent-kernel
// launch on its own stream, so requests that arrive while others run overlap on the GPU.
// A request whose secondaries overflow its reservation is run again with room for exactly
// its count: results depend only on (seed, event id), so the re-run is identical.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "api_internal.h"

using namespace pnuc;
using Clock = std::chrono::steady_clock;

namespace {

// First-fit allocator over [0, size) with 256-byte granules.
class Arena {
  public:
    explicit Arena(size_t size) : size_(size) { free_[0] = size; }
    bool alloc(size_t bytes, size_t &off)
    {
        bytes = (bytes + 255) / 256 * 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            off = it->first;
            size_t rest = it->second - bytes;
            free_.erase(it);
            if (rest) free_[off + bytes] = rest;
            used_ += bytes;
            peak_ = std::max(peak_, used_);
            return true;
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = (bytes + 255) / 256 * 256;
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t size() const { return size_; }
    size_t peak() const { return peak_; }

  private:
    size_t size_, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;
};

enum State { kPending, kRunning, kDone, kFailed };

struct Request {
    uint64_t ticket, n, seed, first;
    std::vector<double> e;
    std::vector<int32_t> t;
    uint64_t cap = 0;  // secondaries reserved
    State state = kPending;
    pnuc_status status = PNUC_OK;
    int stream = -1;
    size_t dev_off = 0, host_off = 0, bytes = 0;
    bool has_dev = false, has_host = false;
    unsigned long long count = 0;
    int reruns = 0;
    Clock::time_point t_submit, t_admit, t_done;
};

// byte offsets inside one reservation
struct Layout {
    size_t count = 0, e, t, r, s, total;
    Layout(uint64_t n, uint64_t cap)
    {
        auto up = [](size_t b) { return (b + 255) / 256 * 256; };
        e = 256;
        t = e + up(8 * n);
        r = t + up(4 * n);
        s = r + up(sizeof(pnuc_residual) * n);
        total = s + up(sizeof(pnuc_secondary) * cap);
    }
};

}  // namespace

struct pnuc_server {
    pnuc_ctx *ctx = nullptr;
    pnuc_server_config cfg;
    unsigned char *dev = nullptr;   // device arena
    unsigned char *host = nullptr;  // pinned host arena (same size)
    std::unique_ptr<Arena> dev_arena, host_arena;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    std::vector<uint64_t> stream_owner;  // ticket of the request on each stream, 0 if free
    std::mutex mu;
    std::condition_variable cv;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    // statistics
    std::vector<double> latencies_ms, queue_ms;
    uint64_t completed = 0, events_done = 0, failed = 0, reruns = 0;
    Clock::time_point t_start;
    char err[256] = {0};
};

namespace {

void finish(pnuc_server *S, Request &r, State st, pnuc_status status)
{
    r.state = st;
    r.status = status;
    r.t_done = Clock::now();
    if (r.has_dev) {
        S->dev_arena->release(r.dev_off, r.bytes);
        r.has_dev = false;
    }
    if (st == kFailed && r.has_host) {
        S->host_arena->release(r.host_off, r.bytes);
        r.has_host = false;
    }
    if (r.stream >= 0) S->stream_owner[r.stream] = 0;
    r.stream = -1;
    if (st == kDone) {
        S->completed++;
        S->events_done += r.n;
        S->latencies_ms.push_back(std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count());
        S->queue_ms.push_back(std::chrono::duration<double, std::milli>(r.t_admit - r.t_submit).count());
    } else {
        S->failed++;
    }
}

// Tries to admit request r on a free stream; returns false if it must wait.
bool admit(pnuc_server *S, Request &r)
{
    int si = -1;
    for (size_t k = 0; k < S->streams.size(); ++k)
        if (S->stream_owner[k] == 0) {
            si = (int)k;
            break;
        }
    if (si < 0) return false;
    Layout L(r.n, r.cap);
    size_t doff, hoff;
    if (!S->dev_arena->alloc(L.total, doff)) return false;
    if (!S->host_arena->alloc(L.total, hoff)) {
        S->dev_arena->release(doff, L.total);
        return false;
    }
    r.dev_off = doff;
    r.host_off = hoff;
    r.bytes = L.total;
    r.has_dev = r.has_host = true;
    r.stream = si;
    S->stream_owner[si] = r.ticket;
    if (r.reruns == 0) r.t_admit = Clock::now();
    unsigned char *d = S->dev + doff, *h = S->host + hoff;
    cudaStream_t s = S->streams[si];
    memcpy(h + L.e, r.e.data(), 8 * r.n);
    memcpy(h + L.t, r.t.data(), 4 * r.n);
    pnuc_batch b = {(const double *)(d + L.e), (const int32_t *)(d + L.t), r.n, r.seed, r.first};
    pnuc_output o = {r.cap ? (pnuc_secondary *)(d + L.s) : nullptr, r.cap, (unsigned long long *)(d + L.count),
                     (pnuc_residual *)(d + L.r), nullptr};
    pnuc_status st = PNUC_OK;
    if (cudaMemcpyAsync(d + L.e, h + L.e, 8 * r.n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(d + L.t, h + L.t, 4 * r.n, cudaMemcpyHostToDevice, s) != cudaSuccess)
        st = PNUC_ERR_CUDA;
    if (st == PNUC_OK) st = launch_batch(S->ctx, (pnuc_precision)S->cfg.precision, PNUC_PERSISTENT, &b, &o, s,
                                         S->ctx->tuning[S->cfg.precision], nullptr);
    // the count, the residuals and the whole reservation of secondaries come back in the same
    // stream order, so one completion event covers them (a count above the reservation
    // sends the request round again)
    if (st == PNUC_OK &&
        (cudaMemcpyAsync(h + L.count, d + L.count, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
         cudaMemcpyAsync(h + L.r, d + L.r, sizeof(pnuc_residual) * r.n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
         (r.cap && cudaMemcpyAsync(h + L.s, d + L.s, sizeof(pnuc_secondary) * r.cap, cudaMemcpyDeviceToHost, s) !=
                       cudaSuccess) ||
         cudaEventRecord(S->events[si], s) != cudaSuccess))
        st = PNUC_ERR_CUDA;
    if (st != PNUC_OK) {
        finish(S, r, kFailed, st);
        return true;
    }
    r.state = kRunning;
    return true;
}

void poll(pnuc_server *S, Request &r)
{
    cudaError_t q = cudaEventQuery(S->events[r.stream]);
    if (q == cudaErrorNotReady) return;
    if (q != cudaSuccess) {
        finish(S, r, kFailed, PNUC_ERR_CUDA);
        return;
    }
    Layout L(r.n, r.cap);
    const unsigned char *h = S->host + r.host_off;
    r.count = *(volatile const unsigned long long *)(h + L.count);
    if (r.count > r.cap) {
        // overflow: release and run again with room for exactly the count
        S->dev_arena->release(r.dev_off, r.bytes);
        S->host_arena->release(r.host_off, r.bytes);
        r.has_dev = r.has_host = false;
        S->stream_owner[r.stream] = 0;
        r.stream = -1;
        if (Layout(r.n, r.count).total > S->cfg.arena_bytes) {
            finish(S, r, kFailed, PNUC_ERR_CAPACITY);
            return;
        }
        r.cap = r.count;
        r.reruns++;
        S->reruns++;
        r.state = kPending;
        S->pending.push_front(r.ticket);
        return;
    }
    finish(S, r, kDone, PNUC_OK);  // results are in the pinned host arena until fetched
}

void scheduler(pnuc_server *S)
{
    cudaSetDevice(S->ctx->cfg.device);
    std::unique_lock<std::mutex> lock(S->mu);
    while (true) {
        for (size_t k = 0; k < S->streams.size(); ++k) {
            if (!S->stream_owner[k]) continue;
            auto it = S->reqs.find(S->stream_owner[k]);
            if (it == S->reqs.end()) continue;
            State before = it->second->state;
            poll(S, *it->second);
            if (it->second->state != before) S->cv.notify_all();
        }
        while (!S->pending.empty()) {
            auto it = S->reqs.find(S->pending.front());
            if (it == S->reqs.end()) {
                S->pending.pop_front();
                continue;
            }
            if (!admit(S, *it->second)) break;
            S->pending.pop_front();
            if (it->second->state == kFailed) S->cv.notify_all();
        }
        bool inflight = false;
        for (uint64_t t : S->stream_owner) inflight = inflight || t != 0;
        if (S->stop && !inflight) break;
        S->cv.wait_for(lock, inflight ? std::chrono::microseconds(50) : std::chrono::milliseconds(2));
    }
}

double percentile(std::vector<double> v, double q)
{
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    size_t k = (size_t)std::min<double>(v.size() - 1, q * (v.size() - 1) + 0.5);
    return v[k];
}

}  // namespace

extern "C" {

void pnuc_server_default_config(pnuc_server_config *cfg)
{
    if (!cfg) return;
    cfg->precision = PNUC_FP32;
    cfg->streams = 8;
    cfg->arena_bytes = 1ull << 30;
    cfg->sec_per_event = 12;
    cfg->max_pending = 4096;
    cfg->max_request_events = 1ull << 24;
}

pnuc_status pnuc_server_destroy(pnuc_server *S)
{
    if (!S) return PNUC_OK;
    if (S->worker.joinable()) {
        {
            std::lock_guard<std::mutex> lock(S->mu);
            S->stop = true;
            S->pending.clear();
        }
        S->cv.notify_all();
        S->worker.join();
    }
    cudaSetDevice(S->ctx->cfg.device);
    for (auto s : S->streams) cudaStreamSynchronize(s);
    for (auto s : S->streams) cudaStreamDestroy(s);
    for (auto e : S->events) cudaEventDestroy(e);
    cudaFree(S->dev);
    cudaFreeHost(S->host);
    delete S;
    return PNUC_OK;
}

pnuc_status pnuc_server_create(pnuc_ctx *ctx, const pnuc_server_config *cfg_in, pnuc_server **out)
{
    if (!ctx || !out) return fail(ctx, PNUC_ERR_ARG, "null argument");
    *out = nullptr;
    pnuc_server_config cfg;
    pnuc_server_default_config(&cfg);
    if (cfg_in) cfg = *cfg_in;
    if ((cfg.precision != PNUC_FP32 && cfg.precision != PNUC_FP64) || cfg.streams < 1 || cfg.streams > 64 ||
        cfg.arena_bytes < (1u << 20) || cfg.sec_per_event < 1 || cfg.sec_per_event > 256 || cfg.max_pending < 1 ||
        cfg.max_request_events < 1)
        return fail(ctx, PNUC_ERR_ARG, "bad server configuration");
    CU(ctx, cudaSetDevice(ctx->cfg.device));
    pnuc_server *S = new pnuc_server();
    S->ctx = ctx;
    S->cfg = cfg;
    S->t_start = Clock::now();
    if (cudaMalloc(&S->dev, cfg.arena_bytes) != cudaSuccess ||
        cudaMallocHost(&S->host, cfg.arena_bytes) != cudaSuccess) {
        pnuc_server_destroy(S);
        return fail(ctx, PNUC_ERR_CUDA, "server arenas of %llu bytes could not be allocated",
                    (unsigned long long)cfg.arena_bytes);
    }
    S->dev_arena.reset(new Arena(cfg.arena_bytes));
    S->host_arena.reset(new Arena(cfg.arena_bytes));
    for (int k = 0; k < cfg.streams; ++k) {
        cudaStream_t s;
        cudaEvent_t e;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            pnuc_server_destroy(S);
            return fail(ctx, PNUC_ERR_CUDA, "stream creation failed");
        }
        S->streams.push_back(s);
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            pnuc_server_destroy(S);
            return fail(ctx, PNUC_ERR_CUDA, "event creation failed");
        }
        S->events.push_back(e);
        S->stream_owner.push_back(0);
    }
    S->worker = std::thread(scheduler, S);
    *out = S;
    return PNUC_OK;
}

pnuc_status pnuc_server_submit(pnuc_server *S, const double *energies, const int32_t *target_ids, uint64_t n,
                               uint64_t seed, uint64_t first_event_id, uint64_t *ticket)
{
    if (!S || !ticket || (n > 0 && (!energies || !target_ids))) return PNUC_ERR_ARG;
    if (n == 0 || n > S->cfg.max_request_events) return fail(S->ctx, PNUC_ERR_ARG, "request of %llu events", (unsigned long long)n);
    uint64_t cap = n * S->cfg.sec_per_event;
    if (Layout(n, cap).total > S->cfg.arena_bytes)
        return fail(S->ctx, PNUC_ERR_ARG, "request of %llu events can never fit the %llu-byte arena",
                    (unsigned long long)n, (unsigned long long)S->cfg.arena_bytes);
    std::unique_ptr<Request> r(new Request());
    r->n = n;
    r->seed = seed;
    r->first = first_event_id;
    r->cap = cap;
    r->e.assign(energies, energies + n);
    r->t.assign(target_ids, target_ids + n);
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lock(S->mu);
        if (S->pending.size() >= S->cfg.max_pending) return PNUC_ERR_CAPACITY;
        r->ticket = S->next_ticket++;
        *ticket = r->ticket;
        S->pending.push_back(r->ticket);
        S->reqs[r->ticket] = std::move(r);
    }
    S->cv.notify_all();
    return PNUC_OK;
}

pnuc_status pnuc_server_wait(pnuc_server *S, uint64_t ticket, int32_t timeout_ms, uint64_t *n_secondaries)
{
    if (!S) return PNUC_ERR_ARG;
    std::unique_lock<std::mutex> lock(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return PNUC_ERR_ARG;
    Request *r = it->second.get();
    auto done = [&] { return r->state == kDone || r->state == kFailed; };
    if (timeout_ms < 0) S->cv.wait(lock, done);
    else if (!S->cv.wait_for(lock, std::chrono::milliseconds(timeout_ms), done)) return PNUC_ERR_TIMEOUT;
    if (n_secondaries) *n_secondaries = r->count;
    return r->status;
}

pnuc_status pnuc_server_fetch(pnuc_server *S, uint64_t ticket, pnuc_secondary *secondaries, uint64_t capacity,
                              pnuc_residual *residuals)
{
    if (!S) return PNUC_ERR_ARG;
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return PNUC_ERR_ARG;
    Request *r = it->second.get();
    if (r->state == kFailed) {
        pnuc_status st = r->status;
        S->reqs.erase(it);
        return st;
    }
    if (r->state != kDone) return PNUC_ERR_STATE;
    if (!residuals || (r->count > 0 && (!secondaries || capacity < r->count))) return PNUC_ERR_CAPACITY;
    Layout L(r->n, r->cap);
    const unsigned char *h = S->host + r->host_off;
    memcpy(residuals, h + L.r, sizeof(pnuc_residual) * r->n);
    if (r->count) memcpy(secondaries, h + L.s, sizeof(pnuc_secondary) * r->count);
    S->host_arena->release(r->host_off, r->bytes);
    S->reqs.erase(it);
    S->cv.notify_all();
    return PNUC_OK;
}

pnuc_status pnuc_server_view(pnuc_server *S, uint64_t ticket, const pnuc_secondary **secondaries,
                             uint64_t *n_secondaries, const pnuc_residual **residuals)
{
    if (!S || !secondaries || !n_secondaries || !residuals) return PNUC_ERR_ARG;
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return PNUC_ERR_ARG;
    Request *r = it->second.get();
    if (r->state == kFailed) {
        pnuc_status st = r->status;
        S->reqs.erase(it);
        return st;
    }
    if (r->state != kDone) return PNUC_ERR_STATE;
    Layout L(r->n, r->cap);
    const unsigned char *h = S->host + r->host_off;
    *residuals = reinterpret_cast<const pnuc_residual *>(h + L.r);
    *secondaries = reinterpret_cast<const pnuc_secondary *>(h + L.s);
    *n_secondaries = r->count;
    return PNUC_OK;
}

pnuc_status pnuc_server_release(pnuc_server *S, uint64_t ticket)
{
    if (!S) return PNUC_ERR_ARG;
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return PNUC_ERR_ARG;
    Request *r = it->second.get();
    if (r->state != kDone && r->state != kFailed) return PNUC_ERR_STATE;
    if (r->has_host) S->host_arena->release(r->host_off, r->bytes);
    S->reqs.erase(it);
    S->cv.notify_all();
    return PNUC_OK;
}

pnuc_status pnuc_server_get_stats(pnuc_server *S, pnuc_server_stats *out)
{
    if (!S || !out) return PNUC_ERR_ARG;
    std::lock_guard<std::mutex> lock(S->mu);
    memset(out, 0, sizeof *out);
    out->completed = S->completed;
    out->failed = S->failed;
    out->reruns = S->reruns;
    out->events = S->events_done;
    out->pending = S->pending.size();
    out->latency_p50_ms = percentile(S->latencies_ms, 0.50);
    out->latency_p99_ms = percentile(S->latencies_ms, 0.99);
    out->latency_max_ms = percentile(S->latencies_ms, 1.0);
    out->queue_p50_ms = percentile(S->queue_ms, 0.50);
    out->queue_p99_ms = percentile(S->queue_ms, 0.99);
    double secs = std::chrono::duration<double>(Clock::now() - S->t_start).count();
    out->elapsed_s = secs;
    out->events_per_s = secs > 0 ? S->events_done / secs : 0.0;
    out->arena_peak_bytes = S->dev_arena->peak();
    return PNUC_OK;
}

pnuc_status pnuc_server_reset_stats(pnuc_server *S)
{
    if (!S) return PNUC_ERR_ARG;
    std::lock_guard<std::mutex> lock(S->mu);
    S->latencies_ms.clear();
    S->queue_ms.clear();
    S->completed = S->events_done = S->failed = S->reruns = 0;
    S->t_start = Clock::now();
    return PNUC_OK;
}

}  // extern "C"
