// Serving loop (host code, plus the partition kernel of merged launches): continuous batching
// of interaction requests from a transport driver. Requests are queued on submit; a scheduler
// thread admits them in order whenever a stream is free and both the device arena and the
// pinned host arena have room (memory-based admission). Queued requests with the same seed
// are merged into one persistent launch ("group"), each event keeping its own id, so that
// many small requests share one launch instead of each paying the tail of its slowest event;
// a partition kernel then gives every request of the group its own contiguous range of
// secondaries, renumbered to its own events. A request whose secondaries overflow its
// reservation is run again alone with room for exactly its count: results depend only on
// (seed, event id), so the re-run is identical.
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

constexpr int kMaxSeg = 64;                   // requests per group
constexpr uint64_t kMaxGroupEvents = 1u << 22;  // events per group

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
    std::vector<uint8_t> proj;  // incident species per event (1 proton, 0 neutron); empty = protons
    uint64_t cap = 0;  // secondaries reserved
    bool solo = false; // run alone (after an overflow)
    State state = kPending;
    pnuc_status status = PNUC_OK;
    uint64_t group = 0;  // its group while running or until released
    unsigned long long count = 0;
    const pnuc_residual *res_view = nullptr;   // results in the group's host region
    const pnuc_secondary *sec_view = nullptr;
    int reruns = 0;
    Clock::time_point t_submit, t_admit, t_done;
    pnuc_server_trace_entry tr{};  // the trace fields of its last run
};

auto up = [](size_t b) { return (b + 255) / 256 * 256; };

// Byte offsets of one group in the arenas. Device: header, inputs, and (for more than one
// request) the launch's secondaries; host: header, residuals, secondaries. The kernels write
// the residuals, and a single request's secondaries, straight into the pinned host region
// (mapped memory); the partition kernel writes merged requests' secondaries there too, so
// only the counts are copied back.
struct GroupLayout {
    // header: [0] launch count, [8 .. 8+8*kMaxSeg) per-request counts (device -> host), then
    // the segment tables (host -> device): seg_start (u32, kMaxSeg + 1), seg_first (u64,
    // kMaxSeg), cap_start (u64, kMaxSeg + 1)
    // the trace's GPU time stamps of the launch (start, end; nanoseconds of the GPU's global
    // timer, written by stamp_kernel into the host region)
    static constexpr size_t count = 0, seg_count = 8, seg_start = 8 + 8 * kMaxSeg, seg_first = 1024,
                            cap_start = seg_first + 8 * kMaxSeg, stamps = 2288, header = 2304;
    static_assert(seg_start + 4 * (kMaxSeg + 1) <= seg_first && cap_start + 8 * (kMaxSeg + 1) <= stamps,
                  "group header fields overlap");
    size_t e, t, pj, s, dev_total, host_r, host_s, host_total;
    GroupLayout(uint64_t n, uint64_t cap, int n_seg)
    {
        e = header;
        t = e + up(8 * n);
        pj = t + up(4 * n);  // incident species, when a request of the group has them
        s = pj + up(n);
        dev_total = n_seg > 1 ? s + up(sizeof(pnuc_secondary) * cap) : s;
        host_r = header;
        host_s = host_r + up(sizeof(pnuc_residual) * n);
        host_total = host_s + up(sizeof(pnuc_secondary) * cap);
    }
    bool fits(uint64_t arena) const { return dev_total <= arena && host_total <= arena; }
};

struct Group {
    uint64_t id;
    uint64_t launch = 0;            // the server's launch number
    bool traced = false;            // its stream's timing events were recorded around it
    Clock::time_point t_launched;   // copies and kernels enqueued
    std::vector<uint64_t> tickets;  // segment order
    uint64_t n = 0, cap = 0;
    size_t dev_off = 0, host_off = 0, dev_bytes = 0, host_bytes = 0;
    bool has_dev = false;
    int stream = -1;
    int live = 0;  // requests not yet released: the host region is freed at 0
};

// The trace's GPU time stamp: the GPU's global timer (nanoseconds) when the stream reaches it.
__global__ void stamp_kernel(unsigned long long *dst)
{
    if (threadIdx.x == 0) {
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        *dst = t;
    }
}

// Partition of a merged launch's secondaries: record i of event e (segment k) goes to
// out[cap_start[k] + (its rank in segment k)], with its event renumbered e - seg_start[k].
// Ranks come from atomics on the per-segment counts, which also report overflows.
__global__ void partition_kernel(const uint4 *__restrict__ in, const unsigned long long *launch_count,
                                 uint64_t cap, const uint32_t *__restrict__ seg_start,
                                 const unsigned long long *__restrict__ cap_start, int n_seg,
                                 unsigned long long *seg_count, uint4 *out)
{
    const unsigned long long n = min(*launch_count, (unsigned long long)cap);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        uint4 a = in[2 * i];
        const uint4 b = in[2 * i + 1];
        const uint32_t ev = a.x;
        int lo = 0, hi = n_seg - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (seg_start[mid] <= ev) lo = mid;
            else hi = mid - 1;
        }
        const unsigned long long rank = atomicAdd(&seg_count[lo], 1ull);
        if (rank < cap_start[lo + 1] - cap_start[lo]) {
            a.x = ev - seg_start[lo];
            out[2 * (cap_start[lo] + rank)] = a;
            out[2 * (cap_start[lo] + rank) + 1] = b;
        }
    }
}

}  // namespace

struct pnuc_server {
    pnuc_ctx *ctx = nullptr;
    pnuc_server_config cfg;
    unsigned char *dev = nullptr;       // device arena
    unsigned char *host = nullptr;      // pinned host arena (same size)
    unsigned char *host_dev = nullptr;  // the host arena's device address
    std::unique_ptr<Arena> dev_arena, host_arena;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    std::vector<uint64_t> stream_owner;  // group on each stream, 0 if free
    std::mutex mu;
    std::condition_variable cv;
    std::deque<uint64_t> pending;
    std::deque<uint64_t> finished;  // tickets in the order they finished, for wait_any
    std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
    std::unordered_map<uint64_t, std::unique_ptr<Group>> groups;
    uint64_t next_ticket = 1, next_group = 1;
    bool stop = false;
    std::thread worker;
    // statistics
    std::vector<double> latencies_ms, queue_ms;
    uint64_t completed = 0, events_done = 0, failed = 0, reruns = 0, launches = 0;
    Clock::time_point t_start;
    // pnuc_server_trace: the epoch (its host time and GPU global timer, read through a pinned
    // word), and the entries
    bool tracing = false;
    Clock::time_point t_epoch;
    unsigned long long gpu_epoch_ns = 0;
    unsigned long long *epoch_word = nullptr;  // pinned, mapped
    std::vector<pnuc_server_trace_entry> trace;
};

namespace {

// Trace times: milliseconds from the trace's start on the host clock; a GPU stamp's time from
// its distance to the epoch's stamp.
double trace_ms(const pnuc_server *S, Clock::time_point t)
{
    return std::chrono::duration<double, std::milli>(t - S->t_epoch).count();
}

double gpu_ms(const pnuc_server *S, unsigned long long ns)
{
    return 1e-6 * (double)(long long)(ns - S->gpu_epoch_ns);
}

// A request leaves the server: its trace entry (if tracing) goes to the record.
void record_release(pnuc_server *S, Request &r)
{
    if (!S->tracing || S->trace.size() >= (1u << 20) || r.tr.launch == 0) return;
    pnuc_server_trace_entry e = r.tr;
    e.ticket = r.ticket;
    e.events = r.n;
    e.reruns = r.reruns;
    e.status = r.status;
    e.t_submit = trace_ms(S, r.t_submit);
    e.t_admit = trace_ms(S, r.t_admit);
    e.t_complete = trace_ms(S, r.t_done);
    e.t_release = trace_ms(S, Clock::now());
    S->trace.push_back(e);
}

// Drops a request's claim on its group; frees the group's host region when none is left.
void leave_group(pnuc_server *S, Request &r)
{
    if (!r.group) return;
    auto it = S->groups.find(r.group);
    r.group = 0;
    r.res_view = nullptr;
    r.sec_view = nullptr;
    if (it == S->groups.end()) return;
    Group &g = *it->second;
    if (--g.live == 0) {
        if (g.has_dev) S->dev_arena->release(g.dev_off, g.dev_bytes);
        S->host_arena->release(g.host_off, g.host_bytes);
        S->groups.erase(it);
    }
}

void finish(pnuc_server *S, Request &r, State st, pnuc_status status)
{
    r.state = st;
    r.status = status;
    r.t_done = Clock::now();
    S->finished.push_back(r.ticket);
    if (S->finished.size() > 2 * S->reqs.size() + 64)  // drop released tickets (amortised)
        S->finished.erase(std::remove_if(S->finished.begin(), S->finished.end(),
                                         [&](uint64_t t) { return S->reqs.find(t) == S->reqs.end(); }),
                          S->finished.end());
    if (st == kDone) {
        S->completed++;
        S->events_done += r.n;
        S->latencies_ms.push_back(std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count());
        S->queue_ms.push_back(std::chrono::duration<double, std::milli>(r.t_admit - r.t_submit).count());
    } else {
        S->failed++;
        leave_group(S, r);
    }
}

// Admits the requests at the front of the queue as one group on a free stream; returns
// false if it must wait (no stream, or no room for even the first request).
bool admit(pnuc_server *S)
{
    int si = -1;
    for (size_t k = 0; k < S->streams.size(); ++k)
        if (S->stream_owner[k] == 0) {
            si = (int)k;
            break;
        }
    if (si < 0) return false;
    if (S->cfg.max_inflight_events) {  // the work in flight bounds new launches
        uint64_t inflight = 0;
        for (uint64_t gid : S->stream_owner) {
            auto it = gid ? S->groups.find(gid) : S->groups.end();
            if (it != S->groups.end()) inflight += it->second->n;
        }
        if (inflight >= S->cfg.max_inflight_events) return false;
    }
    // the candidates: the first pending request, then followers with the same seed
    std::vector<Request *> cand;
    uint64_t n = 0, cap = 0;
    for (uint64_t tk : S->pending) {
        auto it = S->reqs.find(tk);
        if (it == S->reqs.end()) break;  // the candidates are the first entries of the queue
        Request &r = *it->second;
        if (!cand.empty() && (r.solo || cand[0]->solo || r.seed != cand[0]->seed ||
                              (int)cand.size() >= std::min<int>(S->cfg.max_merge, kMaxSeg) ||
                              n + r.n > S->cfg.merge_events))
            break;
        cand.push_back(&r);
        n += r.n;
        cap += r.cap;
        if (r.solo) break;
    }
    if (cand.empty()) return false;
    // the largest prefix of the candidates that fits both arenas
    size_t doff = 0, hoff = 0;
    int k = (int)cand.size();
    for (; k >= 1; --k) {
        if (k < (int)cand.size()) {
            n -= cand[k]->n;
            cap -= cand[k]->cap;
        }
        GroupLayout L(n, cap, k);
        if (!S->dev_arena->alloc(L.dev_total, doff)) continue;
        if (!S->host_arena->alloc(L.host_total, hoff)) {
            S->dev_arena->release(doff, L.dev_total);
            continue;
        }
        break;
    }
    if (k < 1) return false;
    cand.resize(k);
    std::unique_ptr<Group> g(new Group());
    g->id = S->next_group++;
    g->n = n;
    g->cap = cap;
    GroupLayout L(n, cap, k);
    g->dev_off = doff;
    g->host_off = hoff;
    g->dev_bytes = L.dev_total;
    g->host_bytes = L.host_total;
    g->has_dev = true;
    g->stream = si;
    g->live = k;
    unsigned char *d = S->dev + doff, *h = S->host + hoff;
    // inputs and the segment tables, staged in the pinned arena (the header area of the host
    // region, then the device region's own input area)
    uint32_t *h_start = reinterpret_cast<uint32_t *>(h + GroupLayout::seg_start);
    unsigned long long *h_first = reinterpret_cast<unsigned long long *>(h + GroupLayout::seg_first);
    unsigned long long *h_cap = reinterpret_cast<unsigned long long *>(h + GroupLayout::cap_start);
    // the residual area of the host region stages the inputs until the results overwrite it
    // (in stream order): 13 bytes per event in a 64-byte record
    unsigned char *h_in = h + L.host_r;
    bool any_proj = false;
    for (int j = 0; j < k; ++j) any_proj = any_proj || !cand[j]->proj.empty();
    uint64_t pos = 0, cpos = 0;
    for (int j = 0; j < k; ++j) {
        Request &r = *cand[j];
        h_start[j] = (uint32_t)pos;
        h_first[j] = r.first;
        h_cap[j] = cpos;
        memcpy(h_in + 8 * pos, r.e.data(), 8 * r.n);
        memcpy(h_in + 8 * n + 4 * pos, r.t.data(), 4 * r.n);
        if (any_proj) {
            if (r.proj.empty()) memset(h_in + 12 * n + pos, 1, r.n);
            else memcpy(h_in + 12 * n + pos, r.proj.data(), r.n);
        }
        pos += r.n;
        cpos += r.cap;
        r.state = kRunning;
        r.group = g->id;
        if (r.reruns == 0) r.t_admit = Clock::now();
        g->tickets.push_back(r.ticket);
    }
    h_start[k] = (uint32_t)pos;
    h_cap[k] = cpos;
    for (int j = 0; j < k; ++j) S->pending.pop_front();
    cudaStream_t s = S->streams[si];
    pnuc_status st = PNUC_OK;
    const bool traced = S->tracing;
    unsigned char *hd = S->host_dev + hoff;  // the host region, as the kernels address it
    if (traced) {
        stamp_kernel<<<1, 32, 0, s>>>((unsigned long long *)(hd + GroupLayout::stamps));
        if (cudaGetLastError() != cudaSuccess) st = PNUC_ERR_CUDA;
    }
    static_assert(sizeof(pnuc_residual) >= 13, "inputs are staged in the residual area");
    if (st != PNUC_OK || cudaMemcpyAsync(d + L.e, h_in, 8 * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(d + L.t, h_in + 8 * n, 4 * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        (any_proj && cudaMemcpyAsync(d + L.pj, h_in + 12 * n, n, cudaMemcpyHostToDevice, s) != cudaSuccess) ||
        cudaMemcpyAsync(d + GroupLayout::seg_start, h + GroupLayout::seg_start,
                        GroupLayout::header - GroupLayout::seg_start, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(d + GroupLayout::seg_count, 0, 8 * kMaxSeg, s) != cudaSuccess)
        st = PNUC_ERR_CUDA;
    pnuc_batch b = {(const double *)(d + L.e), (const int32_t *)(d + L.t), n, cand[0]->seed, cand[0]->first,
                    any_proj ? (const uint8_t *)(d + L.pj) : nullptr, nullptr};
    pnuc_secondary *launch_sec = k > 1 ? (pnuc_secondary *)(d + L.s) : (pnuc_secondary *)(hd + L.host_s);
    pnuc_output o = {cap ? launch_sec : nullptr, cap, (unsigned long long *)(d + GroupLayout::count),
                     (pnuc_residual *)(hd + L.host_r), nullptr};
    Placement seg;
    {
        const uint64_t per_block = (uint64_t)S->ctx->tuning[tuning_slot(S->cfg.precision)].block_size * S->cfg.lane_events;
        seg.max_blocks = (unsigned)std::min<uint64_t>((n + per_block - 1) / per_block, 1u << 30);
    }
    if (k > 1) {
        seg.first = (const unsigned long long *)(d + GroupLayout::seg_first);
        seg.start = (const uint32_t *)(d + GroupLayout::seg_start);
        seg.n = k;
    }
    if (st == PNUC_OK)
        st = launch_batch(S->ctx, (pnuc_precision)S->cfg.precision, PNUC_PERSISTENT, &b, &o, s,
                          S->ctx->tuning[tuning_slot(S->cfg.precision)], nullptr, seg);
    if (st == PNUC_OK && k > 1 && cap) {
        const int grid = std::max(1, std::min<int>((int)((cap + 255) / 256), S->ctx->sm_count * 4));
        partition_kernel<<<grid, 256, 0, s>>>(
            (const uint4 *)(d + L.s), (const unsigned long long *)(d + GroupLayout::count), cap,
            (const uint32_t *)(d + GroupLayout::seg_start), (const unsigned long long *)(d + GroupLayout::cap_start),
            k, (unsigned long long *)(d + GroupLayout::seg_count), (uint4 *)(hd + L.host_s));
        if (cudaGetLastError() != cudaSuccess) st = PNUC_ERR_CUDA;
    }
    // the counts come back in stream order behind the kernels (the records are already in the
    // host region), so one completion event covers the whole group
    if (st == PNUC_OK && cudaMemcpyAsync(h, d, GroupLayout::seg_start, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        st = PNUC_ERR_CUDA;
    if (st == PNUC_OK && traced) {
        stamp_kernel<<<1, 32, 0, s>>>((unsigned long long *)(hd + GroupLayout::stamps + 8));
        if (cudaGetLastError() != cudaSuccess) st = PNUC_ERR_CUDA;
    }
    if (st == PNUC_OK && cudaEventRecord(S->events[si], s) != cudaSuccess) st = PNUC_ERR_CUDA;
    S->launches++;
    g->launch = S->launches;
    g->traced = traced;
    g->t_launched = Clock::now();
    const uint64_t gid = g->id;
    S->groups[gid] = std::move(g);
    if (st != PNUC_OK) {
        // copies may still be in flight into the group's regions: let them end before the
        // regions go back to the arenas
        cudaStreamSynchronize(s);
        for (Request *r : cand) finish(S, *r, kFailed, st);
        return true;
    }
    S->stream_owner[si] = gid;
    return true;
}

// The group on stream si is complete: hand each request its results, or send overflowing
// requests round again alone.
void complete(pnuc_server *S, Group &g)
{
    S->stream_owner[g.stream] = 0;
    const unsigned char *h = S->host + g.host_off;
    GroupLayout L(g.n, g.cap, (int)g.tickets.size());
    const unsigned long long launch_count = *(volatile const unsigned long long *)(h + GroupLayout::count);
    const unsigned long long *seg_count = (const unsigned long long *)(h + GroupLayout::seg_count);
    const uint32_t *seg_start = (const uint32_t *)(h + GroupLayout::seg_start);
    const unsigned long long *cap_start = (const unsigned long long *)(h + GroupLayout::cap_start);
    const bool single = g.tickets.size() == 1;  // no partition: the launch's count and records
    // the device region is no longer needed: results are in the host region
    S->dev_arena->release(g.dev_off, g.dev_bytes);
    g.has_dev = false;
    // When the launch itself dropped records (count above the group's reservation), every
    // per-request count is a lower bound only, so the whole group runs again.
    const bool dropped = launch_count > g.cap;
    const std::vector<uint64_t> tickets = g.tickets;  // the group may be freed in the loop
    std::vector<uint64_t> again;
    for (size_t j = 0; j < tickets.size(); ++j) {
        auto it = S->reqs.find(tickets[j]);
        if (it == S->reqs.end()) continue;
        Request &r = *it->second;
        const unsigned long long cnt = single ? launch_count : seg_count[j];
        if (dropped || cnt > r.cap) {
            // run again alone, with room for its count (exact unless the launch dropped records;
            // a lone run that drops records learns its exact count and runs once more)
            leave_group(S, r);
            r.solo = true;
            r.cap = std::max<uint64_t>(r.cap, cnt);
            if (!GroupLayout(r.n, r.cap, 1).fits(S->cfg.arena_bytes)) {
                finish(S, r, kFailed, PNUC_ERR_CAPACITY);
                continue;
            }
            r.reruns++;
            S->reruns++;
            r.state = kPending;
            again.push_back(r.ticket);
            continue;
        }
        r.count = cnt;
        r.res_view = (const pnuc_residual *)(h + L.host_r) + seg_start[j];
        r.sec_view = (const pnuc_secondary *)(h + L.host_s) + cap_start[j];
        if (S->tracing && g.traced) {
            r.tr.launch = g.launch;
            r.tr.stream = g.stream;
            r.tr.group_requests = (int32_t)tickets.size();
            r.tr.t_launched = trace_ms(S, g.t_launched);
            const volatile unsigned long long *ts = (const volatile unsigned long long *)(h + GroupLayout::stamps);
            r.tr.t_gpu_start = gpu_ms(S, ts[0]);
            r.tr.t_gpu_end = gpu_ms(S, ts[1]);
        }
        finish(S, r, kDone, PNUC_OK);
    }
    for (auto it = again.rbegin(); it != again.rend(); ++it) S->pending.push_front(*it);
}

void poll(pnuc_server *S, int si)
{
    auto it = S->groups.find(S->stream_owner[si]);
    if (it == S->groups.end()) {
        S->stream_owner[si] = 0;
        return;
    }
    cudaError_t q = cudaEventQuery(S->events[si]);
    if (q == cudaErrorNotReady) return;
    Group &g = *it->second;
    if (q != cudaSuccess) {
        S->stream_owner[si] = 0;
        std::vector<uint64_t> tickets = g.tickets;
        for (uint64_t tk : tickets) {
            auto rt = S->reqs.find(tk);
            if (rt != S->reqs.end()) finish(S, *rt->second, kFailed, PNUC_ERR_CUDA);
        }
        return;
    }
    complete(S, g);
}

void scheduler(pnuc_server *S)
{
    cudaSetDevice(S->ctx->cfg.device);
    std::unique_lock<std::mutex> lock(S->mu);
    while (true) {
        bool changed = false;
        for (size_t k = 0; k < S->streams.size(); ++k) {
            if (!S->stream_owner[k]) continue;
            const uint64_t before = S->stream_owner[k];
            poll(S, (int)k);
            changed = changed || S->stream_owner[k] != before;
        }
        while (!S->pending.empty()) {
            // drop tickets of requests that no longer exist
            if (S->reqs.find(S->pending.front()) == S->reqs.end()) {
                S->pending.pop_front();
                continue;
            }
            if (!admit(S)) break;
            changed = true;
        }
        if (changed) S->cv.notify_all();
        bool inflight = false;
        for (uint64_t g : S->stream_owner) inflight = inflight || g != 0;
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
    memset(cfg, 0, sizeof *cfg);
    cfg->precision = PNUC_FP32;
    cfg->streams = 8;
    cfg->arena_bytes = 1ull << 30;
    cfg->sec_per_event = 12;
    cfg->max_pending = 4096;
    cfg->max_request_events = 1ull << 24;
    cfg->max_merge = 32;
    cfg->merge_events = 1u << 18;
    cfg->lane_events = 4;
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
    if (S->epoch_word) cudaFreeHost(S->epoch_word);
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
    if (!valid_precision(cfg.precision) || cfg.streams < 1 || cfg.streams > 64 ||
        cfg.arena_bytes < (1u << 20) || cfg.sec_per_event < 1 || cfg.sec_per_event > 256 || cfg.max_pending < 1 ||
        cfg.max_request_events < 1 || cfg.max_merge < 1 || cfg.max_merge > (uint32_t)kMaxSeg || cfg.merge_events < 1 ||
        cfg.merge_events > kMaxGroupEvents || cfg.lane_events < 1 || cfg.lane_events > 1024)
        return fail(ctx, PNUC_ERR_ARG, "bad server configuration");
    if (cfg.precision == PNUC_FP32_SCALED && ctx->cfg.level_density != 0)
        return fail(ctx, PNUC_ERR_ARG, "the scaled FP32 widths need the Fermi-gas level density");
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
    void *hd = nullptr;
    if (cudaHostGetDevicePointer(&hd, S->host, 0) != cudaSuccess || !hd) {
        pnuc_server_destroy(S);
        return fail(ctx, PNUC_ERR_CUDA, "the pinned host arena is not mapped into the device's address space");
    }
    S->host_dev = static_cast<unsigned char *>(hd);
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
    return pnuc_server_submit_nucleons(S, energies, target_ids, nullptr, n, seed, first_event_id, ticket);
}

pnuc_status pnuc_server_submit_nucleons(pnuc_server *S, const double *energies, const int32_t *target_ids,
                                        const uint8_t *projectiles, uint64_t n, uint64_t seed,
                                        uint64_t first_event_id, uint64_t *ticket)
{
    if (!S || !ticket || (n > 0 && (!energies || !target_ids))) return PNUC_ERR_ARG;
    if (n == 0 || n > S->cfg.max_request_events)
        return fail(S->ctx, PNUC_ERR_ARG, "request of %llu events", (unsigned long long)n);
    uint64_t cap = n * S->cfg.sec_per_event;
    if (!GroupLayout(n, cap, 1).fits(S->cfg.arena_bytes))
        return fail(S->ctx, PNUC_ERR_ARG, "request of %llu events can never fit the %llu-byte arena",
                    (unsigned long long)n, (unsigned long long)S->cfg.arena_bytes);
    std::unique_ptr<Request> r(new Request());
    r->n = n;
    r->seed = seed;
    r->first = first_event_id;
    r->cap = cap;
    r->solo = n > kMaxGroupEvents;
    r->e.assign(energies, energies + n);
    r->t.assign(target_ids, target_ids + n);
    if (projectiles) r->proj.assign(projectiles, projectiles + n);
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

pnuc_status pnuc_server_wait_any(pnuc_server *S, int32_t timeout_ms, uint64_t *ticket)
{
    if (!S || !ticket) return PNUC_ERR_ARG;
    std::unique_lock<std::mutex> lock(S->mu);
    auto ready = [&] {
        while (!S->finished.empty() && S->reqs.find(S->finished.front()) == S->reqs.end())
            S->finished.pop_front();  // released already
        return !S->finished.empty();
    };
    if (timeout_ms < 0) S->cv.wait(lock, ready);
    else if (!S->cv.wait_for(lock, std::chrono::milliseconds(timeout_ms), ready)) return PNUC_ERR_TIMEOUT;
    *ticket = S->finished.front();
    S->finished.pop_front();
    return PNUC_OK;
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
    memcpy(residuals, r->res_view, sizeof(pnuc_residual) * r->n);
    if (r->count) memcpy(secondaries, r->sec_view, sizeof(pnuc_secondary) * r->count);
    record_release(S, *r);
    leave_group(S, *r);
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
    *residuals = r->res_view;
    *secondaries = r->sec_view;
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
    record_release(S, *r);
    leave_group(S, *r);
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
    out->arena_peak_bytes = std::max(S->dev_arena->peak(), S->host_arena->peak());
    out->launches = S->launches;
    return PNUC_OK;
}

pnuc_status pnuc_server_trace(pnuc_server *S, int32_t enable)
{
    if (!S) return PNUC_ERR_ARG;
    std::lock_guard<std::mutex> lock(S->mu);
    if (!enable) {
        S->tracing = false;
        return PNUC_OK;
    }
    CU(S->ctx, cudaSetDevice(S->ctx->cfg.device));
    if (!S->epoch_word)
        CU(S->ctx, cudaHostAlloc((void **)&S->epoch_word, 64, cudaHostAllocMapped));
    unsigned long long *word_dev = nullptr;
    CU(S->ctx, cudaHostGetDevicePointer((void **)&word_dev, S->epoch_word, 0));
    // the epoch: a stamp of the GPU's global timer on a stream with nothing before it, and the
    // host time halfway through its launch and synchronisation
    cudaStream_t s0 = S->streams[0];
    CU(S->ctx, cudaStreamSynchronize(s0));
    const Clock::time_point before = Clock::now();
    stamp_kernel<<<1, 32, 0, s0>>>(word_dev);
    CU(S->ctx, cudaGetLastError());
    CU(S->ctx, cudaStreamSynchronize(s0));
    const Clock::time_point after = Clock::now();
    S->gpu_epoch_ns = *(volatile unsigned long long *)S->epoch_word;
    S->t_epoch = before + (after - before) / 2;
    S->trace.clear();
    S->tracing = true;
    return PNUC_OK;
}

pnuc_status pnuc_server_trace_read(pnuc_server *S, pnuc_server_trace_entry *out, uint64_t capacity, uint64_t *count)
{
    if (!S || !count || (capacity && !out)) return PNUC_ERR_ARG;
    std::lock_guard<std::mutex> lock(S->mu);
    const uint64_t n = std::min<uint64_t>(capacity, S->trace.size());
    if (n) memcpy(out, S->trace.data(), n * sizeof(pnuc_server_trace_entry));
    *count = S->trace.size();
    return PNUC_OK;
}

pnuc_status pnuc_server_reset_stats(pnuc_server *S)
{
    if (!S) return PNUC_ERR_ARG;
    std::lock_guard<std::mutex> lock(S->mu);
    S->latencies_ms.clear();
    S->queue_ms.clear();
    S->completed = S->events_done = S->failed = S->reruns = S->launches = 0;
    S->t_start = Clock::now();
    return PNUC_OK;
}

}  // extern "C"
