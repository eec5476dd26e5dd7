// Event kernels (paper §3.2-3.3 re-designed for one GB300): the plain kernel runs one
// whole event per thread; the persistent kernel keeps every warp resident and refills
// lanes whose event finished from a device work queue (one atomic per chunk of events),
// so events of uneven length and mixed targets share a launch. Both write secondaries
// through warp-aggregated slot reservation (pnuc_device.cuh).
#pragma once

#include "pnuc_device.cuh"

namespace pnuc {
namespace dev {
namespace {  // internal linkage: each kernel translation unit has its own copy

// Copies the launch's target tables (precision R) and scalars into shared memory.
template <typename R>
__device__ void stage_tables(const SimParams &P, ShellTable<R> *sh, TargetScalars *ts)
{
    constexpr int words = sizeof(ShellTable<R>) / 4;
    for (int t = 0; t < P.n_targets; ++t) {
        const ShellTable<R> *src = sizeof(R) == 8 ? reinterpret_cast<const ShellTable<R> *>(&P.tables[t].d)
                                                  : reinterpret_cast<const ShellTable<R> *>(&P.tables[t].f);
        const uint32_t *s32 = reinterpret_cast<const uint32_t *>(src);
        uint32_t *d32 = reinterpret_cast<uint32_t *>(&sh[t]);
        for (int k = threadIdx.x; k < words; k += blockDim.x) d32[k] = __ldg(&s32[k]);
    }
    for (int t = threadIdx.x; t < P.n_targets; t += blockDim.x) {
        ts[t].M = P.tables[t].M;
        ts[t].R = P.tables[t].R;
        ts[t].Z = P.tables[t].Z;
        ts[t].A = P.tables[t].A;
    }
}

template <typename R>
__host__ __device__ constexpr size_t table_smem_bytes(int n_targets)
{
    return (size_t)n_targets * (sizeof(ShellTable<R>) + sizeof(TargetScalars));
}

// dynamic shared memory: target tables, then each thread's draw ring
template <typename R>
__host__ __device__ constexpr size_t smem_bytes(int n_targets, int block)
{
    return (table_smem_bytes<R>(n_targets) + 15) / 16 * 16 + (size_t)kRing * sizeof(R) * block;
}

// each thread's staging slot of the evaporation kernel's deferred emission (DeferredEmit)
constexpr size_t kStageBytes = 32;

// the persistent cascade kernel: tables and rings
template <typename R>
__host__ __device__ constexpr size_t persistent_smem_bytes(int n_targets, int block)
{
    return smem_bytes<R>(n_targets, block);
}

// the evaporation kernel, which reads no shell table: its rings, each warp's width-job list,
// then the staging slots (45.5 KB for 128-thread FP32 blocks: five blocks fit an SM, where a
// table region sized for the most targets left room for four)
template <typename R, bool kScaled = false>
__host__ __device__ constexpr size_t evap_smem_bytes(int n_targets, int block)
{
    return (size_t)kRing * sizeof(R) * block +
           (size_t)(block / 32) *
               (kWidthSlots * (sizeof(WidthJob<R>) + sizeof(width_t<R, kScaled>)) + 32 * sizeof(R)) +
           kStageBytes * block;
}

// the thread's deferred emitter on the staging slots at `at` ([2][blockDim.x] 16-byte halves)
__device__ __forceinline__ DeferredEmit deferred_emitter(unsigned char *at)
{
    DeferredEmit em;
    em.stage = reinterpret_cast<uint4 *>(at) + threadIdx.x;
    em.stride = (int)blockDim.x;
    em.base = 0;
    em.tag = 0;
    return em;
}

template <typename R>
__device__ __forceinline__ R *ring_base(const SimParams &P, unsigned char *smem)
{
    return reinterpret_cast<R *>(smem + (table_smem_bytes<R>(P.n_targets) + 15) / 16 * 16) + threadIdx.x;
}

template <bool kCount>
__device__ void flush_counters(const SimParams &P, unsigned long long *cnt)
{
    if (!kCount) return;
    __syncthreads();
    if (P.counters)
        for (int k = threadIdx.x; k < PNUC_N_COUNTERS; k += blockDim.x)
            if (cnt[k]) atomicAdd(&P.counters[k], cnt[k]);
}

template <typename R, bool kCount>
__device__ __forceinline__ void finish_event(const SimParams &P, Lane<R> &L, Counters<kCount> &C)
{
    write_residual(P, L);
    C.add(PNUC_C_DRAWS, L.rng.position());  // generated minus unused
    // events whose E* was settled here (a pending one is settled by the evaporation kernel)
    if (!L.pend && !(L.flags & (PNUC_FLAG_BAD_INPUT | PNUC_FLAG_ATTEMPT_CAP))) C.add(PNUC_C_SETTLED);
}

template <typename R, bool kCount, bool kScaled = false, bool kCT = false>
__global__ void __launch_bounds__(512) plain_kernel(const SimParams P)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long cnt[PNUC_N_COUNTERS];
    ShellTable<R> *sh = reinterpret_cast<ShellTable<R> *>(smem);
    TargetScalars *ts = reinterpret_cast<TargetScalars *>(smem + P.n_targets * sizeof(ShellTable<R>));
    stage_tables<R>(P, sh, ts);
    if (kCount)
        for (int k = threadIdx.x; k < PNUC_N_COUNTERS; k += blockDim.x) cnt[k] = 0;
    __syncthreads();
    Counters<kCount> C{cnt};
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < P.n) {
        Lane<R> L;
        Particle<R> stack[kStackCap];
        L.rng.buf = ring_base<R>(P, smem);
        L.rng.stride = blockDim.x;
        begin_event<R>(P, ts, L, (uint32_t)i);
        while (L.phase != kFinish) {
            L.rng.ensure(8);
            step<R, kScaled, kCT, kCount>(P, sh, ts, L, stack, C);
        }
        finish_event<R, kCount>(P, L, C);
    }
    flush_counters<kCount>(P, cnt);
}

// Warp-level reservoir [next, end) of claimed queue indices (warp-uniform state). take()
// gives every idle lane one index, or ~0 once the queue is exhausted, and claims new indices
// with one atomicAdd on the queue head when the reservoir runs short. Guided self-scheduling:
// a claim takes the remaining indices (as of the warp's last claim) over `share`, a multiple
// of 32 between 32 and `chunk`, so claims shrink as the queue drains and the launch ends
// about one event per lane after the queue, not one chunk per warp.
struct WarpQueue {
    unsigned long long next = 0, end = 0, seen = 0;
    bool drained = false;
    __device__ __forceinline__ unsigned long long take(unsigned idle, unsigned lane, unsigned long long *head,
                                                       unsigned long long n, unsigned long long chunk,
                                                       unsigned long long share)
    {
        const unsigned FULL = 0xffffffffu;
        const unsigned long long nidle = (unsigned long long)__popc(idle);
        const unsigned rank = __popc(idle & ((1u << lane) - 1u));
        const unsigned long long avail = end - next;
        unsigned long long ev;
        if (avail >= nidle || drained) {
            ev = rank < avail ? next + rank : ~0ull;
            next = avail >= nidle ? next + nidle : end;
            return ev;
        }
        unsigned long long c = seen < n ? ((n - seen) / share) & ~31ull : 32ull;
        c = c < 32ull ? 32ull : (c > chunk ? chunk : c);  // >= 32 >= nidle - avail
        unsigned long long got = 0;
        if (lane == 0) got = atomicAdd(head, c);
        got = __shfl_sync(FULL, got, 0);
        seen = got + c;
        unsigned long long gend = got + c < n ? got + c : n;
        if (got >= n) {
            drained = true;
            gend = got;
        }
        ev = rank < avail ? next + rank : got + (rank - avail);
        if (rank >= avail && ev >= gend) ev = ~0ull;
        const unsigned long long used_new = nidle - avail;
        next = got + used_new < gend ? got + used_new : gend;
        end = gend;
        return ev;
    }
};

// claims are sized for two per warp of the grid over what remains
__device__ __forceinline__ unsigned long long queue_share()
{
    return 2ull * gridDim.x * (blockDim.x >> 5);
}

// Persistent cascade kernel: grid = resident blocks only. When at least refill_threshold lanes
// of a warp are idle (or none is busy) they take events from the warp's queue reservoir.
// Accepted collisions wait until kin_batch lanes of the warp need their FP64 kinematics (or
// as many lanes wait as would run transport). Events with E* > 0 leave their evaporation
// pending in the residual record for evap_kernel.
template <typename R, bool kCount>
__device__ __forceinline__ void persistent_body(const SimParams &P)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long cnt[PNUC_N_COUNTERS];
    ShellTable<R> *sh = reinterpret_cast<ShellTable<R> *>(smem);
    TargetScalars *ts = reinterpret_cast<TargetScalars *>(smem + P.n_targets * sizeof(ShellTable<R>));
    stage_tables<R>(P, sh, ts);
    if (kCount)
        for (int k = threadIdx.x; k < PNUC_N_COUNTERS; k += blockDim.x) cnt[k] = 0;
    __syncthreads();
    Counters<kCount> C{cnt};
    const unsigned FULL = 0xffffffffu;
    const unsigned lane = threadIdx.x & 31;
    Lane<R> L;
    L.phase = kIdle;
    L.rng.reset(0, 0);
    L.rng.buf = ring_base<R>(P, smem);
    L.rng.stride = blockDim.x;
    Particle<R> stack[kStackCap];
    WarpQueue Q;
    // the cascade emits at once: deferred emission (as in the evaporation kernel) measured 2%
    // slower here, where it holds three more registers across the loop
    EmitNow em;
    const unsigned long long share = queue_share();
    while (true) {
        const long long t_top = kCount ? clock64() : 0;
        if (L.phase == kFinish) {
            finish_event<R, kCount>(P, L, C);
            L.phase = kIdle;
        }
        const unsigned idle = __ballot_sync(FULL, L.phase == kIdle);
        const unsigned busy = __ballot_sync(FULL, L.phase == kEntry || L.phase == kTransport || L.phase == kKinWait);
        const int nidle = __popc(idle);
        if (nidle && (nidle >= P.refill_threshold || busy == 0 || Q.drained)) {
            const unsigned long long ev = Q.take(idle, lane, P.queue_head, P.n, (unsigned long long)P.chunk, share);
            if (L.phase == kIdle) {
                if (ev < P.n) begin_event<R>(P, ts, L, (uint32_t)ev);
                else L.phase = kExhausted;
            }
        }
        if (__all_sync(FULL, L.phase == kExhausted)) break;
        const unsigned run = __ballot_sync(FULL, L.phase == kEntry || L.phase == kTransport);
        const unsigned kin = __ballot_sync(FULL, L.phase == kKinWait);
        // a batch runs once kin_batch lanes wait, or once no more lanes would run transport
        // than wait (a transport step with few lanes costs the warp as much as with many)
        const bool do_kin = kin && (__popc(kin) >= P.kin_batch || __popc(kin) >= __popc(run));
        // the iteration's draws: at most 6 in a transport step, 3 in a collision, 2 at an entry.
        // When a lane must generate, every other live lane with room for a block generates one
        // too, so the warp runs the Philox code less often and with more lanes (the words are
        // the same whenever they are made).
        const bool draws = (L.phase == kKinWait && do_kin) || L.phase == kTransport || L.phase == kEntry;
        if (__any_sync(FULL, draws && L.rng.left < 8)) {
            // only lanes holding an event touch their stream
            if (L.phase == kKinWait || L.phase == kTransport || L.phase == kEntry) {
                int k = draws ? 8 : 0;
                if (L.rng.left < kRing - kDrawsPerBlock + 1 && L.rng.left + 1 > k) k = L.rng.left + 1;
                L.rng.ensure(k);
            }
        }
        if (!kCount) {
            if (L.phase == kKinWait) {
                if (do_kin) finish_collision<R, kCount, true>(P, sh[L.tgt], ts[L.tgt], L, stack, C);
            } else if (L.phase == kTransport) {
                step_transport<R, kCount, true>(P, sh[L.tgt], ts[L.tgt], L, stack, C, em);
            } else if (L.phase == kEntry) {
                step_entry<R, kCount>(P, sh[L.tgt], ts[L.tgt].R, L, C);
            }
        } else {
            // the counting variant times each phase block of the warp (one lane records)
            const int ph = L.phase;
            long long t0 = clock64();
            if (ph == kKinWait && do_kin) finish_collision<R, kCount, true>(P, sh[L.tgt], ts[L.tgt], L, stack, C);
            __syncwarp();
            long long t1 = clock64();
            if (ph == kTransport) step_transport<R, kCount, true>(P, sh[L.tgt], ts[L.tgt], L, stack, C, em);
            else if (ph == kEntry) step_entry<R, kCount>(P, sh[L.tgt], ts[L.tgt].R, L, C);
            __syncwarp();
            long long t2 = clock64();
            if (lane == 0) {
                C.add(PNUC_C_CYCLES_COLLISION, (unsigned)(t1 - t0));
                C.add(PNUC_C_CYCLES_TRANSPORT, (unsigned)(t2 - t1));
                C.add(PNUC_C_CYCLES_REFILL, (unsigned)(t0 - t_top));
            }
        }
    }
    flush_counters<kCount>(P, cnt);
}

// Persistent evaporation kernel (after the cascade kernel on the same stream): every lane
// evaporates, so the width exponentials and the decays run with full warps. Lanes take
// event indices from the evaporation queue and skip events with nothing pending.
template <typename R, bool kCount, bool kScaled = false, bool kCT = false>
__device__ __forceinline__ void evap_body(const SimParams &P)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long cnt[PNUC_N_COUNTERS];
    if (kCount)
        for (int k = threadIdx.x; k < PNUC_N_COUNTERS; k += blockDim.x) cnt[k] = 0;
    __syncthreads();
    Counters<kCount> C{cnt};
    const unsigned FULL = 0xffffffffu;
    const unsigned lane = threadIdx.x & 31;
    Lane<R> L;
    L.phase = kIdle;
    L.rng.reset(0, 0);
    L.rng.buf = reinterpret_cast<R *>(smem) + threadIdx.x;  // the rings first (no tables here)
    L.rng.stride = blockDim.x;
    uint32_t d0 = 0;  // draw index at which the lane's evaporation resumed
    WarpQueue Q;
    const unsigned long long share = queue_share();
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    WidthJob<R> *jobs0 = reinterpret_cast<WidthJob<R> *>(smem + (size_t)kRing * sizeof(R) * blockDim.x);
    WidthJob<R> *jobs = jobs0 + warp * kWidthSlots;
    width_t<R, kScaled> *gw0 = reinterpret_cast<width_t<R, kScaled> *>(jobs0 + nwarps * kWidthSlots);
    width_t<R, kScaled> *gw = gw0 + warp * kWidthSlots;
    R *xms0 = reinterpret_cast<R *>(gw0 + nwarps * kWidthSlots);
    R *xms = xms0 + warp * 32;
    DeferredEmit em = deferred_emitter(reinterpret_cast<unsigned char *>(xms0 + nwarps * 32));
    while (true) {
        const long long t_top = kCount ? clock64() : 0;
        em.store(P, L.flags);  // the records of the last iteration's emissions
        if (L.phase == kFinish) {
            write_residual(P, L);
            C.add(PNUC_C_DRAWS, L.rng.position() - d0);
            L.phase = kIdle;
        }
        const unsigned idle = __ballot_sync(FULL, L.phase == kIdle);
        const int nidle = __popc(idle);
        const unsigned busy = __ballot_sync(FULL, L.phase == kEvap);
        if (nidle && (nidle >= P.refill_threshold || busy == 0 || Q.drained)) {
            const unsigned long long ev = Q.take(idle, lane, P.evap_head, P.n, (unsigned long long)P.chunk, share);
            if (L.phase == kIdle) {
                if (ev < P.n) {
                    begin_evap<R>(P, L, (uint32_t)ev);
                    d0 = L.rng.position();
                    if (L.phase != kIdle) C.add(PNUC_C_SETTLED);
                } else {
                    L.phase = kExhausted;
                }
            }
        }
        if (__all_sync(FULL, L.phase == kExhausted)) break;
        const long long t1 = kCount ? clock64() : 0;
        const bool stepping = L.phase == kEvap;
        if (stepping) L.rng.template ensure<true>(8);
        step_evap_warp<R, kScaled, kCT, kCount>(P, L, stepping, jobs, gw, xms, C, em);
        if (kCount) {
            __syncwarp();
            if (lane == 0) {
                C.add(PNUC_C_CYCLES_EVAPORATION, (unsigned)(clock64() - t1));
                C.add(PNUC_C_CYCLES_REFILL, (unsigned)(t1 - t_top));
            }
        }
    }
    flush_counters<kCount>(P, cnt);
}

// ------------------------------------------------------------------ sorted method
// The block holds blockDim.x events in flight ("slots"), their lane state in shared memory.
// Every iteration each busy slot takes one action (an entry, a transport step, its collision
// kinematics), with its draw ring topped up first if it runs short; the block counts the
// slots by (action, top-up) and its threads take them in that order, so that each warp runs
// one action, and the Philox blocks, with all its lanes. Candidate tests stay inside the
// transport step; accepted collisions wait one iteration and then run together, whatever
// warp their slots started in.
enum SortKey : int { kNoKey = -1, kKeyEntry = 0, kKeyTransport = 2, kKeyKin = 4, kKeys = 6 };

template <typename R>
__host__ __device__ constexpr size_t slot_bytes()
{
    // 16-byte units, an odd number of them (conflict-free 16-byte loads of neighbouring slots)
    return (((sizeof(Lane<R>) + 15) / 16) | 1) * 16;
}

template <typename R>
__host__ __device__ constexpr size_t sorted_smem_bytes(int n_targets, int block)
{
    return smem_bytes<R>(n_targets, block) + (size_t)block * slot_bytes<R>();
}

template <typename R, bool kCount>
__device__ __forceinline__ void sorted_body(const SimParams &P, Particle<R> *stacks)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long cnt[PNUC_N_COUNTERS];
    __shared__ int order[512];
    __shared__ int key_count[kKeys], key_fill[kKeys], key_off[kKeys + 1];
    __shared__ unsigned long long s_base;
    __shared__ int s_rank, s_drained;
    ShellTable<R> *sh = reinterpret_cast<ShellTable<R> *>(smem);
    TargetScalars *ts = reinterpret_cast<TargetScalars *>(smem + P.n_targets * sizeof(ShellTable<R>));
    stage_tables<R>(P, sh, ts);
    if (kCount)
        for (int k = threadIdx.x; k < PNUC_N_COUNTERS; k += blockDim.x) cnt[k] = 0;
    unsigned char *slot_base = smem + smem_bytes<R>(P.n_targets, blockDim.x);
    const int me = threadIdx.x;
    {
        Lane<R> &L0 = *reinterpret_cast<Lane<R> *>(slot_base + (size_t)me * slot_bytes<R>());
        L0.phase = kIdle;
        L0.rng.reset(0, 0);
        L0.rng.buf = ring_base<R>(P, smem);  // slot me's ring column
        L0.rng.stride = blockDim.x;
    }
    if (me == 0) s_drained = 0;
    __syncthreads();
    Counters<kCount> C{cnt};
    Particle<R> *my_stack_base = stacks + (size_t)blockIdx.x * blockDim.x * kStackCap;
    while (true) {
        // finished events leave; idle slots take new events (one queue atomic per round)
        Lane<R> &Lm = *reinterpret_cast<Lane<R> *>(slot_base + (size_t)me * slot_bytes<R>());
        if (Lm.phase == kFinish) {
            finish_event<R, kCount>(P, Lm, C);
            Lm.phase = kIdle;
        }
        const bool idle = Lm.phase == kIdle;
        const int nidle = __syncthreads_count(idle);
        const int nbusy = __syncthreads_count(Lm.phase == kEntry || Lm.phase == kTransport || Lm.phase == kKinWait);
        if (nidle && (nidle >= P.refill_threshold || nbusy == 0) && !s_drained) {
            if (me == 0) {
                s_base = atomicAdd(P.queue_head, (unsigned long long)nidle);
                s_rank = 0;
            }
            __syncthreads();
            if (idle) {
                const unsigned long long ev = s_base + (unsigned long long)atomicAdd(&s_rank, 1);
                if (ev < P.n) begin_event<R>(P, ts, Lm, (uint32_t)ev);
                else Lm.phase = kExhausted;
            }
            __syncthreads();
            if (me == 0 && s_base + nidle >= P.n) s_drained = 1;
        } else if (s_drained && idle) {
            Lm.phase = kExhausted;
        }
        if (__syncthreads_and(Lm.phase == kExhausted || Lm.phase == kIdle) &&
            __syncthreads_and(Lm.phase == kExhausted || s_drained))
            break;
        // accepted collisions wait until a full warp of them (or nothing else) is ready, so
        // that the FP64 kinematics run with all lanes and not in every iteration
        const int nkin = __syncthreads_count(Lm.phase == kKinWait);
        const int nrun = __syncthreads_count(Lm.phase == kEntry || Lm.phase == kTransport);
        const bool kin_now = nkin >= 32 || nrun == 0;
        // sort the busy slots by (action, top-up)
        int key = kNoKey;
        if (Lm.phase == kEntry) key = kKeyEntry;
        else if (Lm.phase == kTransport) key = kKeyTransport;
        else if (Lm.phase == kKinWait && kin_now) key = kKeyKin;
        if (key != kNoKey && Lm.rng.left < 8) key += 1;
        if (me < kKeys) {
            key_count[me] = 0;
            key_fill[me] = 0;
        }
        __syncthreads();
        if (key != kNoKey) atomicAdd(&key_count[key], 1);
        __syncthreads();
        if (me == 0) {
            int o = 0;
            for (int k = 0; k < kKeys; ++k) {
                key_off[k] = o;
                o += key_count[k];
            }
            key_off[kKeys] = o;
        }
        __syncthreads();
        if (key != kNoKey) order[key_off[key] + atomicAdd(&key_fill[key], 1)] = me;
        __syncthreads();
        // each thread takes one slot of the sorted list
        if (me < key_off[kKeys]) {
            const int slot = order[me];
            Lane<R> *lp = reinterpret_cast<Lane<R> *>(slot_base + (size_t)slot * slot_bytes<R>());
            Lane<R> L = *lp;
            Particle<R> *stack = my_stack_base + (size_t)slot * kStackCap;
            if (L.rng.left < 8) L.rng.ensure(8);
            if (L.phase == kKinWait) finish_collision<R, kCount, true>(P, sh[L.tgt], ts[L.tgt], L, stack, C);
            else if (L.phase == kTransport) {
                EmitNow em;
                step_transport<R, kCount, true>(P, sh[L.tgt], ts[L.tgt], L, stack, C, em);
            }
            else if (L.phase == kEntry) step_entry<R, kCount>(P, sh[L.tgt], ts[L.tgt].R, L, C);
            *lp = L;
        }
        __syncthreads();
    }
    flush_counters<kCount>(P, cnt);
}

template <typename R, bool kCount>
__global__ void __launch_bounds__(512) sorted_kernel(const SimParams P, Particle<R> *stacks)
{
    sorted_body<R, kCount>(P, stacks);
}

template <typename K>
cudaError_t allow_smem(K kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename R, bool kCount>
__global__ void __launch_bounds__(512) persistent_kernel(const SimParams P)
{
    persistent_body<R, kCount>(P);
}

template <typename R, bool kCount, bool kScaled = false, bool kCT = false>
__global__ void __launch_bounds__(512) evap_kernel(const SimParams P)
{
    evap_body<R, kCount, kScaled, kCT>(P);
}

template <typename R, bool kCount, bool kScaled = false, bool kCT = false>
cudaError_t launch_evap(const SimParams &p, int grid, int block, cudaStream_t s)
{
    if (p.n == 0) return cudaSuccess;
    size_t smem = evap_smem_bytes<R, kScaled>(p.n_targets, block);
    cudaError_t e = allow_smem(evap_kernel<R, kCount, kScaled, kCT>, smem);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();  // leave no error pending for the next launch's check
        return e;
    }
    evap_kernel<R, kCount, kScaled, kCT><<<grid, block, smem, s>>>(p);
    return cudaGetLastError();
}

template <typename R, bool kCount, bool kScaled = false, bool kCT = false>
cudaError_t launch_plain(const SimParams &p, int block, cudaStream_t s)
{
    if (p.n == 0) return cudaSuccess;
    size_t smem = smem_bytes<R>(p.n_targets, block);
    cudaError_t e = allow_smem(plain_kernel<R, kCount, kScaled, kCT>, smem);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();  // leave no error pending for the next launch's check
        return e;
    }
    unsigned long long grid = (p.n + block - 1) / block;
    plain_kernel<R, kCount, kScaled, kCT><<<(unsigned)grid, block, smem, s>>>(p);
    return cudaGetLastError();
}

template <typename R, bool kCount>
cudaError_t launch_persistent(const SimParams &p, int grid, int block, cudaStream_t s)
{
    if (p.n == 0) return cudaSuccess;
    size_t smem = persistent_smem_bytes<R>(p.n_targets, block);
    cudaError_t e = allow_smem(persistent_kernel<R, kCount>, smem);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();  // leave no error pending for the next launch's check
        return e;
    }
    persistent_kernel<R, kCount><<<grid, block, smem, s>>>(p);
    return cudaGetLastError();
}

template <typename R, bool kCount>
cudaError_t launch_sorted(const SimParams &p, void *stacks, int grid, int block, cudaStream_t s)
{
    if (p.n == 0) return cudaSuccess;
    size_t smem = sorted_smem_bytes<R>(p.n_targets, block);
    cudaError_t e = allow_smem(sorted_kernel<R, kCount>, smem);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();  // leave no error pending for the next launch's check
        return e;
    }
    sorted_kernel<R, kCount><<<grid, block, smem, s>>>(p, static_cast<Particle<R> *>(stacks));
    return cudaGetLastError();
}

template <typename K>
cudaError_t launch_kernel(K kernel, size_t smem, const SimParams &p, int grid, int block, cudaStream_t s)
{
    if (p.n == 0) return cudaSuccess;
    cudaError_t e = allow_smem(kernel, smem);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();  // leave no error pending for the next launch's check
        return e;
    }
    kernel<<<grid, block, smem, s>>>(p);
    return cudaGetLastError();
}

// Resident blocks per SM of `kernel` at a block size and dynamic shared memory, 0 when it does
// not fit. A query that fails (shared memory beyond what a block can have) leaves no error
// pending, so the next launch's cudaGetLastError() does not report it.
template <typename K>
int occupancy_of(K kernel, size_t smem, int block)
{
    int nb = 0;
    if (allow_smem(kernel, smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, block, smem) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return nb;
}

template <typename R, bool kCount>
int occupancy_sorted(int block)
{
    return occupancy_of(sorted_kernel<R, kCount>, sorted_smem_bytes<R>(kMaxTargets, block), block);
}

template <typename R, bool kCount, bool kScaled = false, bool kCT = false>
int occupancy_evap(int block)
{
    return occupancy_of(evap_kernel<R, kCount, kScaled, kCT>, evap_smem_bytes<R, kScaled>(kMaxTargets, block),
                        block);
}

template <typename R, bool kCount>
int occupancy_persistent(int block)
{
    return occupancy_of(persistent_kernel<R, kCount>, persistent_smem_bytes<R>(kMaxTargets, block), block);
}

}  // namespace
}  // namespace dev
}  // namespace pnuc
