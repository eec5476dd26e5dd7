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
    C.add(PNUC_C_DRAWS, 4u * L.rng.block - (unsigned)L.rng.left);  // generated minus unused
}

template <typename R, bool kCount>
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
            step<R, kCount>(P, sh, ts, L, stack, C);
        }
        finish_event<R, kCount>(P, L, C);
    }
    flush_counters<kCount>(P, cnt);
}

// Persistent kernel: grid = resident blocks only. Each warp keeps a reservoir
// [wnext, wend) of claimed event indices; when at least refill_threshold lanes are idle
// (or no lane is busy) the idle lanes take events from it, and the warp claims a new chunk
// with one atomicAdd on the queue head when it runs short.
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
    L.rng.buf = ring_base<R>(P, smem);
    L.rng.stride = blockDim.x;
    Particle<R> stack[kStackCap];
    unsigned long long wnext = 0, wend = 0;  // warp-uniform
    bool drained = false;                    // warp-uniform: the queue returned nothing
    const unsigned long long chunk = (unsigned long long)P.chunk;
    while (true) {
        if (L.phase == kFinish) {
            finish_event<R, kCount>(P, L, C);
            L.phase = kIdle;
        }
        const unsigned idle = __ballot_sync(FULL, L.phase == kIdle);
        const unsigned busy = __ballot_sync(FULL, L.phase == kEntry || L.phase == kTransport || L.phase == kEvap ||
                                                      L.phase == kKinWait);
        const int nidle = __popc(idle);
        if (nidle && (nidle >= P.refill_threshold || busy == 0 || drained)) {
            const unsigned rank = __popc(idle & ((1u << lane) - 1u));
            unsigned long long avail = wend - wnext;
            unsigned long long ev;
            if (avail >= (unsigned long long)nidle || drained) {
                ev = wnext + rank;
                wnext = avail >= (unsigned long long)nidle ? wnext + nidle : wend;
                if (rank >= avail) ev = ~0ull;
            } else {
                unsigned long long got = 0;
                if (lane == 0) got = atomicAdd(P.queue_head, chunk);
                got = __shfl_sync(FULL, got, 0);
                unsigned long long gend = got + chunk < P.n ? got + chunk : P.n;
                if (got >= P.n) {
                    drained = true;
                    gend = got;
                }
                ev = rank < avail ? wnext + rank : got + (rank - avail);
                if (rank >= avail && ev >= gend) ev = ~0ull;
                unsigned long long used_new = (unsigned long long)nidle - avail;
                wnext = got + used_new < gend ? got + used_new : gend;
                wend = gend;
            }
            if (L.phase == kIdle) {
                if (ev < P.n) begin_event<R>(P, ts, L, (uint32_t)ev);
                else L.phase = kExhausted;
            }
        }
        if (__all_sync(FULL, L.phase == kExhausted)) break;
        // FP64-heavy work (collision kinematics, evaporation steps) runs when enough lanes of
        // the warp need it, or when nothing else can progress, so that it executes with many
        // lanes active; the others keep transporting meanwhile.
        const unsigned run = __ballot_sync(FULL, L.phase == kEntry || L.phase == kTransport);
        const unsigned kin = __ballot_sync(FULL, L.phase == kKinWait);
        const unsigned evp = __ballot_sync(FULL, L.phase == kEvap);
        const bool do_kin = kin && (__popc(kin) >= P.kin_batch || run == 0);
        const bool do_evap = evp && (__popc(evp) >= P.evap_batch || (run == 0 && kin == 0));
        // the iteration's draws: at most 6 in a transport step, 3 in a collision, 2 at an
        // entry, 1 before the evaporation sampler (which ensures its own)
        if ((L.phase == kKinWait && do_kin) || (L.phase == kEvap && do_evap) || L.phase == kTransport ||
            L.phase == kEntry)
            L.rng.ensure(8);
        if (L.phase == kKinWait) {
            if (do_kin) finish_collision<R, kCount>(P, sh[L.tgt], ts[L.tgt], L, stack, C);
        } else if (L.phase == kEvap) {
            if (do_evap) step_evap<R, kCount>(P, L, C);
        } else if (L.phase == kTransport) {
            step_transport<R, kCount>(P, sh[L.tgt], ts[L.tgt], L, stack, C);
        } else if (L.phase == kEntry) {
            step_entry<R, kCount>(P, sh[L.tgt], ts[L.tgt].R, L, C);
        }
    }
    flush_counters<kCount>(P, cnt);
}

template <typename R, bool kCount>
__global__ void __launch_bounds__(512) persistent_kernel(const SimParams P)
{
    persistent_body<R, kCount>(P);
}

template <typename K>
cudaError_t allow_smem(K kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename R, bool kCount>
cudaError_t launch_plain(const SimParams &p, int block, cudaStream_t s)
{
    if (p.n == 0) return cudaSuccess;
    size_t smem = smem_bytes<R>(p.n_targets, block);
    cudaError_t e = allow_smem(plain_kernel<R, kCount>, smem);
    if (e != cudaSuccess) return e;
    unsigned long long grid = (p.n + block - 1) / block;
    plain_kernel<R, kCount><<<(unsigned)grid, block, smem, s>>>(p);
    return cudaGetLastError();
}

template <typename R, bool kCount>
cudaError_t launch_persistent(const SimParams &p, int grid, int block, cudaStream_t s)
{
    if (p.n == 0) return cudaSuccess;
    size_t smem = smem_bytes<R>(p.n_targets, block);
    cudaError_t e = allow_smem(persistent_kernel<R, kCount>, smem);
    if (e != cudaSuccess) return e;
    persistent_kernel<R, kCount><<<grid, block, smem, s>>>(p);
    return cudaGetLastError();
}

template <typename R, bool kCount>
int occupancy_persistent(int block)
{
    int nb = 0;
    allow_smem(persistent_kernel<R, kCount>, smem_bytes<R>(kMaxTargets, block));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, persistent_kernel<R, kCount>, block,
                                                  smem_bytes<R>(kMaxTargets, block));
    return nb;
}

}  // namespace
}  // namespace dev
}  // namespace pnuc
