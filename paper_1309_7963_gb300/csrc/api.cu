// Host side of the libpnuc C ABI (include/pnuc.h): contexts, target tables, batch
// launches with device or host buffers, and launch tuning. All model arithmetic runs in
// the kernels (tables.cu, kernel_fp32.cu, kernel_fp64.cu); this file checks arguments,
// owns device-side tables and scratch, and orders the launches on the caller's stream.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

#include "api_internal.h"

namespace pnuc {

pnuc_status fail(pnuc_ctx *ctx, pnuc_status st, const char *fmt, ...)
{
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof ctx->err, fmt, ap);
        va_end(ap);
    }
    return st;
}

namespace {
bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// Resident blocks per SM of a kernel kind (0 cascade, 1 evaporation, 2 sorted cascade) for a
// precision, block size and counting variant. The runtime's occupancy query costs tens of
// microseconds, which small serving requests feel, so results are kept per process (they
// depend only on the compiled kernels and the device, one device per process here).
enum OccKind { kOccCascade = 0, kOccEvap = 1, kOccSorted = 2 };

int occupancy_kind(OccKind kind, pnuc_precision prec, int block, bool count, bool ct = false)
{
    static std::atomic<int> cache[3][3][4][2][2];
    static std::once_flag once;
    std::call_once(once, [] {
        for (auto &a : cache)
            for (auto &b : a)
                for (auto &c : b)
                    for (auto &d : c)
                        for (auto &e : d) e.store(-1);
    });
    const int bi = block == 64 ? 0 : block == 128 ? 1 : block == 256 ? 2 : 3;
    std::atomic<int> &slot =
        cache[kind][prec == PNUC_FP64 ? 1 : prec == PNUC_FP32_SCALED ? 2 : 0][bi][count ? 1 : 0][ct ? 1 : 0];
    int v = slot.load();
    if (v >= 0) return v;
    if (kind == kOccCascade)
        v = prec == PNUC_FP64 ? occupancy_persistent_fp64(block) : occupancy_persistent_fp32(block, count);
    else if (kind == kOccEvap)
        v = prec == PNUC_FP64 ? occupancy_evap_fp64(block, ct)
                              : occupancy_evap_fp32(block, count, prec == PNUC_FP32_SCALED, ct);
    else
        v = prec == PNUC_FP64 ? occupancy_sorted_fp64(block) : occupancy_sorted_fp32(block, count);
    slot.store(v);
    return v;
}

int occupancy(pnuc_precision prec, int block, bool count) { return occupancy_kind(kOccCascade, prec, block, count); }
}  // namespace

pnuc_status check_tuning(pnuc_ctx *ctx, const pnuc_tuning *t)
{
    if (!(t->block_size == 64 || t->block_size == 128 || t->block_size == 256 || t->block_size == 512))
        return fail(ctx, PNUC_ERR_ARG, "block_size %d not in {64,128,256,512}", t->block_size);
    if (t->blocks_per_sm < 1 || t->blocks_per_sm > 32)
        return fail(ctx, PNUC_ERR_ARG, "blocks_per_sm %d not in [1,32]", t->blocks_per_sm);
    if (t->refill_threshold < 1 || t->refill_threshold > 32)
        return fail(ctx, PNUC_ERR_ARG, "refill_threshold %d not in [1,32]", t->refill_threshold);
    if (t->chunk < 32 || t->chunk > (1 << 20))
        return fail(ctx, PNUC_ERR_ARG, "chunk %d not in [32, 2^20]", t->chunk);
    if (t->kin_batch < 1 || t->kin_batch > 32)
        return fail(ctx, PNUC_ERR_ARG, "kin_batch %d not in [1,32]", t->kin_batch);
    return PNUC_OK;
}

pnuc_status check_batch(pnuc_ctx *ctx, pnuc_precision precision, pnuc_method method, const pnuc_batch *batch,
                        const pnuc_output *out)
{
    if (!ctx || !batch || !out) return fail(ctx, PNUC_ERR_ARG, "null argument");
    if (!valid_precision(precision)) return fail(ctx, PNUC_ERR_ARG, "bad precision %d", precision);
    if (precision == PNUC_FP32_SCALED && ctx->cfg.level_density != 0)
        return fail(ctx, PNUC_ERR_ARG, "the scaled FP32 widths need the Fermi-gas level density");
    if (method != PNUC_PLAIN && method != PNUC_PERSISTENT && method != PNUC_SORTED)
        return fail(ctx, PNUC_ERR_ARG, "bad method %d", method);
    if (batch->n > 0xFFFFFFFFull) return fail(ctx, PNUC_ERR_ARG, "n = %llu exceeds 2^32-1", (unsigned long long)batch->n);
    if (!out->count) return fail(ctx, PNUC_ERR_ARG, "out->count is null");
    if (batch->n > 0 && (!batch->energies || !batch->target_ids || !out->residuals))
        return fail(ctx, PNUC_ERR_ARG, "null energies, target_ids or residuals");
    if (out->capacity > 0 && !out->secondaries) return fail(ctx, PNUC_ERR_ARG, "null secondaries with capacity > 0");
    if (!aligned16(out->secondaries) || !aligned16(out->residuals))
        return fail(ctx, PNUC_ERR_ARG, "secondaries and residuals must be 16-byte aligned");
    return PNUC_OK;
}

namespace {

constexpr size_t kMaxTimedLaunches = 4096;

// Three timing events for the next launch on s, or null when timing is off, the stream is
// being captured or the record is full.
cudaEvent_t *timing_slot(pnuc_ctx *ctx, cudaStream_t s)
{
    if (!ctx->timing) return nullptr;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return nullptr;
    if (ctx->tev_used + 3 > ctx->tev.size()) {
        if (ctx->tev.size() >= 3 * kMaxTimedLaunches) return nullptr;
        for (int k = 0; k < 3; ++k) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            ctx->tev.push_back(e);
        }
        ctx->tev_two.push_back(1);
    }
    ctx->tev_two[ctx->tev_used / 3] = 1;
    cudaEvent_t *ev = ctx->tev.data() + ctx->tev_used;
    ctx->tev_used += 3;
    return ev;
}

}  // namespace

// The evaporation kernel after a cascade kernel of the persistent or sorted method, on its
// own resident grid (it uses more registers, and its shared-memory job lists can make the
// block size too large: then it halves).
cudaError_t launch_evap_for(pnuc_ctx *ctx, pnuc_precision precision, const SimParams &p, const pnuc_tuning &t,
                            bool count, uint64_t n, cudaStream_t s, unsigned max_blocks)
{
    auto occ_evap = [&](int b) {
        return occupancy_kind(kOccEvap, precision, b, count, p.level_density == 1);
    };
    int eblock = t.block_size, occ_e = occ_evap(eblock);
    while (occ_e < 1 && eblock > 64) occ_e = occ_evap(eblock /= 2);
    const long long want = (long long)t.blocks_per_sm * t.block_size / eblock;
    unsigned long long egrid =
        (unsigned long long)std::max<long long>(std::min<long long>(want, occ_e), 1) * ctx->sm_count;
    const unsigned long long eneed = (n + eblock - 1) / eblock;
    if (egrid > eneed) egrid = eneed;
    if (max_blocks && egrid > max_blocks) egrid = max_blocks;
    return precision == PNUC_FP64 ? launch_evap_fp64(p, (int)egrid, eblock, s)
                                  : launch_evap_fp32(p, (int)egrid, eblock, count, precision == PNUC_FP32_SCALED, s);
}

pnuc_status launch_batch(pnuc_ctx *ctx, pnuc_precision precision, pnuc_method method, const pnuc_batch *batch,
                         const pnuc_output *out, cudaStream_t s, const pnuc_tuning &t, unsigned long long *queue_head,
                         const Placement &seg)
{
    CU(ctx, cudaSetDevice(ctx->cfg.device));
    // an error an earlier, failed runtime call left pending is not this launch's (errors of
    // earlier kernels that are sticky still show)
    (void)cudaGetLastError();
    CU(ctx, cudaMemsetAsync(out->count, 0, sizeof(unsigned long long), s));
    if (batch->n == 0) return PNUC_OK;
    SimParams p;
    p.energies = batch->energies;
    p.target_ids = batch->target_ids;
    p.projectiles = batch->projectiles;
    p.event_ids = reinterpret_cast<const unsigned long long *>(batch->event_ids);
    p.seg_first = seg.first;
    p.seg_start = seg.start;
    p.n_seg = seg.n;
    p.n = batch->n;
    p.seed = batch->seed;
    p.first_event_id = batch->first_event_id;
    p.sec = out->secondaries;
    p.sec_cap = out->secondaries ? out->capacity : 0;
    p.sec_count = out->count;
    p.res = out->residuals;
    p.counters = out->counters;
    p.tables = ctx->tables;
    p.n_targets = (int32_t)ctx->targets.size();
    p.mass = ctx->mass;
    p.cbrtA = ctx->cbrtA;
    p.ct_table = ctx->ct_table;
    p.qval = ctx->qval;
    p.max_steps = ctx->cfg.max_steps;
    p.max_attempts = ctx->cfg.max_attempts;
    p.max_evap_steps = ctx->cfg.max_evap_steps;
    p.max_evap_trials = ctx->cfg.max_evap_trials;
    p.level_density = ctx->cfg.level_density;
    p.refill_threshold = t.refill_threshold;
    p.chunk = t.chunk;
    p.kin_batch = t.kin_batch;
    p.queue_head = nullptr;
    p.evap_head = nullptr;
    p.split_evap = 0;
    const bool count = out->counters != nullptr;
    cudaEvent_t *ev = timing_slot(ctx, s);
    cudaError_t e = ev ? cudaEventRecord(ev[0], s) : cudaSuccess;
    if (e != cudaSuccess) ctx->tev_used -= 3;
    CU(ctx, e);
    if (method == PNUC_PLAIN) {
        e = precision == PNUC_FP64 ? launch_plain_fp64(p, t.block_size, s)
                                   : launch_plain_fp32(p, t.block_size, count, precision == PNUC_FP32_SCALED, s);
        if (e == cudaSuccess && ev) e = cudaEventRecord(ev[1], s);
        if (ev) ctx->tev_two[ctx->tev_used / 3 - 1] = 0;
    } else if (method == PNUC_SORTED) {
        int occ = occupancy_kind(kOccSorted, precision, t.block_size, count);
        if (occ < 1) return fail(ctx, PNUC_ERR_ARG, "sorted method: block size %d does not fit an SM", t.block_size);
        int bps = std::min(t.blocks_per_sm, occ);
        unsigned long long grid = (unsigned long long)bps * ctx->sm_count;
        unsigned long long need = (batch->n + t.block_size - 1) / t.block_size;
        if (grid > need) grid = need;
        const size_t per_slot = precision == PNUC_FP64 ? sorted_stack_bytes_fp64() : sorted_stack_bytes_fp32();
        const size_t bytes = (size_t)grid * t.block_size * per_slot;
        if (bytes > ctx->sorted_stacks_bytes) {
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
                return fail(ctx, PNUC_ERR_STATE, "sorted method: run one launch of this size before capturing it");
            const size_t want = (size_t)std::max(occ, t.blocks_per_sm) * ctx->sm_count * t.block_size * per_slot;
            CU(ctx, cudaStreamSynchronize(s));
            cudaFree(ctx->sorted_stacks);
            ctx->sorted_stacks = nullptr;
            ctx->sorted_stacks_bytes = 0;
            CU(ctx, cudaMalloc(&ctx->sorted_stacks, std::max(want, bytes)));
            ctx->sorted_stacks_bytes = std::max(want, bytes);
        }
        p.queue_head = queue_head ? queue_head : ctx->queue + (size_t)(ctx->queue_next++ % kQueueSlots) * kQueueStride;
        p.evap_head = p.queue_head + 1;
        p.split_evap = 1;
        CU(ctx, cudaMemsetAsync(p.queue_head, 0, 2 * sizeof(unsigned long long), s));
        e = precision == PNUC_FP64 ? launch_sorted_fp64(p, ctx->sorted_stacks, (int)grid, t.block_size, s)
                                   : launch_sorted_fp32(p, ctx->sorted_stacks, (int)grid, t.block_size, count, s);
        if (e == cudaSuccess && ev) e = cudaEventRecord(ev[1], s);
        e = e == cudaSuccess ? launch_evap_for(ctx, precision, p, t, count, batch->n, s, seg.max_blocks) : e;
    } else {
        int occ = occupancy(precision, t.block_size, count);
        int bps = std::min(t.blocks_per_sm, std::max(occ, 1));
        unsigned long long grid = (unsigned long long)bps * ctx->sm_count;
        unsigned long long need = (batch->n + t.block_size - 1) / t.block_size;
        if (grid > need) grid = need;
        if (seg.max_blocks && grid > seg.max_blocks) grid = seg.max_blocks;
        // queue slot: [0] the cascade kernel's queue head, [1] the evaporation kernel's
        p.queue_head = queue_head ? queue_head : ctx->queue + (size_t)(ctx->queue_next++ % kQueueSlots) * kQueueStride;
        p.evap_head = p.queue_head + 1;
        p.split_evap = 1;
        CU(ctx, cudaMemsetAsync(p.queue_head, 0, 2 * sizeof(unsigned long long), s));
        e = precision == PNUC_FP64 ? launch_persistent_fp64(p, (int)grid, t.block_size, s)
                                   : launch_persistent_fp32(p, (int)grid, t.block_size, count, s);
        if (e == cudaSuccess && ev) e = cudaEventRecord(ev[1], s);
        e = e == cudaSuccess ? launch_evap_for(ctx, precision, p, t, count, batch->n, s, seg.max_blocks) : e;
    }
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[2], s);
    if (e != cudaSuccess && ev) ctx->tev_used -= 3;  // the slot is the last one taken
    if (e != cudaSuccess) return fail(ctx, PNUC_ERR_CUDA, "kernel launch failed: %s", cudaGetErrorString(e));
    return PNUC_OK;
}

}  // namespace pnuc

using namespace pnuc;

extern "C" {

void pnuc_default_config(pnuc_config *cfg)
{
    if (!cfg) return;
    cfg->device = 0;
    cfg->max_steps = 100000;
    cfg->max_attempts = 1000;
    cfg->max_evap_steps = 64;
    cfg->max_evap_trials = 10000;
    cfg->level_density = 0;
}

const char *pnuc_status_string(pnuc_status s)
{
    switch (s) {
    case PNUC_OK: return "ok";
    case PNUC_ERR_ARG: return "invalid argument";
    case PNUC_ERR_RANGE: return "out of range";
    case PNUC_ERR_CAPACITY: return "capacity exceeded";
    case PNUC_ERR_CUDA: return "CUDA error";
    case PNUC_ERR_TIMEOUT: return "timeout";
    case PNUC_ERR_STATE: return "invalid state";
    }
    return "unknown status";
}

pnuc_status pnuc_last_error(const pnuc_ctx *ctx, char *buf, size_t len)
{
    if (!ctx || !buf || len == 0) return PNUC_ERR_ARG;
    snprintf(buf, len, "%s", ctx->err);
    return PNUC_OK;
}

pnuc_status pnuc_create(const pnuc_config *cfg_in, pnuc_ctx **out)
{
    if (!out) return PNUC_ERR_ARG;
    *out = nullptr;
    pnuc_config cfg;
    pnuc_default_config(&cfg);
    if (cfg_in) cfg = *cfg_in;
    if (cfg.max_steps < 1 || cfg.max_attempts < 1 || cfg.max_evap_steps < 1 || cfg.max_evap_trials < 1 ||
        (cfg.level_density != 0 && cfg.level_density != 1))
        return PNUC_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return PNUC_ERR_CUDA;
    if (cfg.device < 0 || cfg.device >= ndev) return PNUC_ERR_ARG;
    pnuc_ctx *ctx = new pnuc_ctx();
    ctx->cfg = cfg;
    pnuc_status st = PNUC_OK;
    do {
        if (cudaSetDevice(cfg.device) != cudaSuccess) { st = PNUC_ERR_CUDA; break; }
        cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, cfg.device);
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, cfg.device) == cudaSuccess)
            snprintf(ctx->device_name, sizeof ctx->device_name, "%s", prop.name);
        if (cudaMalloc(&ctx->mass, sizeof(double) * kMassZ * kMassA) != cudaSuccess ||
            cudaMalloc(&ctx->cbrtA, sizeof(double) * kMassA) != cudaSuccess ||
            cudaMalloc(&ctx->tables, sizeof(TargetTable) * kMaxTargets) != cudaSuccess ||
            cudaMalloc(&ctx->queue, sizeof(unsigned long long) * kQueueSlots * kQueueStride) != cudaSuccess ||
            cudaMalloc(&ctx->ct_table, sizeof(double) * kMassA * kCtStride) != cudaSuccess ||
            cudaMalloc(&ctx->qval, sizeof(double) * kMassZ * kMassA * kQStride) != cudaSuccess) {
            st = PNUC_ERR_CUDA;
            break;
        }
        if (launch_mass_table(ctx->mass, ctx->cbrtA, 0) != cudaSuccess || launch_ct_table(ctx->ct_table, 0) != cudaSuccess ||
            launch_q_table(ctx->qval, ctx->mass, 0) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
            st = PNUC_ERR_CUDA;
            break;
        }
        for (int p = 0; p < 2; ++p) {
            pnuc_tuning &t = ctx->tuning[p];
            t.block_size = 128;
            t.chunk = 256;
            t.kin_batch = 16;
            t.refill_threshold = 4;
            int occ = occupancy((pnuc_precision)p, t.block_size, false);
            t.blocks_per_sm = occ > 0 ? occ : 1;
        }
    } while (0);
    if (st != PNUC_OK) {
        pnuc_destroy(ctx);
        return st;
    }
    *out = ctx;
    return PNUC_OK;
}

pnuc_status pnuc_destroy(pnuc_ctx *ctx)
{
    if (!ctx) return PNUC_OK;
    cudaSetDevice(ctx->cfg.device);
    cudaFree(ctx->mass);
    cudaFree(ctx->cbrtA);
    cudaFree(ctx->ct_table);
    cudaFree(ctx->qval);
    cudaFree(ctx->tables);
    cudaFree(ctx->queue);
    cudaFree(ctx->h_energies);
    cudaFree(ctx->h_tids);
    cudaFree(ctx->h_res);
    cudaFree(ctx->h_sec);
    cudaFree(ctx->h_count);
    cudaFreeHost(ctx->h_count_host);
    for (cudaEvent_t e : ctx->tev) cudaEventDestroy(e);
    cudaFree(ctx->sorted_stacks);
    delete ctx;
    return PNUC_OK;
}

pnuc_status pnuc_create_target(pnuc_ctx *ctx, int32_t Z, int32_t A, int32_t *target_id)
{
    if (!ctx || !target_id) return fail(ctx, PNUC_ERR_ARG, "null argument");
    for (size_t k = 0; k < ctx->targets.size(); ++k)
        if (ctx->targets[k].first == Z && ctx->targets[k].second == A) {
            *target_id = (int32_t)k;
            return PNUC_OK;
        }
    if (A < 6 || A > 250 || Z < 2 || A - Z < 2 || Z > 100)
        return fail(ctx, PNUC_ERR_RANGE, "target Z=%d A=%d outside 6<=A<=250, 2<=Z<=100, A-Z>=2", Z, A);
    if ((int)ctx->targets.size() >= kMaxTargets)
        return fail(ctx, PNUC_ERR_CAPACITY, "at most %d targets per context", kMaxTargets);
    CU(ctx, cudaSetDevice(ctx->cfg.device));
    int id = (int)ctx->targets.size();
    CU(ctx, launch_target_table(ctx->tables + id, Z, A, ctx->mass, 0));
    CU(ctx, cudaDeviceSynchronize());
    int32_t valid = 0;
    CU(ctx, cudaMemcpy(&valid, &ctx->tables[id].valid, sizeof valid, cudaMemcpyDeviceToHost));
    if (!valid) return fail(ctx, PNUC_ERR_RANGE, "target Z=%d A=%d has a non-positive separation energy", Z, A);
    ctx->targets.push_back({Z, A});
    *target_id = id;
    return PNUC_OK;
}

pnuc_status pnuc_target_table(pnuc_ctx *ctx, int32_t target_id, pnuc_target_info *out)
{
    if (!ctx || !out) return fail(ctx, PNUC_ERR_ARG, "null argument");
    if (target_id < 0 || target_id >= (int)ctx->targets.size())
        return fail(ctx, PNUC_ERR_ARG, "unknown target id %d", target_id);
    CU(ctx, cudaSetDevice(ctx->cfg.device));
    TargetTable t;
    CU(ctx, cudaMemcpy(&t, ctx->tables + target_id, sizeof t, cudaMemcpyDeviceToHost));
    out->Z = t.Z;
    out->A = t.A;
    out->R = t.R;
    out->EC = t.d.EC;
    out->M = t.M;
    out->S_n = t.S[0];
    out->S_p = t.S[1];
    memcpy(out->r, t.d.r, sizeof out->r);
    memcpy(out->rho, t.d.rho, sizeof out->rho);
    memcpy(out->vF, t.d.vF, sizeof out->vF);
    memcpy(out->pF, t.d.pF, sizeof out->pF);
    memcpy(out->EF, t.d.EF, sizeof out->EF);
    memcpy(out->V, t.d.V, sizeof out->V);
    return PNUC_OK;
}

pnuc_status pnuc_get_tuning(const pnuc_ctx *ctx, pnuc_precision precision, pnuc_tuning *out)
{
    if (!ctx || !out || !valid_precision(precision)) return PNUC_ERR_ARG;
    *out = ctx->tuning[tuning_slot(precision)];
    return PNUC_OK;
}

pnuc_status pnuc_set_tuning(pnuc_ctx *ctx, pnuc_precision precision, const pnuc_tuning *t)
{
    if (!ctx || !t || !valid_precision(precision)) return fail(ctx, PNUC_ERR_ARG, "bad argument");
    pnuc_status st = check_tuning(ctx, t);
    if (st != PNUC_OK) return st;
    ctx->tuning[tuning_slot(precision)] = *t;
    return PNUC_OK;
}

pnuc_status pnuc_simulate(pnuc_ctx *ctx, pnuc_precision precision, pnuc_method method, const pnuc_batch *batch,
                          const pnuc_output *out, void *stream)
{
    pnuc_status st = check_batch(ctx, precision, method, batch, out);
    if (st != PNUC_OK) return st;
    return launch_batch(ctx, precision, method, batch, out, (cudaStream_t)stream, ctx->tuning[tuning_slot(precision)],
                        nullptr);
}

namespace {
constexpr bool kZeroCopySecondaries = true;
constexpr bool kZeroCopyResiduals = true;

// The device address of the host range [p, p + bytes) if all of it is pinned, mapped into
// the device's address space (one allocation) and 16-byte aligned, else null.
void *mapped_range(void *p, size_t bytes)
{
    if (!p || bytes == 0 || (reinterpret_cast<uintptr_t>(p) & 15)) return nullptr;
    cudaPointerAttributes a, b;
    const unsigned char *last = reinterpret_cast<const unsigned char *>(p) + bytes - 1;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess || cudaPointerGetAttributes(&b, last) != cudaSuccess) {
        cudaGetLastError();  // not a CUDA pointer: clear the error
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || b.type != cudaMemoryTypeHost || !a.devicePointer || !b.devicePointer)
        return nullptr;
    unsigned char *d = static_cast<unsigned char *>(a.devicePointer);
    if (static_cast<unsigned char *>(b.devicePointer) != d + (bytes - 1)) return nullptr;
    return d;
}
}  // namespace

pnuc_status pnuc_simulate_host(pnuc_ctx *ctx, pnuc_precision precision, pnuc_method method, const double *energies,
                               const int32_t *target_ids, uint64_t n, uint64_t seed, uint64_t first_event_id,
                               pnuc_secondary *secondaries, uint64_t sec_capacity, uint64_t *sec_count,
                               pnuc_residual *residuals, void *stream)
{
    if (!ctx || !sec_count) return fail(ctx, PNUC_ERR_ARG, "null argument");
    if (n > 0 && (!energies || !target_ids || !residuals)) return fail(ctx, PNUC_ERR_ARG, "null input/output");
    if (sec_capacity > 0 && !secondaries) return fail(ctx, PNUC_ERR_ARG, "null secondaries with capacity > 0");
    cudaStream_t s = (cudaStream_t)stream;
    CU(ctx, cudaSetDevice(ctx->cfg.device));
    // Output buffers in pinned host memory are written by the kernels themselves (mapped
    // memory over the chip-to-chip link; the kernels emit a few tens of GB/s), so no copy
    // follows the kernels; other buffers are staged on the device and copied back.
    pnuc_secondary *dsec = kZeroCopySecondaries ? static_cast<pnuc_secondary *>(
                                                      mapped_range(secondaries, sizeof(pnuc_secondary) * sec_capacity))
                                                : nullptr;
    pnuc_residual *dres =
        kZeroCopyResiduals ? static_cast<pnuc_residual *>(mapped_range(residuals, sizeof(pnuc_residual) * n)) : nullptr;
    if (n > ctx->h_events_cap || (!dres && n > ctx->h_res_cap)) {
        if (n > ctx->h_events_cap) {
            cudaFree(ctx->h_energies);
            cudaFree(ctx->h_tids);
            ctx->h_energies = nullptr;
            ctx->h_tids = nullptr;
            ctx->h_events_cap = 0;
            CU(ctx, cudaMalloc(&ctx->h_energies, sizeof(double) * n));
            CU(ctx, cudaMalloc(&ctx->h_tids, sizeof(int32_t) * n));
            ctx->h_events_cap = n;
        }
        if (!dres && n > ctx->h_res_cap) {
            cudaFree(ctx->h_res);
            ctx->h_res = nullptr;
            ctx->h_res_cap = 0;
            CU(ctx, cudaMalloc(&ctx->h_res, sizeof(pnuc_residual) * n));
            ctx->h_res_cap = n;
        }
    }
    if (!dsec && sec_capacity > ctx->h_sec_cap) {
        cudaFree(ctx->h_sec);
        ctx->h_sec = nullptr;
        ctx->h_sec_cap = 0;
        CU(ctx, cudaMalloc(&ctx->h_sec, sizeof(pnuc_secondary) * sec_capacity));
        ctx->h_sec_cap = sec_capacity;
    }
    if (!ctx->h_count) CU(ctx, cudaMalloc(&ctx->h_count, sizeof(unsigned long long)));
    if (!ctx->h_count_host) CU(ctx, cudaMallocHost(&ctx->h_count_host, sizeof(unsigned long long)));
    pnuc_batch b = {ctx->h_energies, ctx->h_tids, n, seed, first_event_id, nullptr, nullptr};
    pnuc_output o = {sec_capacity ? (dsec ? dsec : ctx->h_sec) : nullptr, sec_capacity, ctx->h_count,
                     dres ? dres : ctx->h_res, nullptr};
    pnuc_status st = check_batch(ctx, precision, method, &b, &o);
    if (st != PNUC_OK) return st;
    *sec_count = 0;
    if (n > 0) {
        CU(ctx, cudaMemcpyAsync(ctx->h_energies, energies, sizeof(double) * n, cudaMemcpyHostToDevice, s));
        CU(ctx, cudaMemcpyAsync(ctx->h_tids, target_ids, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    }
    st = launch_batch(ctx, precision, method, &b, &o, s, ctx->tuning[tuning_slot(precision)], nullptr);
    if (st != PNUC_OK) return st;
    CU(ctx, cudaMemcpyAsync(ctx->h_count_host, ctx->h_count, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    if (n > 0 && !dres)
        CU(ctx, cudaMemcpyAsync(residuals, ctx->h_res, sizeof(pnuc_residual) * n, cudaMemcpyDeviceToHost, s));
    CU(ctx, cudaStreamSynchronize(s));
    const unsigned long long cnt = *(volatile unsigned long long *)ctx->h_count_host;
    const uint64_t ncopy = cnt < sec_capacity ? cnt : sec_capacity;
    if (!dsec && ncopy > 0) {
        CU(ctx, cudaMemcpyAsync(secondaries, ctx->h_sec, sizeof(pnuc_secondary) * ncopy, cudaMemcpyDeviceToHost, s));
        CU(ctx, cudaStreamSynchronize(s));
    }
    *sec_count = cnt;
    if (cnt > sec_capacity)
        return fail(ctx, PNUC_ERR_CAPACITY, "batch produced %llu secondaries, capacity %llu", cnt,
                    (unsigned long long)sec_capacity);
    return PNUC_OK;
}

// ---------------------------------------------------------------- no-allocation entry point
// Device scratch of pnuc_simulate_host_noalloc: every GPU that loads this library holds
// these 8 MiB until the process exits. In host code the symbol is only a stand-in; the
// device address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[PNUC_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_noalloc_mu;
unsigned char *g_noalloc_ptr[64] = {nullptr};  // per device ordinal, set on first use

size_t round256(size_t b) { return (b + 255) / 256 * 256; }
}  // namespace

pnuc_status pnuc_simulate_host_noalloc(pnuc_ctx *ctx, pnuc_precision precision, pnuc_method method,
                                       const double *energies, const int32_t *target_ids, uint64_t n, uint64_t seed,
                                       uint64_t first_event_id, pnuc_secondary *secondaries, uint64_t sec_capacity,
                                       uint64_t *sec_count, pnuc_residual *residuals, void *stream)
{
    if (!ctx || !sec_count) return fail(ctx, PNUC_ERR_ARG, "null argument");
    if (n > 0 && (!energies || !target_ids || !residuals)) return fail(ctx, PNUC_ERR_ARG, "null input/output");
    if (sec_capacity > 0 && !secondaries) return fail(ctx, PNUC_ERR_ARG, "null secondaries with capacity > 0");
    if (method == PNUC_SORTED) return fail(ctx, PNUC_ERR_ARG, "the sorted method needs a context buffer");
    // outputs in pinned host memory are written in place (as in pnuc_simulate_host) and take
    // no scratch; scratch layout: [queue head | count], energies, target ids, residuals,
    // secondaries
    pnuc_secondary *zsec = static_cast<pnuc_secondary *>(mapped_range(secondaries, sizeof(pnuc_secondary) * sec_capacity));
    pnuc_residual *zres = static_cast<pnuc_residual *>(mapped_range(residuals, sizeof(pnuc_residual) * n));
    const size_t off_e = 256;
    const size_t off_t = off_e + round256(sizeof(double) * n);
    const size_t off_r = off_t + round256(sizeof(int32_t) * n);
    const size_t off_s = off_r + (zres ? 0 : round256(sizeof(pnuc_residual) * n));
    const size_t need = off_s + (zsec ? 0 : round256(sizeof(pnuc_secondary) * sec_capacity));
    if (n > PNUC_NOALLOC_SCRATCH_BYTES || sec_capacity > PNUC_NOALLOC_SCRATCH_BYTES || need > PNUC_NOALLOC_SCRATCH_BYTES)
        return fail(ctx, PNUC_ERR_CAPACITY,
                    "pnuc_simulate_host_noalloc: %llu events with room for %llu secondaries need %llu bytes of "
                    "device scratch; its static scratch holds %llu bytes (use pnuc_simulate_host for larger batches)",
                    (unsigned long long)n, (unsigned long long)sec_capacity, (unsigned long long)need,
                    (unsigned long long)PNUC_NOALLOC_SCRATCH_BYTES);
    const int dev = ctx->cfg.device;
    if (dev < 0 || dev >= 64) return fail(ctx, PNUC_ERR_ARG, "device %d outside the scratch table", dev);
    CU(ctx, cudaSetDevice(dev));
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void *ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess)
                return fail(ctx, PNUC_ERR_CUDA, "cudaGetSymbolAddress of the no-allocation scratch failed: %s",
                            cudaGetErrorString(e));
            g_noalloc_ptr[dev] = (unsigned char *)ptr;
        }
        base = g_noalloc_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *head = (unsigned long long *)base;
    unsigned long long *count = (unsigned long long *)(base + 128);
    double *d_e = (double *)(base + off_e);
    int32_t *d_t = (int32_t *)(base + off_t);
    pnuc_residual *d_r = zres ? zres : (pnuc_residual *)(base + off_r);
    pnuc_secondary *d_s = zsec ? zsec : (pnuc_secondary *)(base + off_s);
    // the scratch keeps the previous call's contents: the queue head and count restart at 0
    // (launch_batch clears both on the stream before the kernel)
    if (n > 0) {
        CU(ctx, cudaMemcpyAsync(d_e, energies, sizeof(double) * n, cudaMemcpyHostToDevice, s));
        CU(ctx, cudaMemcpyAsync(d_t, target_ids, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    }
    pnuc_batch b = {d_e, d_t, n, seed, first_event_id, nullptr, nullptr};
    pnuc_output o = {sec_capacity ? d_s : nullptr, sec_capacity, count, d_r, nullptr};
    pnuc_status st = check_batch(ctx, precision, method, &b, &o);
    if (st != PNUC_OK) return st;
    st = launch_batch(ctx, precision, method, &b, &o, s, ctx->tuning[tuning_slot(precision)], head);
    if (st != PNUC_OK) return st;
    unsigned long long cnt = 0;
    CU(ctx, cudaMemcpyAsync(&cnt, count, sizeof cnt, cudaMemcpyDeviceToHost, s));
    if (n > 0 && !zres) CU(ctx, cudaMemcpyAsync(residuals, d_r, sizeof(pnuc_residual) * n, cudaMemcpyDeviceToHost, s));
    CU(ctx, cudaStreamSynchronize(s));
    uint64_t ncopy = cnt < sec_capacity ? cnt : sec_capacity;
    if (ncopy > 0 && !zsec) {
        CU(ctx, cudaMemcpyAsync(secondaries, d_s, sizeof(pnuc_secondary) * ncopy, cudaMemcpyDeviceToHost, s));
        CU(ctx, cudaStreamSynchronize(s));
    }
    *sec_count = cnt;
    if (cnt > sec_capacity)
        return fail(ctx, PNUC_ERR_CAPACITY, "batch produced %llu secondaries, capacity %llu", cnt,
                    (unsigned long long)sec_capacity);
    return PNUC_OK;
}

pnuc_status pnuc_width_exp(pnuc_ctx *ctx, const float *x, double *out, uint64_t n, void *stream)
{
    if (!ctx || (n > 0 && (!x || !out))) return fail(ctx, PNUC_ERR_ARG, "null argument");
    CU(ctx, cudaSetDevice(ctx->cfg.device));
    CU(ctx, launch_width_exp(x, out, n, ctx->sm_count, (cudaStream_t)stream));
    return PNUC_OK;
}

pnuc_status pnuc_measure_peaks(pnuc_ctx *ctx, pnuc_peaks *out)
{
    if (!ctx || !out) return fail(ctx, PNUC_ERR_ARG, "null argument");
    CU(ctx, cudaSetDevice(ctx->cfg.device));
    double v[4];
    CU(ctx, measure_peaks(ctx->sm_count, v));
    out->fp32_fma = v[0];
    out->fp64_fma = v[1];
    out->mufu = v[2];
    out->int32_mad = v[3];
    return PNUC_OK;
}

pnuc_status pnuc_kernel_timing(pnuc_ctx *ctx, int32_t enable)
{
    if (!ctx) return fail(ctx, PNUC_ERR_ARG, "null argument");
    if (enable) ctx->tev_used = 0;
    ctx->timing = enable != 0;
    return PNUC_OK;
}

pnuc_status pnuc_kernel_times(pnuc_ctx *ctx, double *cascade_ms, double *evaporation_ms, uint64_t *launches)
{
    if (!ctx) return fail(ctx, PNUC_ERR_ARG, "null argument");
    CU(ctx, cudaSetDevice(ctx->cfg.device));
    double c = 0.0, v = 0.0;
    for (size_t i = 0; i + 2 < ctx->tev_used; i += 3) {
        CU(ctx, cudaEventSynchronize(ctx->tev[i + 2]));
        float a = 0.f, b = 0.f;
        CU(ctx, cudaEventElapsedTime(&a, ctx->tev[i], ctx->tev[i + 1]));
        if (ctx->tev_two[i / 3]) CU(ctx, cudaEventElapsedTime(&b, ctx->tev[i + 1], ctx->tev[i + 2]));
        c += a;
        v += b;
    }
    if (cascade_ms) *cascade_ms = c;
    if (evaporation_ms) *evaporation_ms = v;
    if (launches) *launches = ctx->tev_used / 3;
    return PNUC_OK;
}

}  // extern "C"
