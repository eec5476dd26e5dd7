// Host-side internals of libpnuc shared by the API translation units (api.cu,
// autotune.cu, graph.cu): the context object, error helpers and the launch routine.
#pragma once

#include <stdarg.h>
#include <stdio.h>

#include <vector>

#include "pnuc_internal.h"

namespace pnuc {
constexpr int kQueueSlots = 256;  // persistent launches of one context in flight at once
constexpr int kQueueStride = 16;  // 128-byte spacing between queue heads
inline bool valid_precision(int p) { return p == PNUC_FP32 || p == PNUC_FP64 || p == PNUC_FP32_SCALED; }
// The context's tuning slot of a precision: the two FP32 modes run the same cascade kernel
// and share one tuning.
inline int tuning_slot(int p) { return p == PNUC_FP64 ? 1 : 0; }
}  // namespace pnuc

struct pnuc_ctx {
    pnuc_config cfg;
    int sm_count = 0;
    char device_name[256] = {0};
    char err[512] = {0};
    double *mass = nullptr;              // [kMassZ * kMassA]
    double *cbrtA = nullptr;             // [kMassA]
    double *ct_table = nullptr;          // [kMassA * kCtStride] reading M26's constants
    double *qval = nullptr;              // [kMassZ * kMassA * kQStride] evaporation Q-values
    pnuc::TargetTable *tables = nullptr;  // [kMaxTargets]
    std::vector<std::pair<int, int>> targets;
    unsigned long long *queue = nullptr;  // [kQueueSlots * kQueueStride]
    unsigned queue_next = 0;
    pnuc_tuning tuning[2];  // [tuning_slot(precision)]
    // staging for pnuc_simulate_host
    double *h_energies = nullptr;
    int32_t *h_tids = nullptr;
    pnuc_residual *h_res = nullptr;
    uint64_t h_events_cap = 0, h_res_cap = 0;
    pnuc_secondary *h_sec = nullptr;
    uint64_t h_sec_cap = 0;
    unsigned long long *h_count = nullptr;
    unsigned long long *h_count_host = nullptr;  // pinned: the count read back
    // sorted method: particle stacks of every resident slot (grown as needed)
    void *sorted_stacks = nullptr;
    size_t sorted_stacks_bytes = 0;
    // pnuc_kernel_timing: three events per recorded launch
    bool timing = false;
    std::vector<cudaEvent_t> tev;
    std::vector<char> tev_two;  // per recorded launch: 1 if it ran two kernels
    size_t tev_used = 0;
};

namespace pnuc {

pnuc_status fail(pnuc_ctx *ctx, pnuc_status st, const char *fmt, ...);

#define CU(ctx, call)                                                                                       \
    do {                                                                                                    \
        cudaError_t e_ = (call);                                                                            \
        if (e_ != cudaSuccess)                                                                              \
            return ::pnuc::fail(ctx, PNUC_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                                __FILE__, __LINE__);                                                        \
    } while (0)

pnuc_status check_tuning(pnuc_ctx *ctx, const pnuc_tuning *t);
pnuc_status check_batch(pnuc_ctx *ctx, pnuc_precision precision, pnuc_method method, const pnuc_batch *batch,
                        const pnuc_output *out);
// Launch options of the serving loop: merged requests (device arrays; the SimParams fields
// seg_first, seg_start and n_seg) and a cap on each kernel's blocks (0: the resident limit),
// so that a launch leaves SMs to the launches beside it.
struct Placement {
    const unsigned long long *first = nullptr;
    const uint32_t *start = nullptr;
    int n = 0;
    unsigned max_blocks = 0;
};

// Enqueues the count reset, the queue-head reset and the kernel of one batch on stream s
// with tuning t. queue_head: the persistent kernel's queue head, or null for the next slot of
// the context's ring. seg: the launch's placement, if any.
pnuc_status launch_batch(pnuc_ctx *ctx, pnuc_precision precision, pnuc_method method, const pnuc_batch *batch,
                         const pnuc_output *out, cudaStream_t s, const pnuc_tuning &t,
                         unsigned long long *queue_head, const Placement &seg = Placement());

}  // namespace pnuc
