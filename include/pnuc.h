/*
 * pnuc.h — C ABI of libpnuc: event-parallel Monte Carlo of non-elastic proton–nucleus
 * interactions (20–250 MeV) on one GB300 GPU, after arXiv:1309.7963.
 *
 * One event = one incident proton (or, as an extension, a neutron: pnuc_batch.projectiles)
 * on one target nucleus: an intranuclear cascade
 * (paper §2.3) on a 15-shell Fermi-gas nucleus (§2.2, Eq. 1), then evaporation of
 * n, p, d, t, 3He and alpha down to the residual nucleus (§2.4). Every event depends only
 * on (seed, event id): its random numbers are the stream of Philox4x64-10 with key
 * (seed, 0) and counters (j, event id, 0, 0), j = 0, 1, ..., each 64-bit word giving two
 * 32-bit draws, the high half first (the paper used CURAND states, §3.1).
 *
 * Conventions for every entry point:
 *  - Pointers documented "device" must point to memory of the context's device (for
 *    example tensors allocated by PyTorch); "host" pointers to host memory. The caller
 *    owns all buffers it passes; the library never frees them.
 *  - Functions return pnuc_status; PNUC_OK is 0. On error nothing is launched and
 *    pnuc_last_error() gives a message. Argument checks happen on the host before any
 *    launch.
 *  - Launches are asynchronous on the caller's CUDA stream (cudaStream_t passed as
 *    void*; NULL = the legacy default stream). Results are valid after that stream is
 *    synchronised. A context is not thread-safe: use one context per host thread.
 *  - Units: MeV, MeV/c, fm.
 */
#ifndef PNUC_H
#define PNUC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PNUC_OK = 0,
    PNUC_ERR_ARG = 1,      /* null pointer, bad enum, misaligned buffer, n too large */
    PNUC_ERR_RANGE = 2,    /* (Z, A) outside the supported nuclei */
    PNUC_ERR_CAPACITY = 3, /* a fixed-size resource is full (targets, output) */
    PNUC_ERR_CUDA = 4,     /* a CUDA runtime call failed; see pnuc_last_error() */
    PNUC_ERR_TIMEOUT = 5,  /* a bounded wait ran out */
    PNUC_ERR_STATE = 6     /* call not valid in the object's current state */
} pnuc_status;

typedef enum {
    PNUC_FP32 = 0,        /* bulk transport, path and cross-section arithmetic, the evaporation
                             channel parameters, emission sampler and decay in FP32; the NN
                             collision boosts to and from the pair's CM frame, the event's
                             energy/momentum bookkeeping (with the Q-values) and the evaporation
                             widths with their exponentials (§2.4) in FP64 */
    PNUC_FP64 = 1,        /* everything in FP64, no fused multiply-add: reproduces the CPU
                             oracle event by event up to libm rounding */
    PNUC_FP32_SCALED = 2  /* PNUC_FP32 with the evaporation widths and the channel draw in FP32:
                             each width of an evaporation step is evaluated times e^-xm, xm the
                             largest exponent of the step's open channels (the draw needs only
                             the widths' ratios; unscaled they reach e^160, beyond FP32). Shares
                             PNUC_FP32's tuning */
} pnuc_precision;

typedef enum {
    PNUC_PLAIN = 0,     /* one event per thread, one launch of n threads */
    PNUC_PERSISTENT = 1, /* two launches of resident warps that refill finished lanes from device
                            queues: the cascades, then the evaporations they leave pending */
    PNUC_SORTED = 2      /* as PNUC_PERSISTENT, but the cascade kernel keeps its blocks' events in
                            shared memory and regroups them by next action every iteration (each
                            warp runs one action with all its lanes); needs a context buffer for
                            the events' particle stacks, allocated at the first sorted launch
                            (which must not be inside a stream capture) */
} pnuc_method;

/* Secondary particle record, 32 bytes, 16-byte aligned array. */
typedef struct {
    uint32_t event;   /* index of the event in its batch (0 .. n-1) */
    uint8_t species;  /* 0 n, 1 p, 2 d, 3 t, 4 3He, 5 alpha */
    uint8_t origin;   /* 0 escaped from the cascade, 1 evaporated */
    uint16_t index;   /* emission order within the event: cascade escapes, then evaporation */
    double T;         /* lab kinetic energy, MeV */
    float ux, uy, uz; /* lab direction (unit vector); the beam is along +z */
    uint32_t reserved;
} pnuc_secondary;

/* Per-event residual record, 64 bytes. */
typedef struct {
    uint16_t Z_cascade, A_cascade; /* residual after the cascade */
    uint16_t Z_final, A_final;     /* residual after evaporation */
    uint16_t n_cascade;            /* secondaries escaped from the cascade */
    uint16_t n_evaporated;         /* particles evaporated */
    uint16_t n_collisions;         /* accepted (not Pauli-blocked) NN collisions */
    uint16_t n_attempts;           /* entries drawn until the event was non-elastic */
    uint32_t flags;                /* PNUC_FLAG_* */
    uint32_t reserved;
    double Estar_cascade;  /* excitation energy after the cascade (energy balance), MeV */
    double Estar_final;    /* excitation left on the final residual, MeV */
    float P_cascade[3];    /* momentum the static mean field took during the cascade, MeV/c */
    float P_final[3];      /* recoil momentum of the final residual from evaporation, MeV/c */
} pnuc_residual;

#define PNUC_FLAG_BAD_INPUT 1u         /* energy outside [20, 250] MeV, unknown target id or projectile */
#define PNUC_FLAG_ATTEMPT_CAP 2u       /* no non-elastic entry within max_attempts */
#define PNUC_FLAG_STEP_CAP 4u          /* max_steps transport steps; particles in flight captured */
#define PNUC_FLAG_STACK_OVERFLOW 8u    /* particle stack full; the particle was captured */
#define PNUC_FLAG_BAD_RESIDUAL 16u     /* residual with Z < 1 or N < 1: no evaporation */
#define PNUC_FLAG_NO_EXCITATION 32u    /* E* <= 0 after the cascade: no evaporation */
#define PNUC_FLAG_EVAP_TRIAL_CAP 64u   /* emission-energy sampling gave up; evaporation stopped */
#define PNUC_FLAG_EVAP_STEP_CAP 128u   /* max evaporation steps reached */
#define PNUC_FLAG_OUTPUT_OVERFLOW 256u /* a secondary of this event did not fit the output */

/* Work counters (optional output), summed over a batch. */
enum {
    PNUC_C_STEPS = 0, PNUC_C_CANDIDATES, PNUC_C_KINEMATICS, PNUC_C_PAULI_BLOCKED, PNUC_C_COLLISIONS,
    PNUC_C_CROSSINGS, PNUC_C_REFLECTIONS, PNUC_C_ESCAPES, PNUC_C_CAPTURES, PNUC_C_ATTEMPTS,
    PNUC_C_EVAP_STEPS, PNUC_C_EVAP_TRIALS, PNUC_C_DRAWS,
    /* E* settlements (events whose cascade ended), six-channel width evaluations, and the
     * open channels among them evaluated with the exponential (x >= 1) or the series (x < 1) */
    PNUC_C_SETTLED, PNUC_C_EVAP_PASSES, PNUC_C_EVAP_EXPS, PNUC_C_EVAP_SERIES,
    /* persistent method only: SM clock cycles its warps spent in each phase of the loop
     * (summed over warps), the counterpart of the paper's kernel time split (§4.2) */
    PNUC_C_CYCLES_TRANSPORT, PNUC_C_CYCLES_COLLISION, PNUC_C_CYCLES_EVAPORATION, PNUC_C_CYCLES_REFILL,
    PNUC_N_COUNTERS
};

typedef struct {
    int32_t device;            /* CUDA device ordinal */
    int32_t max_steps;         /* transport steps per event (default 100000) */
    int32_t max_attempts;      /* entries per event until non-elastic (default 1000) */
    int32_t max_evap_steps;    /* evaporation steps per event (default 64) */
    int32_t max_evap_trials;   /* rejection trials per emission (default 10000) */
    int32_t level_density;     /* the daughters' level density in the evaporation (§2.4): 0 (default) the
                                  Fermi gas exp(2 sqrt(a U)), a = A/8; 1 the composite form of GEM after
                                  Gilbert and Cameron, constant temperature below U_x = 2.5 + 150/A MeV,
                                  joined to the Fermi gas in value and slope at U_x (not with
                                  PNUC_FP32_SCALED: PNUC_ERR_ARG) */
} pnuc_config;

/* One batch of incident nucleons. */
typedef struct {
    const double *energies;    /* device, n entries: incident kinetic energy, MeV */
    const int32_t *target_ids; /* device, n entries: ids from pnuc_create_target */
    uint64_t n;                /* events; at most 2^32 - 1 */
    uint64_t seed;             /* Philox key word 0 */
    uint64_t first_event_id;   /* event i of the batch has id first_event_id + i */
    const uint8_t *projectiles; /* device, n entries: incident nucleon, 1 proton, 0 neutron
                                  (other values: PNUC_FLAG_BAD_INPUT); NULL = all protons.
                                  Neutron-induced events take the neutron's mass and the
                                  neutron well at entry, and the residual keeps the target's
                                  charge (an extension of the paper's proton-induced model) */
    const uint64_t *event_ids;  /* device, n entries: the id of each event, in place of
                                  first_event_id + i; NULL = first_event_id + i. Ids may repeat:
                                  a batch of one repeated id runs one event on every lane, the
                                  divergence-free bound of the paper's same-seed experiment (§3) */
} pnuc_batch;

/* Where a batch's results go. */
typedef struct {
    pnuc_secondary *secondaries; /* device, capacity records, 16-byte aligned */
    uint64_t capacity;
    unsigned long long *count;   /* device, 1 entry: set to the number of secondaries the
                                    batch produced, which may exceed capacity; records past
                                    capacity are dropped and their events flagged
                                    PNUC_FLAG_OUTPUT_OVERFLOW */
    pnuc_residual *residuals;    /* device, n records (entry i = event i) */
    unsigned long long *counters;/* device, PNUC_N_COUNTERS entries added to, or NULL */
} pnuc_output;

/* Launch tuning of the persistent method (the plain method uses block_size only). None of
 * these changes any event's result, only the order in which lanes do their work. */
typedef struct {
    int32_t block_size;       /* threads per block: 64, 128, 256 or 512 */
    int32_t blocks_per_sm;    /* resident blocks per SM for the persistent grid (<= occupancy) */
    int32_t refill_threshold; /* a warp refills when at least this many lanes are idle (1..32) */
    int32_t chunk;            /* most events a warp takes from the queue per atomic (32 .. 2^20); claims
                                 shrink towards 32 as the queue drains */
    int32_t kin_batch;        /* accepted collisions a warp gathers before their FP64 kinematics (1..32);
                                 a batch also runs once as many lanes wait as would run transport */
} pnuc_tuning;

typedef struct pnuc_ctx pnuc_ctx;

/* Fills *cfg with the defaults. */
void pnuc_default_config(pnuc_config *cfg);

/* Creates a context on cfg->device (cfg may be NULL for defaults): builds the nuclide mass
 * table on the device (semi-empirical masses, §2.2). *out receives the context. */
pnuc_status pnuc_create(const pnuc_config *cfg, pnuc_ctx **out);

/* Releases the context and its device memory. Safe on NULL. */
pnuc_status pnuc_destroy(pnuc_ctx *ctx);

/* Human-readable name of a status; the last error message of a context. */
const char *pnuc_status_string(pnuc_status s);
pnuc_status pnuc_last_error(const pnuc_ctx *ctx, char *buf, size_t len);

/* Builds the target table of nucleus (Z, A) on the device (§2.2, Eq. 1: 15-shell density
 * steps of the Fermi distribution with c = 1.07 A^(1/3) fm, delta = 0.545 fm, radius
 * c + 2.5 fm; two Fermi gases; potential = Fermi energy + SEMF separation energy; Coulomb
 * barrier) and returns its id (0, 1, ...) in *target_id. Supported: 6 <= A <= 250,
 * 2 <= Z <= 100, A - Z >= 2, positive SEMF separation energies (else PNUC_ERR_RANGE).
 * At most 16 targets per context (PNUC_ERR_CAPACITY). Synchronous. Creating the same
 * (Z, A) twice returns the existing id. */
pnuc_status pnuc_create_target(pnuc_ctx *ctx, int32_t Z, int32_t A, int32_t *target_id);

/* Host copy of a target table, for inspection (FP64 values as the kernels use them). */
typedef struct {
    int32_t Z, A;
    double R, EC, M, S_n, S_p;
    double r[16];
    double rho[15], vF[15];
    double pF[2][15], EF[2][15], V[2][15]; /* [0] neutrons, [1] protons */
} pnuc_target_info;
pnuc_status pnuc_target_table(pnuc_ctx *ctx, int32_t target_id, pnuc_target_info *out);

/* Simulates batch->n events (the hot path: §2.3 cascade + §2.4 evaporation) with the
 * given precision and method, writing out->residuals[0..n-1], the secondaries and
 * *out->count. Asynchronous on stream. n = 0 writes *count = 0 and returns. Buffers must
 * not overlap. Per-event problems are reported in residual flags, not in the status. */
pnuc_status pnuc_simulate(pnuc_ctx *ctx, pnuc_precision precision, pnuc_method method,
                          const pnuc_batch *batch, const pnuc_output *out, void *stream);

/* pnuc_simulate with HOST buffers: energies/target_ids (host, n entries) are copied to
 * device staging buffers the context owns (grown as needed), the batch runs, and the
 * residuals (host, n entries), up to sec_capacity secondaries (host) and the produced
 * count (host) are copied back. Output buffers in pinned host memory (cudaHostAlloc,
 * cudaHostRegister, a framework's pinned tensor), 16-byte aligned, are instead written by
 * the kernels directly (secondaries and residuals each, where it holds), with no copy after
 * them. Synchronous: returns after the results are on the host.
 * Returns PNUC_ERR_CAPACITY if *sec_count > sec_capacity (the first sec_capacity
 * records are still written). Incident protons (neutron-induced events go through
 * pnuc_simulate with pnuc_batch.projectiles). */
pnuc_status pnuc_simulate_host(pnuc_ctx *ctx, pnuc_precision precision, pnuc_method method,
                               const double *energies, const int32_t *target_ids, uint64_t n,
                               uint64_t seed, uint64_t first_event_id, pnuc_secondary *secondaries,
                               uint64_t sec_capacity, uint64_t *sec_count, pnuc_residual *residuals,
                               void *stream);

/* pnuc_simulate_host without any device allocation (the paper has no counterpart: this
 * serves embedding). For callers that cannot call cudaMalloc at simulation time: host
 * applications whose device memory is owned by another allocator (a framework's caching
 * allocator or a pre-reserved pool) or that must not grow their device footprint while
 * running, which pnuc_simulate_host would do the first time it meets a larger batch.
 *
 * Same arguments, results and errors as pnuc_simulate_host, but the device copies of the
 * inputs and outputs and the persistent kernel's queue head live in one static device
 * array of PNUC_NOALLOC_SCRATCH_BYTES (8 MiB) that every GPU loading this library holds
 * until the process exits; output buffers in pinned host memory are written in place and
 * take none of it. A batch whose layout does not fit (about 8 MiB / (76 + 32 k) events for
 * room for k secondaries per event with pageable outputs: 24,000 events at k = 8; 8 MiB / 12
 * = 690,000 events with pinned ones) is rejected with PNUC_ERR_CAPACITY before anything
 * runs. The entry point calls no cudaMalloc, cudaFree or
 * allocating library routine. Its first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first call before any
 * stream capture. Every call shares the array and it keeps the last call's contents; the
 * call clears what must start at zero. Calls whose work overlaps on the GPU (several host
 * threads, or several contexts of one device) race on the array: serialise them. */
#define PNUC_NOALLOC_SCRATCH_BYTES (8u << 20)
pnuc_status pnuc_simulate_host_noalloc(pnuc_ctx *ctx, pnuc_precision precision, pnuc_method method,
                                       const double *energies, const int32_t *target_ids, uint64_t n, uint64_t seed,
                                       uint64_t first_event_id, pnuc_secondary *secondaries, uint64_t sec_capacity,
                                       uint64_t *sec_count, pnuc_residual *residuals, void *stream);

/* Persistent-method tuning of the context (per precision). set checks the ranges above. */
pnuc_status pnuc_get_tuning(const pnuc_ctx *ctx, pnuc_precision precision, pnuc_tuning *out);
pnuc_status pnuc_set_tuning(pnuc_ctx *ctx, pnuc_precision precision, const pnuc_tuning *t);

/* Autotuner of the persistent method: from the context's current tuning for `precision`,
 * a coordinate search over block_size, kin_batch,
 * refill_threshold and chunk (two passes; each candidate timed with CUDA events over `reps`
 * launches after one warm-up, on the given batch and output buffers, whose contents it
 * overwrites). The fastest tuning is kept in the context and written to *best (and its
 * mean launch time in ms to *best_ms); either may be NULL. Tuning never changes an event's
 * result. Synchronous on `stream`. Errors: PNUC_ERR_ARG for an empty batch or reps outside
 * [1, 100]; PNUC_ERR_CUDA if a launch fails. Not in the paper (its kernels were hand-sized);
 * it serves the batched method. */
pnuc_status pnuc_autotune(pnuc_ctx *ctx, pnuc_precision precision, const pnuc_batch *batch, const pnuc_output *out,
                          int32_t reps, pnuc_tuning *best, double *best_ms, void *stream);

/* Tuning cache: pnuc_save_tuning writes both precisions' tunings of the context into the
 * JSON file at `path` under the device's name, keeping other devices' entries (a malformed
 * file is replaced). pnuc_load_tuning reads them back; PNUC_ERR_RANGE if the file is missing
 * or has no entry for this device, PNUC_ERR_ARG if it is malformed or a stored tuning is
 * invalid (the context is then unchanged). */
pnuc_status pnuc_save_tuning(pnuc_ctx *ctx, const char *path);
pnuc_status pnuc_load_tuning(pnuc_ctx *ctx, const char *path);

/* CUDA-graph launch plans. pnuc_graph_create captures one pnuc_simulate launch (output
 * count reset, queue-head reset, event kernel) for fixed batch and output buffers, the
 * given precision and method and the context's current tuning; pnuc_graph_launch replays
 * it on `stream` (asynchronous, same results as pnuc_simulate). pnuc_graph_update re-captures
 * for new buffers, n or seed and updates the executable graph in place when CUDA allows,
 * else re-instantiates it. A plan owns its queue head, so replays of different plans may run
 * concurrently; replays of one plan must not overlap. Buffers must stay valid while a plan
 * that uses them may run. The plan holds pointers into the context: destroy plans before
 * their context. */
typedef struct pnuc_graph pnuc_graph;
pnuc_status pnuc_graph_create(pnuc_ctx *ctx, pnuc_precision precision, pnuc_method method, const pnuc_batch *batch,
                              const pnuc_output *out, pnuc_graph **graph);
pnuc_status pnuc_graph_update(pnuc_graph *graph, const pnuc_batch *batch, const pnuc_output *out);
pnuc_status pnuc_graph_launch(pnuc_graph *graph, void *stream);
pnuc_status pnuc_graph_destroy(pnuc_graph *graph);

/* Serving loop (not in the paper: it motivates the code as a component of a GPU proton
 * transport Monte Carlo, §1 and §4.2). A transport driver submits interaction requests as
 * they arise; a scheduler thread admits queued requests in order whenever one of `streams`
 * CUDA streams is free and both a device arena (the inputs, and a merged launch's
 * secondaries) and a pinned host arena (residuals and sec_per_event secondaries per event,
 * written there by the kernels) of arena_bytes each have room (memory-based admission).
 * Queued requests with the same seed are merged, up to max_merge of them and merge_events
 * events, into one persistent launch on a free stream, each event keeping its own id; a
 * partition kernel then gives every request a contiguous range of secondaries. Launches on
 * different streams overlap on the GPU (continuous batching). A
 * request that produces more secondaries than reserved is run again alone, with room for
 * exactly its count; as results depend only on (seed, event id), every request's results
 * equal those of a lone pnuc_simulate call. Latency is measured from submit to results ready
 * on the host. */
typedef struct {
    int32_t precision;           /* pnuc_precision */
    int32_t streams;             /* requests in flight at once, 1..64 (default 8) */
    uint64_t arena_bytes;        /* device arena and pinned host arena, each (default 1 GiB, >= 1 MiB) */
    uint32_t sec_per_event;      /* secondaries reserved per event at admission, 1..256 (default 12) */
    uint32_t max_pending;        /* queued requests before submit refuses (default 4096) */
    uint64_t max_request_events; /* largest request accepted (default 2^24) */
    uint32_t max_merge;          /* requests merged into one launch, 1..64 (default 32; 1 = never) */
    uint32_t merge_events;       /* a group takes no further request that would bring it above this
                                    many events, 1..2^22 (default 2^18) */
    uint32_t lane_events;        /* a launch gets blocks for about this many events per lane (at
                                    most the resident limit), so that small launches leave SMs to
                                    the others and do not each wait on their slowest event with
                                    the whole GPU, 1..1024 (default 4) */
    uint32_t max_inflight_events; /* no new launch while launches of at least this many events
                                    are in flight (0: no limit; default 0): under heavy load
                                    requests then wait and merge instead of splitting the GPU
                                    among more launches */
} pnuc_server_config;

typedef struct {
    uint64_t completed, failed, reruns, events, pending;
    double latency_p50_ms, latency_p99_ms, latency_max_ms; /* submit -> results on the host */
    double queue_p50_ms, queue_p99_ms;                     /* submit -> admission */
    double elapsed_s, events_per_s;                        /* since creation or the last reset */
    uint64_t arena_peak_bytes;                             /* largest use of either arena */
    uint64_t launches;                                     /* kernel launches (merged groups and re-runs) */
} pnuc_server_stats;

typedef struct pnuc_server pnuc_server;
void pnuc_server_default_config(pnuc_server_config *cfg);
/* Allocates the arenas (device and pinned host), the streams and the scheduler thread. */
pnuc_status pnuc_server_create(pnuc_ctx *ctx, const pnuc_server_config *cfg, pnuc_server **server);
/* Queues a request of n events (host inputs, copied before returning; target ids from
 * pnuc_create_target) and returns its ticket. PNUC_ERR_ARG if n is 0, above
 * max_request_events or can never fit the arena; PNUC_ERR_CAPACITY if max_pending requests
 * are queued (submit again later). Thread-safe. */
pnuc_status pnuc_server_submit(pnuc_server *server, const double *energies, const int32_t *target_ids, uint64_t n,
                               uint64_t seed, uint64_t first_event_id, uint64_t *ticket);
/* pnuc_server_submit with the incident nucleon of each event (projectiles: host, n entries,
 * 1 proton, 0 neutron, other values flagged PNUC_FLAG_BAD_INPUT as in pnuc_batch; NULL =
 * protons): a transport code's secondary neutrons go through the same loop. Requests with
 * and without species merge as usual. */
pnuc_status pnuc_server_submit_nucleons(pnuc_server *server, const double *energies, const int32_t *target_ids,
                                        const uint8_t *projectiles, uint64_t n, uint64_t seed,
                                        uint64_t first_event_id, uint64_t *ticket);
/* Waits up to timeout_ms (negative: no limit) for the request; PNUC_ERR_TIMEOUT if it is not
 * done by then, else the request's status, and *n_secondaries its number of secondaries. */
pnuc_status pnuc_server_wait(pnuc_server *server, uint64_t ticket, int32_t timeout_ms, uint64_t *n_secondaries);
/* Waits up to timeout_ms (negative: no limit) for any request to finish that no earlier
 * pnuc_server_wait_any returned, in the order they finished; PNUC_ERR_TIMEOUT if none does,
 * else PNUC_OK with *ticket the finished request (done or failed: view, fetch or release it
 * as after pnuc_server_wait). Requests released before they are returned are skipped. Lets
 * a driver take results as they complete rather than in submission order. */
pnuc_status pnuc_server_wait_any(pnuc_server *server, int32_t timeout_ms, uint64_t *ticket);
/* Copies a finished request's residuals (n records) and secondaries (host buffers; capacity
 * at least its count, else PNUC_ERR_CAPACITY and nothing is released) and releases it.
 * PNUC_ERR_STATE if it is not finished; a failed request returns its error and is released.
 * Finished requests hold pinned host memory until fetched. */
pnuc_status pnuc_server_fetch(pnuc_server *server, uint64_t ticket, pnuc_secondary *secondaries, uint64_t capacity,
                              pnuc_residual *residuals);
/* Zero-copy alternative to pnuc_server_fetch: points *secondaries (*n_secondaries records)
 * and *residuals (n records) at a finished request's results where they landed, in the
 * server's pinned host arena. They stay valid, and the arena space stays taken, until
 * pnuc_server_release(ticket) or pnuc_server_destroy(). PNUC_ERR_STATE if the request is not
 * finished; a failed request returns its error and is released. */
pnuc_status pnuc_server_view(pnuc_server *server, uint64_t ticket, const pnuc_secondary **secondaries,
                             uint64_t *n_secondaries, const pnuc_residual **residuals);
/* Releases a finished request without copying (after pnuc_server_view). */
pnuc_status pnuc_server_release(pnuc_server *server, uint64_t ticket);
pnuc_status pnuc_server_get_stats(pnuc_server *server, pnuc_server_stats *out);
pnuc_status pnuc_server_reset_stats(pnuc_server *server);
/* Drops queued requests, waits for those in flight, frees everything. Safe on NULL. */
pnuc_status pnuc_server_destroy(pnuc_server *server);

/* Per-request trace of the serving loop (measurement support; the paper has no counterpart),
 * to attribute latency to the queue, the host, the GPU or the client. pnuc_server_trace(S, 1)
 * clears the record and records one entry per request released from then on (up to 2^20);
 * pnuc_server_trace(S, 0) stops and keeps the record. Times are milliseconds on the host's
 * steady clock from the trace's start; the GPU times (the GPU's global timer, stamped by a
 * one-warp kernel on the request's stream before its launch's first copy and after its last
 * one) are put on that clock by a stamp taken when the trace starts (aligned to a few tens of
 * microseconds). The stamps are plain kernels, so tracing leaves the streams' concurrency as
 * it is (CUDA events with timing enabled did not: they raised the median latency 3-fold). A
 * request that ran more than once (an overflow re-run) carries its last launch. */
typedef struct {
    uint64_t ticket, events, launch; /* launch: the server's launch number of the request's run */
    int32_t stream, group_requests;  /* its stream and the requests merged into that launch */
    int32_t reruns, status;
    double t_submit, t_admit;        /* submitted; admitted into a launch (first admission) */
    double t_launched;               /* the launch's copies and kernels enqueued (host) */
    double t_gpu_start, t_gpu_end;   /* the launch ran on the GPU from .. to */
    double t_complete;               /* the server saw the launch complete */
    double t_release;                /* the client released or fetched the request */
} pnuc_server_trace_entry;
pnuc_status pnuc_server_trace(pnuc_server *server, int32_t enable);
/* Copies up to capacity entries (in release order) to out and their total to *count. */
pnuc_status pnuc_server_trace_read(pnuc_server *server, pnuc_server_trace_entry *out, uint64_t capacity,
                                   uint64_t *count);

/* Yield tallies of a batch (paper §4.1, Figs. 1-2: secondary yields per energy and angle;
 * §4.2: yields of positron emitters, i.e. of residual nuclei, per incident energy). One pass
 * over the output records on the device, accumulated (+=) into caller-owned device
 * histograms of unsigned 64-bit counts, so several batches can add up.
 *
 * Secondaries: bin (origin, species, cos theta, T) of each record with T in [T_min, T_max):
 *   iT = floor((T - T_min) * sT) with sT = n_T / (T_max - T_min),
 *   ic = min(floor((uz + 1) * (n_cos / 2)), n_cos - 1), histogram
 *   [2 origins][6 species][n_cos][n_T]; records outside the T range are not counted.
 * Residuals: events without PNUC_FLAG_BAD_INPUT or PNUC_FLAG_ATTEMPT_CAP, with incident
 *   energy E in [E_min, E_max), Z_final <= Z_max (<= 255) and A_final <= A_max (<= 511):
 *   iE = floor((E - E_min) * sE) with sE = n_E / (E_max - E_min), histogram
 *   [n_E][Z_max + 1][A_max + 1].
 * The bins are those of FP64 arithmetic, each operation rounded to nearest in the order
 * written (the kernels decide most of them in FP32 where an error bound proves the same
 * result, and take the FP64 expression near a bin edge). Either
 * histogram may be NULL (that part is skipped). sec and
 * res/energies are the device arrays of one batch (n_sec records, n events).
 * PNUC_ERR_ARG for a bad spec (empty or inverted ranges, more than 2^28 cells). */
typedef struct {
    int32_t n_T, n_cos;
    double T_min, T_max;
    int32_t n_E, Z_max;
    double E_min, E_max;
    int32_t A_max, reserved;
} pnuc_tally_spec;
pnuc_status pnuc_tally(pnuc_ctx *ctx, const pnuc_tally_spec *spec, const pnuc_secondary *secondaries,
                       uint64_t n_secondaries, const pnuc_residual *residuals, const double *energies, uint64_t n,
                       unsigned long long *secondary_hist, unsigned long long *residual_hist, void *stream);

/* Secondary yields in angular windows (paper §4.1, Fig. 2: energy spectra of the secondaries
 * in narrow windows around fixed laboratory angles). Window k holds the records with
 *   cos_lo[k] <= uz < cos_hi[k],
 * uz being the record's direction cosine to the beam (a float, compared exactly with the
 * double edges); T bins as in pnuc_tally (n_T bins over [T_min, T_max), the bins of FP64
 * arithmetic). cos_lo and cos_hi are host arrays of n_windows (1 .. PNUC_MAX_WINDOWS) finite
 * values with cos_lo[k] < cos_hi[k]; windows must not overlap. One pass over the records on
 * the device, accumulated (+=) into the caller's device histogram of unsigned 64-bit counts
 * [2 origins][6 species][n_windows][n_T]; records outside every window or the T range are not
 * counted. Asynchronous on stream. PNUC_ERR_ARG for a bad window list or T range, or a null
 * pointer with records to count. */
#define PNUC_MAX_WINDOWS 64
pnuc_status pnuc_tally_windows(pnuc_ctx *ctx, int32_t n_T, double T_min, double T_max, const double *cos_lo,
                               const double *cos_hi, int32_t n_windows, const pnuc_secondary *secondaries,
                               uint64_t n_secondaries, unsigned long long *hist, void *stream);

/* Per-kernel timing of pnuc_simulate's launches (measurement support; the paper has no
 * counterpart). pnuc_kernel_timing(ctx, 1) clears the record and makes later launches
 * through pnuc_simulate and the entry points built on it record CUDA events on the
 * launching stream: before the first kernel, between the cascade kernel and the evaporation
 * kernel (persistent method), and after the last kernel. Launches made while the stream is
 * being captured into a graph, and launches beyond the first 4096 since the clear, are not
 * recorded. pnuc_kernel_timing(ctx, 0) stops recording and keeps the record.
 * pnuc_kernel_times waits for the recorded events and returns, summed over the recorded
 * launches, the milliseconds of the first kernel (the cascade kernel, or the plain kernel)
 * and of the evaporation kernel (0 for the plain method), and the number of recorded
 * launches. Any output pointer may be NULL. The record is not locked: enable it only while one
 * host thread launches on the context (not while a pnuc_server runs on it). */
pnuc_status pnuc_kernel_timing(pnuc_ctx *ctx, int32_t enable);
pnuc_status pnuc_kernel_times(pnuc_ctx *ctx, double *cascade_ms, double *evaporation_ms, uint64_t *launches);

/* The double-precision exponential the FP32 mode's evaporation widths take (§2.4: the widths'
 * e^x, x = 2 sqrt(a Y)), evaluated on the integer pipes by a fixed-point table method (the FP64
 * pipe is scarce on GB300), exposed so that its accuracy can be tested: out[i] = e^x[i] for
 * x[i] in [1, 256), -1 for other arguments. x and out: device arrays of n entries. Asynchronous
 * on stream. The paper has no counterpart. */
pnuc_status pnuc_width_exp(pnuc_ctx *ctx, const float *x, double *out, uint64_t n, void *stream);

/* Measured throughput of the pipes the event kernels use, in lane operations per second
 * (one fused multiply-add = one operation): FP32 FMA, FP64 FMA, special-function unit
 * (reciprocal square root) and 32-bit integer multiply-add. Independent FMA chains on 8
 * blocks of 256 threads per SM, timed with CUDA events. These are the denominators of
 * the ALU roofline (the method has no dense contraction and its HBM traffic is small).
 * Synchronous; takes about a second. Not part of the paper: measurement support. */
typedef struct {
    double fp32_fma, fp64_fma, mufu, int32_mad;
} pnuc_peaks;
pnuc_status pnuc_measure_peaks(pnuc_ctx *ctx, pnuc_peaks *out);

#ifdef __cplusplus
}
#endif
#endif /* PNUC_H */
