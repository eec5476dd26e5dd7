// Internal declarations shared by the libpnuc translation units (host API, table
// kernels, and the FP32 / FP64 event kernels). Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pnuc.h"

namespace pnuc {

constexpr int kShells = 15;      // equal-thickness density steps (paper §2.2)
constexpr int kMaxTargets = 16;  // targets per context
constexpr int kStackCap = 64;    // particles waiting in one event's cascade
constexpr int kMassZ = 102;      // nuclide table covers Z in [0, 101]
constexpr int kMassA = 252;      //                     and A in [0, 251]
constexpr int kCtStride = 16;    // doubles per daughter in the table of reading M26's constants
constexpr int kQStride = 8;      // doubles per parent (Z, A) in the Q-value table (six channels used)

// Evaporated ejectiles n, p, d, t, 3He, alpha (paper §2.4: He and lighter): masses (MeV),
// charge and mass numbers.
constexpr double kEjectileMass[6] = {939.565, 938.272, 1875.613, 2808.921, 2808.391, 3727.379};
constexpr int kEjectileZ[6] = {0, 1, 1, 1, 2, 2};
constexpr int kEjectileA[6] = {1, 1, 2, 3, 3, 4};

// One target's shell table in precision R (paper §2.2). Index [0] = neutrons, [1] = protons.
template <typename R>
struct ShellTable {
    R r[16];        // shell radii r_k = k R / 15, fm
    R rho[15];      // nucleon density of shell i, fm^-3
    R vF[15];       // largest Fermi velocity of the two species in shell i (units of c)
    R pF[2][15];    // Fermi momentum, MeV/c
    R EF[2][15];    // Fermi kinetic energy, MeV
    R V[2][15];     // well depth = Fermi energy + separation energy, MeV
    R EC;           // Coulomb barrier e^2 (Z-1)/R, MeV
    R ZoverA;       // probability that a partner is a proton
    R pad[2];
};

// Device-resident description of one target: the shell table in both precisions plus
// the FP64 scalars the bookkeeping needs.
struct TargetTable {
    ShellTable<double> d;
    ShellTable<float> f;
    double M;     // SEMF nuclear mass, MeV
    double S[2];  // separation energies, MeV
    double R;     // radius c + 2.5 fm
    int32_t Z, A;
    int32_t valid, pad;
};

// Everything a simulation launch reads; passed by value to the kernels.
struct SimParams {
    const double *energies;
    const int32_t *target_ids;
    const uint8_t *projectiles;      // per event 1 proton, 0 neutron; null = all protons
    const unsigned long long *event_ids;  // per-event ids, or null
    // merged requests (serving): event i of segment k (seg_start[k] <= i < seg_start[k+1]) has
    // id seg_first[k] + i - seg_start[k]; n_seg = 0: id first_event_id + i
    const unsigned long long *seg_first;
    const uint32_t *seg_start;
    int32_t n_seg;
    uint64_t n;
    uint64_t seed;
    uint64_t first_event_id;
    pnuc_secondary *sec;
    uint64_t sec_cap;
    unsigned long long *sec_count;
    pnuc_residual *res;
    unsigned long long *counters;  // may be null
    const TargetTable *tables;     // n_targets entries
    int32_t n_targets;
    const double *mass;            // [kMassZ * kMassA] SEMF masses, MeV (0 where undefined)
    const double *cbrtA;           // [kMassA] A^(1/3)
    const double *ct_table;        // [kMassA * kCtStride] reading M26's constants per daughter A
    // [kMassZ * kMassA * kQStride] Q-values of the six channels of a parent (Z, A):
    // (M(Z - z_j, A - a_j) + m_j) - M(Z, A), entry j of row Z * kMassA + A
    const double *qval;
    unsigned long long *queue_head;  // persistent method: next unclaimed event of the cascade kernel
    unsigned long long *evap_head;   // persistent method: next unclaimed event of the evaporation kernel
    int32_t split_evap;              // 1: persistent method (the cascade kernel leaves evaporation to evap_kernel)
    int32_t max_steps, max_attempts, max_evap_steps, max_evap_trials;
    int32_t level_density;  // 0 Fermi gas (reading M20), 1 constant temperature below U_x (M26)
    int32_t refill_threshold, chunk;
    int32_t kin_batch;  // persistent kernel: accepted collisions a warp gathers before their kinematics
};

// Launchers, one per compiled variant (kernel_fp32.cu, kernel_fp64.cu).
cudaError_t launch_plain_fp64(const SimParams &p, int block, cudaStream_t s);
cudaError_t launch_persistent_fp64(const SimParams &p, int grid, int block, cudaStream_t s);
cudaError_t launch_evap_fp64(const SimParams &p, int grid, int block, cudaStream_t s);
// FP32 launchers of kernels that evaporate take `scaled`: the evaporation widths in FP32,
// scaled by the largest channel's exponential (PNUC_FP32_SCALED), instead of FP64 (PNUC_FP32).
cudaError_t launch_evap_fp32(const SimParams &p, int grid, int block, bool count, bool scaled, cudaStream_t s);
cudaError_t launch_plain_fp32(const SimParams &p, int block, bool count, bool scaled, cudaStream_t s);
cudaError_t launch_persistent_fp32(const SimParams &p, int grid, int block, bool count, cudaStream_t s);
// Resident blocks per SM of the persistent kernels at a block size.
int occupancy_persistent_fp64(int block);
int occupancy_persistent_fp32(int block, bool count);
int occupancy_evap_fp64(int block, bool ct);
int occupancy_evap_fp32(int block, bool count, bool scaled, bool ct);
// Sorted method (cascade kernel regrouping slots by action): launchers, resident blocks per
// SM, and the bytes of one slot's particle stack (the stacks live in a context buffer).
cudaError_t launch_sorted_fp64(const SimParams &p, void *stacks, int grid, int block, cudaStream_t s);
cudaError_t launch_sorted_fp32(const SimParams &p, void *stacks, int grid, int block, bool count, cudaStream_t s);
int occupancy_sorted_fp64(int block);
int occupancy_sorted_fp32(int block, bool count);
size_t sorted_stack_bytes_fp64();
size_t sorted_stack_bytes_fp32();

// The FP32 mode's double-precision width exponential on n float arguments (kernel_fp32.cu).
cudaError_t launch_width_exp(const float *x, double *out, uint64_t n, int sm_count, cudaStream_t s);

// Pipe microbenchmarks (microbench.cu): FP32 FMA, FP64 FMA, MUFU, INT32 MAD lane ops/s.
cudaError_t measure_peaks(int sm_count, double out[4]);

// Table builders (tables.cu).
cudaError_t launch_mass_table(double *mass, double *cbrtA, cudaStream_t s);
cudaError_t launch_ct_table(double *tab, cudaStream_t s);
cudaError_t launch_q_table(double *q, const double *mass, cudaStream_t s);
cudaError_t launch_target_table(TargetTable *dst, int Z, int A, const double *mass, cudaStream_t s);

}  // namespace pnuc
