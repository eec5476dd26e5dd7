// Nucleus set-up on the device (paper §2.2, Eq. 1): the nuclide mass table and the
// 15-shell table of a target. Both run once per context / target; FP64 throughout.
#include "pnuc_internal.h"

namespace pnuc {
namespace {

constexpr double kHbarc = 197.3269804;  // MeV fm
constexpr double kE2 = 1.44;            // e^2, MeV fm
constexpr double kMp = 938.272, kMn = 939.565;
constexpr double kPi = 3.141592653589793;

// Semi-empirical nuclear mass (liquid drop with pairing), MeV.
__device__ double semf(int Z, int A)
{
    double a = A, z = Z, n = A - Z;
    double a13 = cbrt(a);
    double asym = a - 2.0 * z;
    double B = 15.75 * a - 17.8 * (a13 * a13) - 0.711 * z * (z - 1.0) / a13 - 23.7 * asym * asym / a;
    bool zodd = Z & 1, nodd = (A - Z) & 1;
    if (!zodd && !nodd) B += 11.18 / sqrt(a);
    else if (zodd && nodd) B -= 11.18 / sqrt(a);
    return z * kMp + n * kMn - B;
}

__global__ void mass_table_kernel(double *mass, double *cbrtA)
{
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < kMassA) cbrtA[idx] = cbrt((double)idx);
    if (idx >= kMassZ * kMassA) return;
    int Z = idx / kMassA, A = idx % kMassA;
    mass[idx] = (A >= 1 && Z <= A) ? semf(Z, A) : 0.0;
}

// Reading M26's constants of a daughter of mass number A (a = A/8; the level density is
// constant-temperature below the matching energy U_x = 2.5 + 150/A MeV): [0] U_x, [1] k = 1/T
// = sqrt(a / U_x), [2] C = e^{sqrt(a U_x)}, [3] e^{k U_x} - 1, [4] e^{k U_x} - 1 - k U_x (k U_x
// >= 4.3 for A >= 5, so no series is needed), and with x_x = 2 sqrt(a U_x) the Fermi-gas
// integrals below U_x, [5] G(x_x) = e^x_x (x_x - 1) + 1 and [6] H(x_x) = e^x_x (x_x^3 - 3 x_x^2
// + 6 x_x - 6) + 6. The FP32 mode's widths take them as factors, so that they divide by
// nothing: [7] C [3] / k, [8] C [4] / k^2, [9] [5] / (2a), [10] [6] / (8 a^2), [11] C / k,
// [12] C / k^2.
__global__ void ct_table_kernel(double *tab)
{
    const int A = blockIdx.x * blockDim.x + threadIdx.x;
    if (A >= kMassA) return;
    double *t = tab + kCtStride * A;
    for (int k = 0; k < kCtStride; ++k) t[k] = 0.0;
    if (A < 5) return;
    const double a = A / 8.0;
    const double Ux = 2.5 + 150.0 / (8.0 * a), k = sqrt(a / Ux), xx = 2.0 * sqrt(a * Ux), kU = k * Ux;
    const double ex = exp(xx);
    t[0] = Ux;
    t[1] = k;
    t[2] = exp(0.5 * xx);
    t[3] = expm1(kU);
    t[4] = expm1(kU) - kU;
    t[5] = ex * (xx - 1.0) + 1.0;
    t[6] = ex * (((xx - 3.0) * xx + 6.0) * xx - 6.0) + 6.0;
    t[7] = t[2] * t[3] / k;
    t[8] = t[2] * t[4] / (k * k);
    t[9] = t[5] / (2.0 * a);
    t[10] = t[6] / (8.0 * a * a);
    t[11] = t[2] / k;
    t[12] = t[2] / (k * k);
}

// The evaporation Q-values of every parent (Z, A) and channel j (paper §2.4): the daughter's
// mass plus the ejectile's, less the parent's, summed in that order (the same FP64 operations
// as the evaporation step would do per channel, so the values are the same bits). Rows whose
// daughter does not exist (Z_d < 1, N_d < 1, A_d < 5) hold 0; the kernels never read them.
__global__ void q_table_kernel(double *q, const double *mass)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= kMassZ * kMassA) return;
    const int Z = idx / kMassA, A = idx % kMassA;
    const double mj[6] = {kEjectileMass[0], kEjectileMass[1], kEjectileMass[2],
                          kEjectileMass[3], kEjectileMass[4], kEjectileMass[5]};
    const int zj[6] = {kEjectileZ[0], kEjectileZ[1], kEjectileZ[2], kEjectileZ[3], kEjectileZ[4], kEjectileZ[5]};
    const int aj[6] = {kEjectileA[0], kEjectileA[1], kEjectileA[2], kEjectileA[3], kEjectileA[4], kEjectileA[5]};
    double *row = q + (size_t)kQStride * idx;
    for (int j = 0; j < kQStride; ++j) {
        double v = 0.0;
        if (j < 6) {
            const int Zd = Z - zj[j], Ad = A - aj[j];
            if (Zd >= 1 && Ad - Zd >= 1 && Ad >= 5 && Z <= A) v = (mass[Zd * kMassA + Ad] + mj[j]) - mass[idx];
        }
        row[j] = v;
    }
}

__device__ double fermi_density(double r, double c) { return 1.0 / (1.0 + exp((r - c) / 0.545)); }

// One block of 15 warps: warp i integrates r^2 f(r) over shell i, each lane one 1/32 of it
// with a 128-panel Simpson rule (4096 panels per shell), then lane 0.. fills the table.
__global__ void target_table_kernel(TargetTable *dst, int Z, int A, const double *mass)
{
    __shared__ double I[kShells];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double c = 1.07 * cbrt((double)A);
    const double R = c + 2.5;  // radius after Chen et al.
    if (warp < kShells) {
        double r0 = warp * R / kShells, r1 = (warp + 1) * R / kShells;
        double h = (r1 - r0) / 4096.0;
        double acc = 0.0;
        for (int k = 0; k <= 128; ++k) {
            int g = lane * 128 + k;  // global panel-point index in [0, 4096]
            double r = r0 + g * h;
            double w = (k == 0 || k == 128) ? 1.0 : ((k & 1) ? 4.0 : 2.0);
            acc += w * r * r * fermi_density(r, c);
        }
        acc *= h / 3.0;
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
        if (lane == 0) I[warp] = acc;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double total = 0.0;
    for (int i = 0; i < kShells; ++i) total += I[i];
    TargetTable t;
    t.Z = Z;
    t.A = A;
    t.R = R;
    t.M = mass[Z * kMassA + A];
    t.S[0] = mass[Z * kMassA + (A - 1)] + kMn - t.M;
    t.S[1] = mass[(Z - 1) * kMassA + (A - 1)] + kMp - t.M;
    t.valid = (t.S[0] > 0.0 && t.S[1] > 0.0) ? 1 : 0;
    t.pad = 0;
    t.d.EC = kE2 * (Z - 1) / R;
    t.d.ZoverA = (double)Z / A;
    t.d.pad[0] = t.d.pad[1] = 0.0;
    for (int k = 0; k <= kShells; ++k) t.d.r[k] = k * R / kShells;
    for (int i = 0; i < kShells; ++i) {
        double r0 = t.d.r[i], r1 = t.d.r[i + 1];
        double rho = 3.0 * A * I[i] / (4.0 * kPi * (r1 * r1 * r1 - r0 * r0 * r0) * total);
        t.d.rho[i] = rho;
        double vmax = 0.0;
        for (int s = 0; s < 2; ++s) {
            double m = s ? kMp : kMn;
            double frac = s ? (double)Z / A : (double)(A - Z) / A;
            double pf = kHbarc * cbrt(3.0 * kPi * kPi * (frac * rho));
            t.d.pF[s][i] = pf;
            t.d.EF[s][i] = pf * pf / (sqrt(pf * pf + m * m) + m);
            t.d.V[s][i] = t.d.EF[s][i] + t.S[s];
            double v = pf / sqrt(pf * pf + m * m);
            vmax = v > vmax ? v : vmax;
        }
        t.d.vF[i] = vmax;
    }
    // FP32 mirror
    for (int k = 0; k <= kShells; ++k) t.f.r[k] = (float)t.d.r[k];
    for (int i = 0; i < kShells; ++i) {
        t.f.rho[i] = (float)t.d.rho[i];
        t.f.vF[i] = (float)t.d.vF[i];
        for (int s = 0; s < 2; ++s) {
            t.f.pF[s][i] = (float)t.d.pF[s][i];
            t.f.EF[s][i] = (float)t.d.EF[s][i];
            t.f.V[s][i] = (float)t.d.V[s][i];
        }
    }
    t.f.EC = (float)t.d.EC;
    t.f.ZoverA = (float)t.d.ZoverA;
    t.f.pad[0] = t.f.pad[1] = 0.f;
    *dst = t;
}

}  // namespace

cudaError_t launch_ct_table(double *tab, cudaStream_t s)
{
    ct_table_kernel<<<1, 256, 0, s>>>(tab);
    return cudaGetLastError();
}

cudaError_t launch_q_table(double *q, const double *mass, cudaStream_t s)
{
    const int n = kMassZ * kMassA;
    q_table_kernel<<<(n + 255) / 256, 256, 0, s>>>(q, mass);
    return cudaGetLastError();
}

cudaError_t launch_mass_table(double *mass, double *cbrtA, cudaStream_t s)
{
    int n = kMassZ * kMassA;
    mass_table_kernel<<<(n + 255) / 256, 256, 0, s>>>(mass, cbrtA);
    return cudaGetLastError();
}

cudaError_t launch_target_table(TargetTable *dst, int Z, int A, const double *mass, cudaStream_t s)
{
    target_table_kernel<<<1, 32 * kShells, 0, s>>>(dst, Z, A, mass);
    return cudaGetLastError();
}

}  // namespace pnuc
