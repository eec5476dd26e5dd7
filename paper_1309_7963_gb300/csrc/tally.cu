// Yield tallies (pnuc_tally): histograms of a batch's secondaries by (origin, species,
// cos theta, T) and of its residual nuclei by (incident energy, Z, A), the outputs the paper
// plots (§4.1, Figs. 1-2) and the positron-emitter yields it proposes (§4.2).
//
// Both kernels are one streaming pass over the output records: coalesced 16-byte loads
// (the residual kernel reads only the first 32 bytes of each 64-byte record), per-block
// shared-memory histograms when the histogram fits, and warp-aggregated 64-bit atomics
// (lanes that hit the same cell add once) otherwise. The bin arithmetic is FP64 with
// explicit round-to-nearest operations, so the host can reproduce every bin index; the
// floors and range tests are taken from the bit fields on the integer pipes.
#include <algorithm>
#include <climits>

#include "api_internal.h"
#include "fpconv.h"

namespace pnuc {
namespace {

constexpr int kTallyBlock = 256;
constexpr int kSmemBins = 12288;  // 32-bit shared counters per block (48 KB)
constexpr int kUnroll = 4;        // records in flight per thread

// floor(t) from the bit fields of t on the integer pipes (the FP64 pipe, GB300's scarce one,
// would otherwise take a conversion and two comparisons per record): -1 for t < 0, INT_MAX
// for t >= 2^31, infinities and NaN; -0 counts as 0.
__device__ __forceinline__ int floor_bits(double t)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(t);
    if (b >> 63) return (b << 1) == 0ull ? 0 : -1;
    const int e = (int)((b >> 52) & 0x7ffu) - 1023;
    if (e < 0) return 0;
    if (e > 30) return INT_MAX;
    const unsigned long long m = (b & 0xfffffffffffffull) | (1ull << 52);
    return (int)(m >> (52 - e));
}

__device__ __forceinline__ void add_cell(unsigned long long *hist, int idx)
{
    // lanes of the warp that reach here with the same cell add once
    const unsigned peers = __match_any_sync(__activemask(), idx);
    if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&hist[idx], (unsigned long long)__popc(peers));
}

__device__ __forceinline__ void add_cell_shared(unsigned int *cells, int idx)
{
    // the same for shared counters: most records fall in a few low-energy bins, and lanes
    // adding to one address would otherwise serialise
    const unsigned peers = __match_any_sync(__activemask(), idx);
    if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&cells[idx], (unsigned int)__popc(peers));
}

__global__ void __launch_bounds__(kTallyBlock)
    secondary_tally_kernel(const uint4 *__restrict__ rec, uint64_t n, double T_min, double sT, int nT, double hc,
                           int ncos, unsigned long long *hist, int nbins)
{
    // shared counters: one copy per warp when they fit (the low-energy evaporation bins
    // take most records, so per-warp copies spread the contention), else one per block
    extern __shared__ unsigned int cells[];
    const bool priv = nbins <= kSmemBins;
    const int copies = priv && nbins * (kTallyBlock / 32) <= kSmemBins ? kTallyBlock / 32 : 1;
    const int total = priv ? nbins * copies : 0;
    if (priv) {
        for (int i = threadIdx.x; i < total; i += blockDim.x) cells[i] = 0u;
        __syncthreads();
    }
    unsigned int *mine = cells + (copies > 1 ? (int)(threadIdx.x >> 5) * nbins : 0);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    // four records in flight per thread: the loads of a group are issued together
    for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += kUnroll * stride) {
        uint4 ra[kUnroll], rb[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const uint64_t i = i0 + u * stride;
            if (i < n) {
                ra[u] = __ldcs(rec + 2 * i);
                rb[u] = __ldcs(rec + 2 * i + 1);
            } else {
                ra[u] = make_uint4(0u, 0xffu, 0u, 0u);  // species 255: skipped below
                rb[u] = make_uint4(0u, 0u, 0u, 0u);
            }
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const uint4 a = ra[u], b = rb[u];
            const unsigned sp = a.y & 0xffu, org = (a.y >> 8) & 0xffu;
            const double T = __hiloint2double((int)a.w, (int)a.z);
            const int iT = floor_bits(__dmul_rn(__dsub_rn(T, T_min), sT));
            if (iT < 0 || iT >= nT || sp > 5u || org > 1u) continue;
            int ic = 0;
            if (ncos > 1) {
                ic = floor_bits(__dmul_rn(__dadd_rn(f2d(__uint_as_float(b.z)), 1.0), hc));
                if (ic < 0) ic = 0;
                if (ic > ncos - 1) ic = ncos - 1;
            }
            const int idx = (((int)org * 6 + (int)sp) * ncos + ic) * nT + iT;
            if (priv) add_cell_shared(mine, idx);
            else add_cell(hist, idx);
        }
    }
    if (priv) {
        __syncthreads();
        for (int i = threadIdx.x; i < nbins; i += blockDim.x) {
            unsigned long long c = 0;
            for (int k = 0; k < copies; ++k) c += cells[k * nbins + i];
            if (c) atomicAdd(&hist[i], c);
        }
    }
}

__global__ void __launch_bounds__(kTallyBlock)
    residual_tally_kernel(const uint4 *__restrict__ res, const double *__restrict__ energies, uint64_t n,
                          double E_min, double sE, int nE, int Zmax, int Amax, unsigned long long *hist, int nbins)
{
    extern __shared__ unsigned int cells[];
    const bool priv = nbins <= kSmemBins;
    if (priv) {
        for (int i = threadIdx.x; i < nbins; i += blockDim.x) cells[i] = 0u;
        __syncthreads();
    }
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += kUnroll * stride) {
        uint4 ra[kUnroll], rb[kUnroll];
        double re[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {  // the Z/A fields, the flags, the energy
            const uint64_t i = i0 + u * stride;
            if (i < n) {
                ra[u] = __ldcs(res + 4 * i);
                rb[u] = __ldcs(res + 4 * i + 1);
                re[u] = __ldcs(energies + i);
            } else {
                ra[u] = make_uint4(0u, 0u, 0u, 0u);
                rb[u] = make_uint4(PNUC_FLAG_BAD_INPUT, 0u, 0u, 0u);  // skipped below
                re[u] = 0.0;
            }
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            if (rb[u].x & (PNUC_FLAG_BAD_INPUT | PNUC_FLAG_ATTEMPT_CAP)) continue;
            const int iE = floor_bits(__dmul_rn(__dsub_rn(re[u], E_min), sE));
            const int Z = (int)(ra[u].y & 0xffffu), A = (int)(ra[u].y >> 16);
            if (iE < 0 || iE >= nE || Z > Zmax || A > Amax) continue;
            const int idx = (iE * (Zmax + 1) + Z) * (Amax + 1) + A;
            if (priv) add_cell_shared(cells, idx);
            else add_cell(hist, idx);
        }
    }
    if (priv) {
        __syncthreads();
        for (int i = threadIdx.x; i < nbins; i += blockDim.x)
            if (cells[i]) atomicAdd(&hist[i], (unsigned long long)cells[i]);
    }
}

// two resident blocks per SM: enough loads in flight with four records per thread, and few
// per-block histograms to add up at the end
int tally_grid(uint64_t n, int sm_count)
{
    const uint64_t need = (n + kTallyBlock - 1) / kTallyBlock;
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(need, (uint64_t)sm_count * 2));
}

}  // namespace
}  // namespace pnuc

using namespace pnuc;

extern "C" pnuc_status pnuc_tally(pnuc_ctx *ctx, const pnuc_tally_spec *spec, const pnuc_secondary *secondaries,
                                  uint64_t n_secondaries, const pnuc_residual *residuals, const double *energies,
                                  uint64_t n, unsigned long long *secondary_hist, unsigned long long *residual_hist,
                                  void *stream)
{
    if (!ctx || !spec) return fail(ctx, PNUC_ERR_ARG, "null argument");
    const pnuc_tally_spec &s = *spec;
    cudaStream_t st = (cudaStream_t)stream;
    CU(ctx, cudaSetDevice(ctx->cfg.device));
    if (secondary_hist) {
        if (s.n_T < 1 || s.n_cos < 1 || !(s.T_max > s.T_min))
            return fail(ctx, PNUC_ERR_ARG, "secondary tally: bad T bins or range");
        const uint64_t cells = 12ull * (uint64_t)s.n_cos * (uint64_t)s.n_T;
        if (cells > (1ull << 28)) return fail(ctx, PNUC_ERR_ARG, "secondary tally: %llu cells", (unsigned long long)cells);
        if (n_secondaries > 0 && !secondaries) return fail(ctx, PNUC_ERR_ARG, "null secondaries");
        if (n_secondaries > 0) {
            const double sT = (double)s.n_T / (s.T_max - s.T_min);
            const double hc = 0.5 * (double)s.n_cos;
            const uint64_t copies = cells * (kTallyBlock / 32) <= (uint64_t)kSmemBins ? kTallyBlock / 32 : 1;
            const size_t smem = cells <= (uint64_t)kSmemBins ? cells * copies * sizeof(unsigned int) : 0;
            secondary_tally_kernel<<<tally_grid(n_secondaries, ctx->sm_count), kTallyBlock, smem, st>>>(
                reinterpret_cast<const uint4 *>(secondaries), n_secondaries, s.T_min, sT, s.n_T, hc, s.n_cos,
                secondary_hist, (int)cells);
            CU(ctx, cudaGetLastError());
        }
    }
    if (residual_hist) {
        if (s.n_E < 1 || !(s.E_max > s.E_min) || s.Z_max < 0 || s.A_max < 0 || s.Z_max > 255 || s.A_max > 511)
            return fail(ctx, PNUC_ERR_ARG, "residual tally: bad E bins or (Z, A) range");
        const uint64_t cells = (uint64_t)s.n_E * (uint64_t)(s.Z_max + 1) * (uint64_t)(s.A_max + 1);
        if (cells > (1ull << 28)) return fail(ctx, PNUC_ERR_ARG, "residual tally: %llu cells", (unsigned long long)cells);
        if (n > 0 && (!residuals || !energies)) return fail(ctx, PNUC_ERR_ARG, "null residuals or energies");
        if (n > 0) {
            const double sE = (double)s.n_E / (s.E_max - s.E_min);
            const size_t smem = cells <= (uint64_t)kSmemBins ? cells * sizeof(unsigned int) : 0;
            residual_tally_kernel<<<tally_grid(n, ctx->sm_count), kTallyBlock, smem, st>>>(
                reinterpret_cast<const uint4 *>(residuals), energies, n, s.E_min, sE, s.n_E, s.Z_max, s.A_max,
                residual_hist, (int)cells);
            CU(ctx, cudaGetLastError());
        }
    }
    return PNUC_OK;
}
