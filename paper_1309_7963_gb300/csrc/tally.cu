// Yield tallies (pnuc_tally): histograms of a batch's secondaries by (origin, species,
// cos theta, T) and of its residual nuclei by (incident energy, Z, A), the outputs the paper
// plots (§4.1, Figs. 1-2) and the positron-emitter yields it proposes (§4.2).
//
// Both kernels are one streaming pass over the output records: coalesced 16-byte loads
// (the residual kernel reads only the first 32 bytes of each 64-byte record), per-block
// shared-memory histograms when the histogram fits, and warp-aggregated 64-bit atomics
// (lanes that hit the same cell add once) otherwise. The bin arithmetic is FP64 with
// explicit round-to-nearest operations, so the host can reproduce every bin index.
#include <algorithm>

#include "api_internal.h"

namespace pnuc {
namespace {

constexpr int kTallyBlock = 256;
constexpr int kSmemBins = 12288;  // 32-bit shared counters per block (48 KB)

__device__ __forceinline__ void add_cell(unsigned long long *hist, int idx)
{
    // lanes of the warp that reach here with the same cell add once
    const unsigned peers = __match_any_sync(__activemask(), idx);
    if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&hist[idx], (unsigned long long)__popc(peers));
}

__global__ void __launch_bounds__(kTallyBlock)
    secondary_tally_kernel(const uint4 *__restrict__ rec, uint64_t n, double T_min, double sT, int nT, double hc,
                           int ncos, unsigned long long *hist, int nbins)
{
    extern __shared__ unsigned int cells[];
    const bool priv = nbins <= kSmemBins;
    if (priv) {
        for (int i = threadIdx.x; i < nbins; i += blockDim.x) cells[i] = 0u;
        __syncthreads();
    }
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint4 a = __ldcs(rec + 2 * i), b = __ldcs(rec + 2 * i + 1);
        const unsigned sp = a.y & 0xffu, org = (a.y >> 8) & 0xffu;
        const double T = __hiloint2double((int)a.w, (int)a.z);
        const double t = __dmul_rn(__dsub_rn(T, T_min), sT);
        if (!(t >= 0.0 && t < (double)nT) || sp > 5u || org > 1u) continue;
        const double c = __dmul_rn((double)__uint_as_float(b.z) + 1.0, hc);
        int ic = c > 0.0 ? (int)c : 0;
        if (ic > ncos - 1) ic = ncos - 1;
        const int idx = (((int)org * 6 + (int)sp) * ncos + ic) * nT + (int)t;
        if (priv) atomicAdd(&cells[idx], 1u);
        else add_cell(hist, idx);
    }
    if (priv) {
        __syncthreads();
        for (int i = threadIdx.x; i < nbins; i += blockDim.x)
            if (cells[i]) atomicAdd(&hist[i], (unsigned long long)cells[i]);
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
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint4 a = __ldcs(res + 4 * i), b = __ldcs(res + 4 * i + 1);  // Z/A fields, then flags
        if (b.x & (PNUC_FLAG_BAD_INPUT | PNUC_FLAG_ATTEMPT_CAP)) continue;
        const double e = __dmul_rn(__dsub_rn(__ldcs(energies + i), E_min), sE);
        const int Z = (int)(a.y & 0xffffu), A = (int)(a.y >> 16);
        if (!(e >= 0.0 && e < (double)nE) || Z > Zmax || A > Amax) continue;
        const int idx = ((int)e * (Zmax + 1) + Z) * (Amax + 1) + A;
        if (priv) atomicAdd(&cells[idx], 1u);
        else add_cell(hist, idx);
    }
    if (priv) {
        __syncthreads();
        for (int i = threadIdx.x; i < nbins; i += blockDim.x)
            if (cells[i]) atomicAdd(&hist[i], (unsigned long long)cells[i]);
    }
}

int tally_grid(uint64_t n, int sm_count)
{
    const uint64_t need = (n + kTallyBlock - 1) / kTallyBlock;
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(need, (uint64_t)sm_count * 8));
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
            const size_t smem = cells <= (uint64_t)kSmemBins ? cells * sizeof(unsigned int) : 0;
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
