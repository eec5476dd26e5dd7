// Yield tallies (pnuc_tally, pnuc_tally_windows): histograms of a batch's secondaries by
// (origin, species, cos theta or angular window, T) and of its residual nuclei by (incident
// energy, Z, A), the outputs the paper plots (§4.1, Figs. 1-2) and the positron-emitter
// yields it proposes (§4.2).
//
// Both kernels are one streaming pass over the output records: coalesced 16-byte loads
// (the residual kernel asks for the first 32 bytes of each 64-byte record, though DRAM
// returns the whole record), shared-memory counters per block when the histogram fits (four
// 256-thread blocks per SM up to 48 KB of counters, one 1024-thread block per SM up to the
// block limit of 227 KB), and warp-aggregated 64-bit global atomics (lanes that hit the same
// cell add once) otherwise. The bins are those of FP64 arithmetic with each operation rounded
// to nearest (so the host can reproduce every bin index); the kernels decide almost every bin
// in FP32 with a proven error bound and fall back to the FP64 expression only near a bin edge
// (bin_of below), keeping the FP64 pipe, GB300's scarce one, free; floors and range tests
// come from bit fields on the integer pipes.
#include <algorithm>
#include <climits>
#include <cmath>

#include "api_internal.h"
#include "fpconv.h"

namespace pnuc {
namespace {

constexpr int kTallyBlock = 256;
constexpr int kSmemBins = 12288;  // 32-bit shared counters of a 256-thread block (48 KB)
constexpr int kUnroll = 4;        // records in flight per thread
constexpr int kBlocksPerSM = 4;   // resident blocks per SM

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

// One axis of a histogram: bin t = RN(RN(x - x0) * s) in FP64, floor taken by floor_bits,
// bins 0 .. n-1. The FP32 copy of the map decides the bin when it provably agrees.
struct BinMap {
    double x0, s;
    float x0f, sf;   // x0 and s rounded to FP32
    float errs;      // s * 2^-20 rounded up
    float abs_err;   // max(s * 2^-120, 2^-126) rounded up
    int n;
    int fast;        // 0: every bin from the FP64 expression (parameters outside the proof's range)
};

// Bin of x (xf: x rounded to FP32 to nearest, or flushed to zero below the smallest normal
// float). Error bound, with u = 2^-24 and B = s * (|x| + |x0|):
//   the FP32 value t = RN32(RN32(xf - x0f) * sf) is within 4.0002 u B of the exact (x - x0) s
//   (relative roundings in xf, x0f, the subtraction, sf and the product), plus less than
//   2 s 2^-126 + 2^-149 from values below the normal range;
//   the FP64 value is within 2^-52 B (+ 2^-1074 s) of the exact one.
// err >= 16 u B (1 - 5u) + abs_err, with abs_err >= max(64 s 2^-126, 2^-126), exceeds the
// sum by a factor of about 4. So when t lies farther than err from every integer, t and the
// FP64 value have the same floor; below -err or above n + err both are out of range. The
// distances t - f and (f + 1) - t are exact for t >= 1/2 (Sterbenz); for 0 <= t < 1/2 the
// upper distance 1 - t exceeds 1/2 > t > err whenever the lower test passes; a NaN or an
// infinity fails every comparison. What is left (about 2 err of each unit interval) takes
// the FP64 expression.
__device__ __forceinline__ int bin_of(float xf, double x, const BinMap &m)
{
    if (m.fast) {
        const float t = __fmul_rn(__fsub_rn(xf, m.x0f), m.sf);
        const float err = __fadd_rn(__fmul_rn(__fadd_rn(fabsf(xf), fabsf(m.x0f)), m.errs), m.abs_err);
        if (__fadd_rn(t, err) < 0.f) return -1;
        if (__fsub_rn(t, err) > (float)m.n) return m.n;
        const float f = floorf(t);
        if (__fsub_rn(t, f) > err && __fsub_rn(__fadd_rn(f, 1.f), t) > err) return (int)f;
    }
    return floor_bits(__dmul_rn(__dsub_rn(x, m.x0), m.s));
}

__device__ __forceinline__ void add_cell(unsigned long long *hist, int idx)
{
    // lanes of the warp that reach here with the same cell add once
    const unsigned peers = __match_any_sync(__activemask(), idx);
    if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&hist[idx], (unsigned long long)__popc(peers));
}

__device__ __forceinline__ void add_cell_shared(unsigned int *cells, int idx)
{
    // one shared atomic per record: lanes that add to one address serialise in the atomic
    // unit, but that costs less than finding them first (__match_any_sync runs on the SM's
    // address-divergence pipe, which it kept 75% busy; measured 17% slower over the pass)
    atomicAdd(&cells[idx], 1u);
}

// Angular windows of pnuc_tally_windows: window k holds lo[k] <= uz < hi[k], the edges being
// the smallest floats at or above the caller's double edges (for a float uz, uz >= c exactly
// when uz >= that float of c), so the test is two FP32 comparisons and exact.
struct Windows {
    float lo[PNUC_MAX_WINDOWS], hi[PNUC_MAX_WINDOWS];
    int n;
};

// kWin: the second axis is the window of uz (records in none are skipped), else ncos uniform
// bins of cos theta (ncos = 1: angle-integrated).
template <int kBlock, bool kWin>
__global__ void __launch_bounds__(kBlock)
    secondary_tally_kernel(const uint4 *__restrict__ rec, uint64_t n, const BinMap mT, const BinMap mc, int ncos,
                           const Windows W, unsigned long long *hist, int nbins, int copies)
{
    // shared counters: two copies per block when they fit (odd and even warps), else one;
    // more copies (one per warp) measured no faster and leave less of the SM's 256 KB to L1
    extern __shared__ unsigned int cells[];
    const bool priv = copies > 0;
    const int total = nbins * copies;
    if (priv) {
        for (int i = threadIdx.x; i < total; i += blockDim.x) cells[i] = 0u;
        __syncthreads();
    }
    unsigned int *mine = cells + (copies > 1 ? (int)((threadIdx.x >> 5) & 1) * nbins : 0);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const int nT = mT.n;
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
            const int iT = bin_of(d2f(T), T, mT);
            if (iT < 0 || iT >= nT || sp > 5u || org > 1u) continue;
            int ic = 0;
            if (kWin) {
                const float c = __uint_as_float(b.z);
                ic = -1;
                for (int k = 0; k < W.n; ++k)
                    if (c >= W.lo[k] && c < W.hi[k]) {
                        ic = k;
                        break;
                    }
                if (ic < 0) continue;
            } else if (ncos > 1) {
                const float c = __uint_as_float(b.z);  // x - x0 = uz + 1, exact in FP64
                ic = bin_of(c, f2d(c), mc);
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

template <int kBlock>
__global__ void __launch_bounds__(kBlock)
    residual_tally_kernel(const uint4 *__restrict__ res, const double *__restrict__ energies, uint64_t n,
                          const BinMap mE, int Zmax, int Amax, unsigned long long *hist, int nbins, int shared)
{
    extern __shared__ unsigned int cells[];
    const bool priv = shared != 0;
    if (priv) {
        for (int i = threadIdx.x; i < nbins; i += blockDim.x) cells[i] = 0u;
        __syncthreads();
    }
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const int nE = mE.n;
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
            const int iE = bin_of(d2f(re[u]), re[u], mE);
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

template <typename K>
cudaError_t allow_shared(K kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) (void)cudaGetLastError();  // leave no error pending for the next launch's check
    return e;
}

// Launch shape of a pass over n records with a histogram of nbins cells: 256-thread blocks,
// four per SM, with their counters in shared memory when two copies (else one) fit 48 KB;
// else one 1024-thread block per SM (the same 32 warps) when one copy fits the block's
// shared-memory limit; else the 256-thread blocks with global atomics. 32 resident warps per
// SM keep enough loads in flight (16 measured 18% slower, 48 or 64 no faster); each block
// adds its counters to the histogram at its end.
struct TallyShape {
    int block, grid, copies;
    size_t smem;
};

TallyShape tally_shape(uint64_t n, uint64_t nbins, int max_copies, int sm_count, int smem_optin)
{
    TallyShape t{kTallyBlock, kBlocksPerSM, 0, 0};
    if (nbins * max_copies <= (uint64_t)kSmemBins) t.copies = max_copies;
    else if (nbins <= (uint64_t)kSmemBins) t.copies = 1;
    else if (nbins * sizeof(unsigned int) <= (uint64_t)smem_optin) t = TallyShape{1024, 1, 1, 0};
    t.smem = (size_t)(nbins * t.copies) * sizeof(unsigned int);
    const uint64_t need = (n + t.block - 1) / t.block;
    t.grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(need, (uint64_t)sm_count * t.grid));
    return t;
}

template <bool kWin>
pnuc_status launch_secondary(pnuc_ctx *ctx, const TallyShape &t, const uint4 *rec, uint64_t n, const BinMap &mT,
                             const BinMap &mc, int ncos, const Windows &W, unsigned long long *hist, int nbins,
                             cudaStream_t st)
{
    if (t.block == 1024) {
        CU(ctx, allow_shared(secondary_tally_kernel<1024, kWin>, t.smem));
        secondary_tally_kernel<1024, kWin><<<t.grid, 1024, t.smem, st>>>(rec, n, mT, mc, ncos, W, hist, nbins, t.copies);
    } else {
        secondary_tally_kernel<kTallyBlock, kWin>
            <<<t.grid, kTallyBlock, t.smem, st>>>(rec, n, mT, mc, ncos, W, hist, nbins, t.copies);
    }
    CU(ctx, cudaGetLastError());
    return PNUC_OK;
}

float round_up_f32(double v)
{
    float f = (float)v;
    if ((double)f < v) f = std::nextafter(f, INFINITY);
    return f;
}

// The map of bin_of, its FP32 decision enabled where the error bound holds: x0 zero or a
// normal float, s a normal float at least 2^-100 with s * 2^-20 finite, and n < 2^24 (so
// that n and f + 1 are exact in FP32).
BinMap bin_map(double x0, double s, int n)
{
    BinMap m{};
    m.x0 = x0;
    m.s = s;
    m.n = n;
    m.x0f = (float)x0;
    m.sf = (float)s;
    m.errs = round_up_f32(s * 0x1p-20);
    m.abs_err = std::max(round_up_f32(s * 0x1p-120), 0x1p-126f);
    m.fast = std::isfinite(m.x0f) && std::isfinite(m.sf) && std::isfinite(m.errs) && m.sf >= 0x1p-100f &&
             n < (1 << 24) && (x0 == 0.0 || std::fabs(x0) >= 0x1p-100);
    return m;
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
    int smem_optin = 0;
    CU(ctx, cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->cfg.device));
    if (secondary_hist) {
        if (s.n_T < 1 || s.n_cos < 1 || !(s.T_max > s.T_min))
            return fail(ctx, PNUC_ERR_ARG, "secondary tally: bad T bins or range");
        const uint64_t cells = 12ull * (uint64_t)s.n_cos * (uint64_t)s.n_T;
        if (cells > (1ull << 28)) return fail(ctx, PNUC_ERR_ARG, "secondary tally: %llu cells", (unsigned long long)cells);
        if (n_secondaries > 0 && !secondaries) return fail(ctx, PNUC_ERR_ARG, "null secondaries");
        if (n_secondaries > 0) {
            const double sT = (double)s.n_T / (s.T_max - s.T_min);
            const double hc = 0.5 * (double)s.n_cos;
            const TallyShape t = tally_shape(n_secondaries, cells, 2, ctx->sm_count, smem_optin);
            const BinMap mT = bin_map(s.T_min, sT, s.n_T), mc = bin_map(-1.0, hc, s.n_cos);
            const uint4 *rec = reinterpret_cast<const uint4 *>(secondaries);
            const pnuc_status ls = launch_secondary<false>(ctx, t, rec, n_secondaries, mT, mc, s.n_cos, Windows{},
                                                           secondary_hist, (int)cells, st);
            if (ls != PNUC_OK) return ls;
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
            const TallyShape t = tally_shape(n, cells, 1, ctx->sm_count, smem_optin);
            const BinMap mE = bin_map(s.E_min, sE, s.n_E);
            const uint4 *rr = reinterpret_cast<const uint4 *>(residuals);
            if (t.block == 1024) {
                CU(ctx, allow_shared(residual_tally_kernel<1024>, t.smem));
                residual_tally_kernel<1024><<<t.grid, 1024, t.smem, st>>>(rr, energies, n, mE, s.Z_max, s.A_max,
                                                                           residual_hist, (int)cells, t.copies);
            } else {
                residual_tally_kernel<kTallyBlock><<<t.grid, kTallyBlock, t.smem, st>>>(
                    rr, energies, n, mE, s.Z_max, s.A_max, residual_hist, (int)cells, t.copies);
            }
            CU(ctx, cudaGetLastError());
        }
    }
    return PNUC_OK;
}

extern "C" pnuc_status pnuc_tally_windows(pnuc_ctx *ctx, int32_t n_T, double T_min, double T_max, const double *cos_lo,
                                          const double *cos_hi, int32_t n_windows, const pnuc_secondary *secondaries,
                                          uint64_t n_secondaries, unsigned long long *hist, void *stream)
{
    if (!ctx || !cos_lo || !cos_hi || !hist) return fail(ctx, PNUC_ERR_ARG, "null argument");
    if (n_T < 1 || !(T_max > T_min)) return fail(ctx, PNUC_ERR_ARG, "window tally: bad T bins or range");
    if (n_windows < 1 || n_windows > PNUC_MAX_WINDOWS)
        return fail(ctx, PNUC_ERR_ARG, "window tally: %d windows (1 .. %d)", n_windows, PNUC_MAX_WINDOWS);
    Windows W{};
    W.n = n_windows;
    for (int k = 0; k < n_windows; ++k) {
        if (!std::isfinite(cos_lo[k]) || !std::isfinite(cos_hi[k]) || !(cos_lo[k] < cos_hi[k]))
            return fail(ctx, PNUC_ERR_ARG, "window tally: window %d is not a finite [lo, hi) with lo < hi", k);
        for (int j = 0; j < k; ++j)
            if (cos_lo[k] < cos_hi[j] && cos_lo[j] < cos_hi[k])
                return fail(ctx, PNUC_ERR_ARG, "window tally: windows %d and %d overlap", j, k);
        W.lo[k] = round_up_f32(cos_lo[k]);
        W.hi[k] = round_up_f32(cos_hi[k]);
    }
    const uint64_t cells = 12ull * (uint64_t)n_windows * (uint64_t)n_T;
    if (cells > (1ull << 28)) return fail(ctx, PNUC_ERR_ARG, "window tally: %llu cells", (unsigned long long)cells);
    if (n_secondaries == 0) return PNUC_OK;
    if (!secondaries) return fail(ctx, PNUC_ERR_ARG, "null secondaries");
    CU(ctx, cudaSetDevice(ctx->cfg.device));
    int smem_optin = 0;
    CU(ctx, cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->cfg.device));
    const TallyShape t = tally_shape(n_secondaries, cells, 2, ctx->sm_count, smem_optin);
    return launch_secondary<true>(ctx, t, reinterpret_cast<const uint4 *>(secondaries), n_secondaries,
                                  bin_map(T_min, (double)n_T / (T_max - T_min), n_T), BinMap{}, n_windows, W, hist,
                                  (int)cells, (cudaStream_t)stream);
}
