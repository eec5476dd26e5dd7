// Device-side model of one event (paper §2): nucleon transport through the 15-shell
// nucleus by delta tracking, NN collisions with Pauli blocking, cutoff and refraction,
// energy-balance excitation, then Weisskopf–Ewing evaporation. Written as a per-lane
// state machine so that the plain kernel (one event per thread) and the persistent
// kernel (warps refilling finished lanes) run the same steps.
//
// Precision: R = double reproduces the CPU oracle event by event (compiled without FMA
// contraction); R = float keeps transport, paths, cross sections, the channel parameters and
// the emission sampler in FP32 while the NN collision boosts, the Q-values, the event's
// energy/momentum bookkeeping and the evaporation widths with their exponentials stay FP64.
// The evaporation templates' kScaled variant (FP32 only) evaluates the widths in FP32, each
// scaled by the largest channel's exponential, and draws the channel in FP32.
#pragma once

#include <cooperative_groups.h>
#include <cstddef>

#include "expfixed.h"
#include "fpconv.h"
#include "pnuc_internal.h"

namespace pnuc {
namespace dev {
namespace {  // internal linkage: each kernel translation unit has its own copy

namespace cg = cooperative_groups;

constexpr double kE2 = 1.44;  // e^2, MeV fm
constexpr double kMp = 938.272, kMn = 939.565;
constexpr double kTwoPi = 6.283185307179586;

// ejectiles n, p, d, t, 3He, alpha (§2.4: He and lighter)
__constant__ double cEjM[6] = {kEjectileMass[0], kEjectileMass[1], kEjectileMass[2],
                               kEjectileMass[3], kEjectileMass[4], kEjectileMass[5]};
__constant__ double cEjG[6] = {2.0, 2.0, 3.0, 2.0, 2.0, 1.0};
__constant__ float cEjMf[6] = {939.565f, 938.272f, 1875.613f, 2808.921f, 2808.391f, 3727.379f};
__constant__ float cEjGf[6] = {2.f, 2.f, 3.f, 2.f, 2.f, 1.f};
__constant__ int cEjZ[6] = {kEjectileZ[0], kEjectileZ[1], kEjectileZ[2], kEjectileZ[3], kEjectileZ[4], kEjectileZ[5]};
__constant__ int cEjA[6] = {kEjectileA[0], kEjectileA[1], kEjectileA[2], kEjectileA[3], kEjectileA[4], kEjectileA[5]};

// kKinWait: an accepted candidate waits for its collision kinematics (batched per warp).
enum Phase : int { kIdle = 0, kEntry = 1, kTransport = 2, kEvap = 3, kFinish = 4, kExhausted = 5, kKinWait = 6 };

// ------------------------------------------------------------------ Philox4x64-10
// Salmon et al., SC'11: ten rounds, multipliers and Weyl key increments of the paper.
__device__ __forceinline__ void philox4x64_10(uint64_t c0, uint64_t c1, uint64_t k0, uint64_t k1, uint64_t &o0,
                                              uint64_t &o1, uint64_t &o2, uint64_t &o3)
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    uint64_t c2 = 0, c3 = 0;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B97F4A7C15ULL;
            k1 += 0xBB67AE8584CAA73BULL;
        }
        uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
        uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
        uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    o0 = c0;
    o1 = c1;
    o2 = c2;
    o3 = c3;
}

// A Philox block out of line, its four words returned by value (in registers): the
// evaporation's draws take it, since the evaporation kernel's loop is bound partly by
// instruction fetch and has three places that may generate (inline, the kernel ran 5%
// slower); the cascade kernel, with one such place, keeps it inline (1.5% faster).
struct PhiloxWords {
    uint64_t w[4];
};
__device__ __noinline__ PhiloxWords philox_block(uint64_t c0, uint64_t c1, uint64_t k0)
{
    PhiloxWords o;
    philox4x64_10(c0, c1, k0, 0, o.w[0], o.w[1], o.w[2], o.w[3]);
    return o;
}

// One 32-bit half h of a Philox word -> uniform in (0, 1).
template <typename R> __device__ __forceinline__ R to_uniform(uint32_t h);
template <> __device__ __forceinline__ double to_uniform<double>(uint32_t h)
{
    return ((double)h + 0.5) * 0x1p-32;  // 32 bits + 1/2: exact, open interval
}
template <> __device__ __forceinline__ float to_uniform<float>(uint32_t h)
{
    // (m + 1/2) 2^-23 for the top 23 bits m of h (the FP64 uniform on the float grid), built
    // as (1 + m 2^-23) - (1 - 2^-24): both operands and the difference are exact floats, and
    // no int->float conversion is needed
    return __uint_as_float(0x3f800000u | (h >> 9)) - 0x1.fffffep-1f;
}

// The event's draw stream: Philox((d div 8, event, 0, 0), (seed, 0)) gives 4 words = 8
// draws; draw d is half d mod 2 (the high 32 bits first) of word (d div 2) mod 4.
// Converted draws wait in a 32-slot ring in shared memory (slot k of thread t at
// buf[k * stride], stride = block size: conflict-free). Draws are generated only by
// ensure(k), which the kernels call once per loop iteration (and the evaporation sampler
// once per trial), so lanes generate together; ensure<true> generates through the
// out-of-line philox_block().
constexpr int kRing = 32;
constexpr int kDrawsPerBlock = 8;

template <typename R>
struct Stream {
    uint64_t seed, event;
    uint32_t block;
    int left, head;
    R *buf;
    int stride;
    __device__ void reset(uint64_t s, uint64_t e)
    {
        seed = s;
        event = e;
        block = 0;
        left = 0;
        head = 0;
    }
    // at least k (<= kRing - kDrawsPerBlock + 1) draws available afterwards
    template <bool kCall = false>
    __device__ __forceinline__ void ensure(int k)
    {
#pragma unroll 1
        while (left < k) {
            uint64_t w[4];
            if constexpr (kCall) {
                const PhiloxWords pw = philox_block(block, event, seed);
#pragma unroll
                for (int q = 0; q < 4; ++q) w[q] = pw.w[q];
            } else {
                philox4x64_10(block, event, seed, 0, w[0], w[1], w[2], w[3]);
            }
            ++block;
            const int t = head + left;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                buf[((t + 2 * q) & (kRing - 1)) * stride] = to_uniform<R>((uint32_t)(w[q] >> 32));
                buf[((t + 2 * q + 1) & (kRing - 1)) * stride] = to_uniform<R>((uint32_t)w[q]);
            }
            left += kDrawsPerBlock;
        }
    }
    // positions the stream at draw d (the next draw returned is draw d)
    __device__ void seek(uint64_t d)
    {
        block = (uint32_t)(d / kDrawsPerBlock);
        left = 0;
        head = 0;
        ensure<true>(kDrawsPerBlock);
        head = (int)(d % kDrawsPerBlock);
        left -= (int)(d % kDrawsPerBlock);
    }
    __device__ __forceinline__ uint32_t position() const
    {
        return (uint32_t)kDrawsPerBlock * block - (uint32_t)left;
    }
    __device__ __forceinline__ R next()
    {
        R u = buf[head * stride];
        head = (head + 1) & (kRing - 1);
        --left;
        return u;
    }
};

// ------------------------------------------------------------------ small helpers
template <typename R> __device__ __forceinline__ R dot3(const R *a, const R *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
// kinetic energy from |p|^2 without cancellation
template <typename R> __device__ __forceinline__ R kinetic(R p2, R m) { return p2 / (sqrt(p2 + m * m) + m); }
__device__ __forceinline__ double nucleon_mass(int s) { return s ? kMp : kMn; }
template <typename R> __device__ __forceinline__ R nucleon_mass_R(int s) { return s ? R(kMp) : R(kMn); }
// u^(1/3) for a uniform u in (0, 1): cbrt in FP64; in FP32 2^(log2(u) / 3) from the hardware
// base-2 logarithm and exponential (relative error of order 1e-7), in place of the library cbrtf
template <typename R> __device__ __forceinline__ R cbrt_uniform(R u) { return cbrt(u); }
template <> __device__ __forceinline__ float cbrt_uniform<float>(float u) { return exp2f(log2f(u) * (1.f / 3.f)); }

// Conversions: in FP32 mode on the integer pipes (fpconv.h), in FP64 mode plain casts.
template <typename R> __device__ __forceinline__ R to_R(double x) { return (R)x; }
template <> __device__ __forceinline__ float to_R<float>(double x) { return d2f(x); }
template <typename R> __device__ __forceinline__ double to_d(R x) { return (double)x; }
template <> __device__ __forceinline__ double to_d<float>(float x) { return f2d(x); }
template <typename R> __device__ __forceinline__ float out_f(double x) { return (float)x; }
template <> __device__ __forceinline__ float out_f<float>(double x) { return d2f(x); }
// ejectile mass and spin factor of channel j in precision R
template <typename R> __device__ __forceinline__ R ej_M(int j) { return cEjM[j]; }
template <> __device__ __forceinline__ float ej_M<float>(int j) { return cEjMf[j]; }
template <typename R> __device__ __forceinline__ R ej_G(int j) { return cEjG[j]; }
template <> __device__ __forceinline__ float ej_G<float>(int j) { return cEjGf[j]; }

// ------------------------------------------------------------------ NN cross sections (§2.3, Cugnon et al.)
template <typename R> __device__ __forceinline__ R clamp_p(R p) { return p < R(0.1) ? R(0.1) : (p > R(2.0) ? R(2.0) : p); }

template <typename R>
__device__ R sigma_nn(bool like, R p)  // p in GeV/c -> mb
{
    p = clamp_p(p);
    if (like) {
        if (p < R(0.44)) return R(34.0) * pow(p / R(0.4), R(-2.104));
        if (p < R(0.8)) {
            R d = p - R(0.7);
            return R(23.5) + R(1000.0) * d * d * d * d;
        }
        R d = p - R(1.3);
        return R(1250.0) / (p + R(50.0)) - R(4.0) * d * d;
    }
    if (p < R(0.8)) return R(33.0) + R(196.0) * pow(fabs(p - R(0.95)), R(2.5));
    return R(31.0) / sqrt(p);
}

__device__ double slope_nn(bool like, double p)  // (GeV/c)^-2
{
    if (like) {
        double p8 = p * p;
        p8 = p8 * p8;
        p8 = p8 * p8;
        return 5.5 * p8 / (7.7 + p8);
    }
    if (p < 0.225) return 0.0;
    if (p < 0.6) return 16.53 * (p - 0.225);
    if (p < 1.6) return 7.16 - 1.63 * p;
    return 4.552;
}

// Majorant of sigma * v_rel * E1 (GeV mb) over the shell's Fermi partners (v <= vF):
// p_lab lies in [p_lo, p_hi] and sigma v_rel E1 <= p_lab sigma(p_lab), bounded piecewise.
template <typename R>
__device__ R g_hat(R p1, R E1, R vF)
{
    R plo = (p1 - vF * E1) * R(1e-3);
    if (plo < R(0)) plo = R(0);
    R phi = (p1 + vF * E1) * R(1e-3) / sqrt((R(1) - vF) * (R(1) + vF));
    R pc = clamp_p(plo);
    R glo = pc < R(0.44) ? pc * sigma_nn<R>(true, pc) : R(0);
    R ph = phi > R(0.8) ? phi : R(0.8);
    R g1 = R(28.1) * ph;
    R g2 = R(31.0) * ph / sqrt(ph < R(2.0) ? ph : R(2.0));
    R g = R(31.0);
    if (glo > g) g = glo;
    if (g1 > g) g = g1;
    if (g2 > g) g = g2;
    return g;
}

// ------------------------------------------------------------------ geometry (§2.3)
// Distance to the boundary of shell i along unit d; dir = -1 inward, +1 outward.
template <typename R>
__device__ R boundary_distance(const ShellTable<R> &t, int shell, const R *r, const R *d, int &dir)
{
    R beta = dot3(r, d), q = dot3(r, r);
    if (shell > 0 && beta < R(0)) {
        R ri = t.r[shell];
        R c = q - ri * ri, D = beta * beta - c;
        if (D > R(0)) {
            dir = -1;
            R s = c / (-beta + sqrt(D));
            return s > R(0) ? s : R(0);
        }
    }
    R ro = t.r[shell + 1];
    R c = q - ro * ro;
    dir = 1;
    // moving inward the particle is on or inside its outer sphere: rounding that puts it
    // outside must not shorten the chord (else it bounces in place at a grazing reflection)
    if (beta <= R(0)) return -beta + sqrt(beta * beta - (c > R(0) ? R(0) : c));
    R D = beta * beta - c;
    if (D < R(0)) D = R(0);
    R s = -c / (beta + sqrt(D));
    return s > R(0) ? s : R(0);
}

// FP32 mode only: after a crossing the momentum's component along n points the way the
// particle now goes, back (reflection) or on (refraction), with at least kGrazeFloor of |p|
// (1 mrad from the tangent plane). A specular reflection inside a sphere keeps its angle to the
// surface, so a near-tangent one bounces along chords of about 2 R theta, one step each; in
// FP32 a tangent one can round to zero-length chords that repeat until the step cap (one
// p-208Pb event in 1e6 did). The FP64 mode, like the model, has no floor (the FP64 model
// reached the step cap in none of 1.5e7 heavy-target events). The tests use the exact scalars
// already at hand; the root only when the floor applies.
constexpr double kGrazeFloor = 1e-3;

// Potential step (after Chen et al.): kinetic energy changes by dT at fixed tangential
// momentum; reflection when that is impossible. dir: +1 for a crossing outward (along n),
// -1 inward: the refracted normal component takes its sign. Returns true if refracted.
template <typename R>
__device__ bool refract(const R *n, R *p, R m, R dT, int dir)
{
    R pp = dot3(p, p);
    R T = kinetic(pp, m), Tn = T + dT;
    R pn = dot3(p, n);
    R q2 = pn * pn + (Tn - T) * (Tn + T + R(2) * m);
    if constexpr (sizeof(R) == 8) {
        if (Tn <= 0.0 || q2 <= 0.0) {
#pragma unroll
            for (int k = 0; k < 3; ++k) p[k] -= 2.0 * pn * n[k];
            return false;
        }
        const double pnn = dir * sqrt(q2);
#pragma unroll
        for (int k = 0; k < 3; ++k) p[k] += (pnn - pn) * n[k];
        return true;
    } else {
        const R floor2 = R(kGrazeFloor * kGrazeFloor);
        if (Tn <= R(0) || q2 <= R(0)) {
            const R to = pn * pn < floor2 * pp ? R(-dir) * (R(kGrazeFloor) * sqrt(pp)) : -pn;
#pragma unroll
            for (int k = 0; k < 3; ++k) p[k] += (to - pn) * n[k];
            return false;
        }
        const R p2n = pp - pn * pn + q2;  // |p|^2 after the crossing
        const R pnn = q2 < floor2 * p2n ? R(dir) * (R(kGrazeFloor) * sqrt(p2n)) : R(dir) * sqrt(q2);
#pragma unroll
        for (int k = 0; k < 3; ++k) p[k] += (pnn - pn) * n[k];
        return true;
    }
}

// ------------------------------------------------------------------ NN collision kinematics (FP64)
__device__ void boost(const double *beta, double gamma, double sign, double e, const double *p, double *po)
{
    double bp = dot3(beta, p);
    double g2 = gamma * gamma / (gamma + 1.0);
    double f = g2 * bp + sign * gamma * e;
#pragma unroll
    for (int k = 0; k < 3; ++k) po[k] = p[k] + beta[k] * f;
}

__device__ void rotate(const double *n, double ct, double st, double phi, double *d)
{
    double rho = sqrt(n[0] * n[0] + n[1] * n[1]);
    double sp, cp;
    sincos(phi, &sp, &cp);
    if (rho > 0.0) {
        double e1x = n[0] * n[2] / rho, e1y = n[1] * n[2] / rho, e1z = -rho;
        double e2x = -n[1] / rho, e2y = n[0] / rho;
        d[0] = ct * n[0] + st * (cp * e1x + sp * e2x);
        d[1] = ct * n[1] + st * (cp * e1y + sp * e2y);
        d[2] = ct * n[2] + st * (cp * e1z + sp * 0.0);
    } else {
        d[0] = st * cp;
        d[1] = st * sp;
        d[2] = (n[2] >= 0.0 ? 1.0 : -1.0) * ct;
    }
}

// Elastic collision of (s1, p1) on (s2, p2), relativistic; uniforms for t, phi*, flip.
__device__ void collide(int s1, const double *p1, int s2, const double *p2, double ut, double uphi, double uf,
                        double *q1, double *q2)
{
    double m1 = nucleon_mass(s1), m2 = nucleon_mass(s2);
    bool like = s1 == s2;
    double pp1 = dot3(p1, p1), pp2 = dot3(p2, p2);
    double E1 = sqrt(pp1 + m1 * m1), E2 = sqrt(pp2 + m2 * m2);
    double T1 = kinetic(pp1, m1), T2 = kinetic(pp2, m2);
    double X = T1 * T2 + T1 * m2 + T2 * m1 - dot3(p1, p2);
    if (X < 0.0) X = 0.0;
    double k = sqrt(X * (X + 2.0 * m1 * m2));
    double plab = k / m2;
    double rs = sqrt((m1 + m2) * (m1 + m2) + 2.0 * X);
    double pst = k / rs;
    double Et = E1 + E2;
    double beta[3] = {(p1[0] + p2[0]) / Et, (p1[1] + p2[1]) / Et, (p1[2] + p2[2]) / Et};
    double gamma = Et / rs;
    double p1c[3];
    boost(beta, gamma, -1.0, E1, p1, p1c);
    double nrm = sqrt(dot3(p1c, p1c));
    double n[3] = {p1c[0] / nrm, p1c[1] / nrm, p1c[2] / nrm};
    double B = slope_nn(like, plab * 1e-3);
    double pg = pst * 1e-3;
    double b = 4.0 * B * pg * pg;
    double y = b > 0.0 ? -log1p(ut * expm1(-b)) / b : ut;
    double ct = 1.0 - 2.0 * y;
    if (!like) {
        double pl = plab * 1e-3;
        double a = pl <= 0.8 ? 1.0 : (0.8 / pl) * (0.8 / pl);
        if (uf < a / (1.0 + a)) ct = -ct;
    }
    double st = sqrt((1.0 - ct) * (1.0 + ct));
    double d[3];
    rotate(n, ct, st, kTwoPi * uphi, d);
    double k1[3] = {pst * d[0], pst * d[1], pst * d[2]};
    double k2[3] = {-k1[0], -k1[1], -k1[2]};
    double e1 = sqrt(pst * pst + m1 * m1), e2 = sqrt(pst * pst + m2 * m2);
    boost(beta, gamma, 1.0, e1, k1, q1);
    boost(beta, gamma, 1.0, e2, k2, q2);
}

// ------------------------------------------------------------------ per-lane state
// Per-target scalars the steps need, staged in shared memory beside the shell tables.
struct TargetScalars {
    double M;  // SEMF mass of the target, MeV
    double R;  // nuclear radius, fm
    int32_t Z, A;
};

template <typename R>
struct Particle {
    R r[3], p[3];
    int s, shell;
};

template <typename R>
struct Lane {
    Stream<R> rng;
    uint32_t ev;
    int tgt;
    int phase;
    double T0;
    int proj;  // incident nucleon: 1 proton, 0 neutron
    // particle in flight
    R r[3], p[3];
    int s, shell, sp;
    // accepted candidate waiting for its kinematics: the partner's momentum and species
    R jp[3];
    int js;
    // event bookkeeping (FP64)
    int steps, attempts, n_coll, n_index, n_esc, n_p_esc, n_evap;
    uint32_t flags;
    uint32_t pend;  // 1 + the draw index at which a pending evaporation resumes, else 0
    double Esum, Px, Py, Pz;
    // residual / evaporation
    int Z, A, Zc, Ac;
    double Estar, Estar_c, Er, Prx, Pry, Prz;
};

template <bool kCount>
struct Counters {
    unsigned long long *s;  // shared-memory block counters
    __device__ void add(int k, unsigned v = 1)
    {
        if (kCount) atomicAdd(&s[k], (unsigned long long)v);
    }
};

// The 32-byte secondary record (pnuc_secondary) as two 16-byte halves.
__device__ __forceinline__ void pack_secondary(uint32_t ev, int species, int origin, int index, double T, float ux,
                                               float uy, float uz, uint4 &a, uint4 &b)
{
    const unsigned long long tbits = (unsigned long long)__double_as_longlong(T);
    a = make_uint4(ev, (uint32_t)species | ((uint32_t)origin << 8) | ((uint32_t)index << 16), (uint32_t)tbits,
                   (uint32_t)(tbits >> 32));
    b = make_uint4(__float_as_uint(ux), __float_as_uint(uy), __float_as_uint(uz), 0u);
}

// Warp-aggregated reservation of one output slot per calling lane: one atomic per
// converged group, then 2 x 16-byte stores of the 32-byte record.
__device__ __forceinline__ void emit_secondary(const SimParams &P, uint32_t ev, int species, int origin, int index,
                                               double T, float ux, float uy, float uz, uint32_t &flags)
{
    cg::coalesced_group g = cg::coalesced_threads();
    unsigned long long base = 0;
    if (g.thread_rank() == 0) base = atomicAdd(P.sec_count, (unsigned long long)g.size());
    base = g.shfl(base, 0);
    unsigned long long slot = base + g.thread_rank();
    if (slot >= P.sec_cap) {
        flags |= PNUC_FLAG_OUTPUT_OVERFLOW;
        return;
    }
    uint4 a, b;
    pack_secondary(ev, species, origin, index, T, ux, uy, uz, a, b);
    uint4 *dst = reinterpret_cast<uint4 *>(P.sec + slot);
    dst[0] = a;
    dst[1] = b;
}

// Emission as the record is made (the plain and sorted methods).
struct EmitNow {
    __device__ __forceinline__ void emit(const SimParams &P, uint32_t ev, int species, int origin, int index, double T,
                                         float ux, float uy, float uz, uint32_t &flags)
    {
        emit_secondary(P, ev, species, origin, index, T, ux, uy, uz, flags);
    }
};

// Emission in the persistent evaporation kernel, whose lanes emit at most one record per loop
// iteration. The converged group reserves its slots with one atomic when the record is made,
// the record waits in the thread's staging slot in shared memory, and store(), at the top of
// the next iteration, writes it: no warp waits for the atomic's result in the middle of a step
// (a global atomic on one counter returns after hundreds of cycles; an iteration later it
// has). A record past the output's capacity flags the lane's event there, before the event's
// residual is written. The slots are the same dense range [0, count) as with EmitNow.
struct DeferredEmit {
    uint4 *stage;             // the thread's two 16-byte halves: stage[0] and stage[stride]
    int stride;
    unsigned long long base;  // the group's first slot (held by the group's first lane)
    uint32_t tag = 0;         // 0: nothing staged; else 1 | first lane << 1 | rank << 6
    __device__ __forceinline__ void emit(const SimParams &P, uint32_t ev, int species, int origin, int index, double T,
                                         float ux, float uy, float uz, uint32_t &)
    {
        const unsigned m = __activemask(), lane = threadIdx.x & 31;
        const unsigned first = (unsigned)__ffs(m) - 1u, rank = __popc(m & ((1u << lane) - 1u));
        if (lane == first) base = atomicAdd(P.sec_count, (unsigned long long)__popc(m));
        uint4 a, b;
        pack_secondary(ev, species, origin, index, T, ux, uy, uz, a, b);
        stage[0] = a;
        stage[stride] = b;
        tag = 1u | (first << 1) | (rank << 6);
    }
    // called by all 32 lanes of the warp
    __device__ __forceinline__ void store(const SimParams &P, uint32_t &flags)
    {
        const unsigned FULL = 0xffffffffu;
        if (!__any_sync(FULL, tag != 0)) return;
        const unsigned long long b = __shfl_sync(FULL, base, (tag >> 1) & 31u);
        if (tag) {
            const unsigned long long slot = b + (tag >> 6);
            if (slot < P.sec_cap) {
                uint4 *dst = reinterpret_cast<uint4 *>(P.sec + slot);
                dst[0] = stage[0];
                dst[1] = stage[stride];
            } else {
                flags |= PNUC_FLAG_OUTPUT_OVERFLOW;
            }
            tag = 0;
        }
    }
};

// A residual record with a pending evaporation (persistent method, between its two kernels)
// carries the escape sums at full precision: Esum in Estar_cascade, Pz in Estar_final, Px and
// Py in the 16 bytes from P_cascade[0].
static_assert(offsetof(pnuc_residual, P_cascade) == 40 && sizeof(pnuc_residual) == 64, "residual layout");

__device__ __forceinline__ void write_pending_sums(pnuc_residual &o, double Esum, double Px, double Py, double Pz)
{
    o.Estar_cascade = Esum;
    o.Estar_final = Pz;
    unsigned char *b = reinterpret_cast<unsigned char *>(&o);
    memcpy(b + 40, &Px, 8);
    memcpy(b + 48, &Py, 8);
}

__device__ __forceinline__ void read_pending_sums(const pnuc_residual &o, double &Esum, double &Px, double &Py,
                                                  double &Pz)
{
    Esum = o.Estar_cascade;
    Pz = o.Estar_final;
    const unsigned char *b = reinterpret_cast<const unsigned char *>(&o);
    memcpy(&Px, b + 40, 8);
    memcpy(&Py, b + 48, 8);
}

template <typename R>
__device__ void write_residual(const SimParams &P, const Lane<R> &L)
{
    alignas(16) pnuc_residual o;
    o.Z_cascade = (uint16_t)L.Zc;
    o.A_cascade = (uint16_t)L.Ac;
    o.Z_final = (uint16_t)L.Z;
    o.A_final = (uint16_t)L.A;
    o.n_cascade = (uint16_t)min(L.n_esc, 65535);
    o.n_evaporated = (uint16_t)min(L.n_evap, 65535);
    o.n_collisions = (uint16_t)min(L.n_coll, 65535);
    o.n_attempts = (uint16_t)min(L.attempts, 65535);
    o.flags = L.flags;
    o.reserved = L.pend;
    if (L.pend) {
        write_pending_sums(o, L.Esum, L.Px, L.Py, L.Pz);
        o.P_final[1] = o.P_final[2] = 0.f;
    } else {
        o.Estar_cascade = L.Estar_c;
        o.Estar_final = L.Estar;
        o.P_cascade[0] = out_f<R>(L.Px);  // set by settle_cascade; zero for events without a cascade
        o.P_cascade[1] = out_f<R>(L.Py);
        o.P_cascade[2] = out_f<R>(L.Pz);
        o.P_final[0] = out_f<R>(L.Prx);
        o.P_final[1] = out_f<R>(L.Pry);
        o.P_final[2] = out_f<R>(L.Prz);
    }
    const uint4 *src = reinterpret_cast<const uint4 *>(&o);
    uint4 *dst = reinterpret_cast<uint4 *>(P.res + L.ev);
#pragma unroll
    for (int k = 0; k < 4; ++k) dst[k] = src[k];
}

// Id of event ev of the launch: the batch's per-event id if it has them; else its position in
// its segment plus the segment's first id (merged serving requests); else first_event_id + ev.
__device__ __forceinline__ unsigned long long event_id(const SimParams &P, uint32_t ev)
{
    if (P.event_ids) return __ldg(&P.event_ids[ev]);
    if (P.n_seg <= 0) return P.first_event_id + ev;
    int lo = 0, hi = P.n_seg - 1;  // the last segment k with seg_start[k] <= ev
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&P.seg_start[mid]) <= ev) lo = mid;
        else hi = mid - 1;
    }
    return __ldg(&P.seg_first[lo]) + (ev - __ldg(&P.seg_start[lo]));
}

// Starts event ev in lane L (reads its energy and target id).
template <typename R>
__device__ void begin_event(const SimParams &P, const TargetScalars *tabs, Lane<R> &L, uint32_t ev)
{
    L.ev = ev;
    L.rng.reset(P.seed, event_id(P, ev));
    L.T0 = __ldg(&P.energies[ev]);
    L.tgt = __ldg(&P.target_ids[ev]);
    L.proj = P.projectiles ? (int)__ldg(&P.projectiles[ev]) : 1;
    L.steps = L.attempts = L.n_coll = L.n_index = L.n_esc = L.n_p_esc = L.n_evap = 0;
    L.flags = 0;
    L.pend = 0;
    L.Esum = L.Px = L.Py = L.Pz = 0.0;
    L.Estar = L.Estar_c = 0.0;
    L.Er = L.Prx = L.Pry = L.Prz = 0.0;
    L.sp = 0;
    bool tgt_ok = L.tgt >= 0 && L.tgt < P.n_targets;
    L.Z = L.Zc = tgt_ok ? tabs[L.tgt].Z : 0;
    L.A = L.Ac = tgt_ok ? tabs[L.tgt].A : 0;
    const R T0r = to_R<R>(L.T0);
    if (!tgt_ok || !(T0r >= R(20) && T0r <= R(250)) || (L.proj != 0 && L.proj != 1)) {
        L.flags = PNUC_FLAG_BAD_INPUT;
        L.phase = kFinish;
        return;
    }
    L.phase = kEntry;
}

// Entry on the projected disk of radius R, refracted into the surface shell.
template <typename R, bool kCount>
__device__ void step_entry(const SimParams &P, const ShellTable<R> &t, double Rad, Lane<R> &L, Counters<kCount> &C)
{
    if (L.attempts >= P.max_attempts) {
        L.flags |= PNUC_FLAG_ATTEMPT_CAP;
        L.phase = kFinish;
        return;
    }
    ++L.attempts;
    C.add(PNUC_C_ATTEMPTS);
    R Rr = to_R<R>(Rad);
    R b = Rr * sqrt(L.rng.next());
    R phi = R(kTwoPi) * L.rng.next();
    R sphi, cphi;
    sincos(phi, &sphi, &cphi);
    L.r[0] = b * cphi;
    L.r[1] = b * sphi;
    L.r[2] = -sqrt(Rr * Rr - b * b);
    const R T0 = to_R<R>(L.T0);
    L.p[0] = R(0);
    L.p[1] = R(0);
    const R mproj = nucleon_mass_R<R>(L.proj);
    L.p[2] = sqrt(T0 * T0 + R(2) * T0 * mproj);
    R rr = sqrt(dot3(L.r, L.r));
    R n[3] = {L.r[0] / rr, L.r[1] / rr, L.r[2] / rr};
    refract(n, L.p, mproj, t.V[L.proj][kShells - 1], -1);
    L.s = L.proj;
    L.shell = kShells - 1;
    L.sp = 0;
    L.phase = kTransport;
}

// E* from the energy balance once the cascade is over: the static mean field takes the
// momentum imbalance (kept in Px..Pz from here on) and the residual evaporates from rest.
// Needs the cascade residual's Z, A in L.Z, L.A, the projectile energy in L.T0 and the
// escape sums Esum, Px..Pz; Mt is the target's mass.
template <typename R>
__device__ void settle_cascade(const SimParams &P, double Mt, Lane<R> &L)
{
    const int Z = L.Z, A = L.A;
    const double mproj = nucleon_mass(L.proj);
    double p0 = sqrt(L.T0 * L.T0 + 2.0 * L.T0 * mproj);
    L.Px = -L.Px;
    L.Py = -L.Py;
    L.Pz = p0 - L.Pz;
    double Er = L.T0 + mproj + Mt - L.Esum;
    L.Er = Er;
    L.Prx = L.Pry = L.Prz = 0.0;
    if (Z < 1 || A - Z < 1) {
        L.flags |= PNUC_FLAG_BAD_RESIDUAL;
        L.phase = kFinish;
        return;
    }
    const double Mc = __ldg(&P.mass[Z * kMassA + A]);
    double Estar = Er - Mc;
    L.Estar = L.Estar_c = Estar;
    if (!(Estar > 0.0)) {
        L.flags |= PNUC_FLAG_NO_EXCITATION;
        L.phase = kFinish;
        return;
    }
    L.Er = Mc + Estar;  // the excited residual at rest: its total energy is M + E*
    L.phase = kEvap;
}

// The cascade of this attempt is over: retry if it was elastic (unless forced by the
// step cap), else settle E*, here or (kSplit: the persistent method) in the evaporation
// kernel, whose lanes do it together when they take the event. kSplit is a compile-time
// choice so that the cascade kernel keeps no evaporation state in registers.
template <typename R, bool kSplit>
__device__ void end_cascade(const SimParams &P, const TargetScalars &tab, Lane<R> &L, bool force)
{
    if (L.n_coll == 0 && !force) {
        L.phase = kEntry;
        return;
    }
    L.Z = L.Zc = tab.Z + L.proj - L.n_p_esc;
    L.A = L.Ac = tab.A + 1 - L.n_esc;
    if (kSplit) {
        // the residual record carries the raw escape sums and the draw position
        L.pend = L.rng.position() + 1u;
        L.phase = kFinish;
        return;
    }
    settle_cascade(P, tab.M, L);
}

// Resumes event ev from the residual record the cascade kernel wrote (the evaporation
// kernel of the persistent method): settles E*, then evaporates. Leaves the lane idle if
// nothing is pending.
template <typename R>
__device__ void begin_evap(const SimParams &P, Lane<R> &L, uint32_t ev)
{
    const uint4 *src = reinterpret_cast<const uint4 *>(P.res + ev);
    alignas(16) pnuc_residual o;
    uint4 *dst = reinterpret_cast<uint4 *>(&o);
#pragma unroll
    for (int k = 0; k < 4; ++k) dst[k] = src[k];
    if (o.reserved == 0) {
        L.phase = kIdle;
        return;
    }
    L.ev = ev;
    L.Z = L.Zc = o.Z_cascade;
    L.A = L.Ac = o.A_cascade;
    L.n_esc = L.n_index = o.n_cascade;
    L.n_coll = o.n_collisions;
    L.attempts = o.n_attempts;
    L.n_evap = 0;
    L.flags = o.flags;
    L.pend = 0;
    L.Estar = L.Estar_c = 0.0;
    read_pending_sums(o, L.Esum, L.Px, L.Py, L.Pz);
    L.T0 = __ldg(&P.energies[ev]);
    const int tgt = __ldg(&P.target_ids[ev]);
    L.proj = P.projectiles ? (int)__ldg(&P.projectiles[ev]) : 1;
    L.rng.reset(P.seed, event_id(P, ev));
    L.rng.seek(o.reserved - 1u);
    if (tgt < 0 || tgt >= P.n_targets) {  // cannot happen: the cascade checked it
        L.flags |= PNUC_FLAG_BAD_INPUT;
        L.phase = kFinish;
        return;
    }
    settle_cascade(P, __ldg(&P.tables[tgt].M), L);
}

// Pops the next particle of the stack, or ends the attempt.
template <typename R, bool kSplit>
__device__ __forceinline__ void next_particle(const SimParams &P, const TargetScalars &tab, Lane<R> &L, Particle<R> *stack)
{
    if (L.sp > 0) {
        const Particle<R> &q = stack[--L.sp];
        L.r[0] = q.r[0];
        L.r[1] = q.r[1];
        L.r[2] = q.r[2];
        L.p[0] = q.p[0];
        L.p[1] = q.p[1];
        L.p[2] = q.p[2];
        L.s = q.s;
        L.shell = q.shell;
    } else {
        end_cascade<R, kSplit>(P, tab, L, false);
    }
}

// One transport step of the particle in flight (§2.3): a path from the majorant rate,
// then a candidate collision or a boundary crossing. An accepted candidate leaves the
// lane in kKinWait with its partner stored; finish_collision() completes it.
template <typename R, bool kCount, bool kSplit, typename Em>
__device__ void step_transport(const SimParams &P, const ShellTable<R> &t, const TargetScalars &tab, Lane<R> &L,
                               Particle<R> *stack, Counters<kCount> &C, Em &em)
{
    if (L.steps >= P.max_steps) {
        // step cap: the particles in flight stay in the nucleus and the event goes on to
        // its excitation energy with what has escaped so far
        L.flags |= PNUC_FLAG_STEP_CAP;
        L.sp = 0;
        end_cascade<R, kSplit>(P, tab, L, true);
        return;
    }
    ++L.steps;
    C.add(PNUC_C_STEPS);
    const int s1 = L.s, i = L.shell;
    const R m1 = nucleon_mass_R<R>(s1);
    const R pp = dot3(L.p, L.p), pm = sqrt(pp);
    const R E1 = sqrt(pp + m1 * m1);
    R d[3] = {L.p[0] / pm, L.p[1] / pm, L.p[2] / pm};
    int dir;
    R sb = boundary_distance(t, i, L.r, d, dir);
    R gh = g_hat<R>(pm, E1, t.vF[i]);
    R Sigma = R(0.1) * t.rho[i] * gh / (pm * R(1e-3));
    R s = -log(L.rng.next()) / Sigma;
    if (s < sb) {
        // ---- candidate collision
#pragma unroll
        for (int k = 0; k < 3; ++k) L.r[k] += s * d[k];
        C.add(PNUC_C_CANDIDATES);
        int s2 = (L.rng.next() < t.ZoverA) ? 1 : 0;
        R m2 = nucleon_mass_R<R>(s2);
        R q = t.pF[s2][i] * cbrt_uniform(L.rng.next());
        R ct = R(2) * L.rng.next() - R(1);
        R sn = sqrt((R(1) - ct) * (R(1) + ct));
        R ph = R(kTwoPi) * L.rng.next();
        R sph, cph;
        sincos(ph, &sph, &cph);
        R p2[3] = {q * sn * cph, q * sn * sph, q * ct};
        R T1 = kinetic(pp, m1), T2 = kinetic(q * q, m2);
        R E2 = sqrt(q * q + m2 * m2);
        R X = T1 * T2 + T1 * m2 + T2 * m1 - dot3(L.p, p2);
        if (X < R(0)) X = R(0);
        R kk = sqrt(X * (X + R(2) * m1 * m2));
        R plab = kk / m2;
        R vrel = kk / (E1 * E2);
        R sig = sigma_nn<R>(s1 == s2, plab * R(1e-3));
        R ua = L.rng.next();
        if (!(ua * gh < sig * vrel * E1 * R(1e-3))) return;  // null collision
        C.add(PNUC_C_KINEMATICS);
        L.jp[0] = p2[0];
        L.jp[1] = p2[1];
        L.jp[2] = p2[2];
        L.js = s2;
        L.phase = kKinWait;
        return;
    }
    // ---- move to the boundary and cross it
#pragma unroll
    for (int k = 0; k < 3; ++k) L.r[k] += sb * d[k];
    C.add(PNUC_C_CROSSINGS);
    const int j = i + dir;  // kShells = outside
    R dT = -t.V[s1][i] + (j == kShells ? R(0) : t.V[s1][j]);
    R rr = sqrt(dot3(L.r, L.r));
    R n[3] = {L.r[0] / rr, L.r[1] / rr, L.r[2] / rr};
    R Tb = kinetic(pp, m1);
    if (!refract(n, L.p, m1, dT, dir)) {
        C.add(PNUC_C_REFLECTIONS);
        return;
    }
    L.shell = j;
    if (j < kShells) return;
    // escape: recorded only once the attempt is non-elastic
    R Tout = Tb + dT;
    if (L.n_coll > 0) {
        C.add(PNUC_C_ESCAPES);
        R pn = sqrt(dot3(L.p, L.p));
        const double Toutd = to_d<R>(Tout);
        em.emit(P, L.ev, s1, 0, L.n_index++, Toutd, (float)(L.p[0] / pn), (float)(L.p[1] / pn),
                (float)(L.p[2] / pn), L.flags);
        L.Esum += Toutd + nucleon_mass(s1);
        L.Px += to_d<R>(L.p[0]);
        L.Py += to_d<R>(L.p[1]);
        L.Pz += to_d<R>(L.p[2]);
        ++L.n_esc;
        if (s1 == 1) ++L.n_p_esc;
    }
    next_particle<R, kSplit>(P, tab, L, stack);
}

// ------------------------------------------------------------------ FP32-mode collision
__device__ float slope_f(bool like, float p)
{
    if (like) {
        float p8 = p * p;
        p8 = p8 * p8;
        p8 = p8 * p8;
        return 5.5f * p8 / (7.7f + p8);
    }
    if (p < 0.225f) return 0.f;
    if (p < 0.6f) return 16.53f * (p - 0.225f);
    if (p < 1.6f) return 7.16f - 1.63f * p;
    return 4.552f;
}

// FP32 mode: kinetic energies, the pair invariant and the angular sampling in FP32; the
// boost of the pair into its CM frame and back and the products' energies in FP64. The
// boost is built from E = m + T and the pair's own s = E_t^2 - P^2, so it is an exact
// Lorentz transformation and conserves the pair's energy and momentum to FP64 rounding.
// It is written with beta = P / E_t and gamma = E_t / sqrt(s) substituted, so that one
// reciprocal, D = 1 / (E_t + sqrt(s)), stands for both 1 / E_t and gamma^2 / (gamma + 1):
//   p_cm  = p + P/sqrt(s) (D P.p - E)          (into the CM frame)
//   q_lab = k + P/sqrt(s) (D P.k + e)          (back to the lab)
//   T_lab = (E_t e + P.k) / sqrt(s) - m
__device__ void collide_mixed(int s1, const float *p1, int s2, const float *p2, float ut, float uphi, float uf,
                              float *q1, float *q2, double &T1n, double &T2n)
{
    const double m1 = nucleon_mass(s1), m2 = nucleon_mass(s2);
    const float m1f = nucleon_mass_R<float>(s1), m2f = nucleon_mass_R<float>(s2);
    const bool like = s1 == s2;
    const float T1 = kinetic(dot3(p1, p1), m1f), T2 = kinetic(dot3(p2, p2), m2f);
    float Xf = T1 * T2 + T1 * m2f + T2 * m1f - dot3(p1, p2);  // four-product p1.p2 - m1 m2
    if (Xf < 0.f) Xf = 0.f;
    const float kf = sqrtf(Xf * (Xf + 2.f * m1f * m2f));        // sqrt(s) p* = m2 p_lab
    const double P1[3] = {f2d(p1[0]), f2d(p1[1]), f2d(p1[2])};
    const double P[3] = {P1[0] + f2d(p2[0]), P1[1] + f2d(p2[1]), P1[2] + f2d(p2[2])};
    const double E1 = m1 + f2d(T1), Et = E1 + (m2 + f2d(T2));
    const double s = Et * Et - dot3(P, P);
    const double irs = rsqrt(s);
    const double rs = s * irs;
    const double D = 1.0 / (Et + rs);
    const double f = (D * dot3(P, P1) - E1) * irs;
    float n[3] = {d2f(P1[0] + P[0] * f), d2f(P1[1] + P[1] * f), d2f(P1[2] + P[2] * f)};
    const float rn = rsqrtf(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    n[0] *= rn;
    n[1] *= rn;
    n[2] *= rn;
    const float plab = kf / m2f * 1e-3f;
    const double pst = f2d(kf) * irs;
    const float pg = d2f(pst) * 1e-3f;
    const float b = 4.f * slope_f(like, plab) * pg * pg;
    const float y = b > 0.f ? -log1pf(ut * expm1f(-b)) / b : ut;
    float ct = 1.f - 2.f * y;
    if (!like) {
        float a = plab <= 0.8f ? 1.f : (0.8f / plab) * (0.8f / plab);
        if (uf < a / (1.f + a)) ct = -ct;
    }
    const float st = sqrtf((1.f - ct) * (1.f + ct));
    float sp, cp;
    __sincosf(6.2831853f * uphi, &sp, &cp);
    float d[3];
    const float rho = sqrtf(n[0] * n[0] + n[1] * n[1]);
    if (rho > 0.f) {
        const float ir = 1.f / rho;
        d[0] = ct * n[0] + st * (cp * n[0] * n[2] * ir - sp * n[1] * ir);
        d[1] = ct * n[1] + st * (cp * n[1] * n[2] * ir + sp * n[0] * ir);
        d[2] = ct * n[2] - st * cp * rho;
    } else {
        d[0] = st * cp;
        d[1] = st * sp;
        d[2] = (n[2] >= 0.f ? 1.f : -1.f) * ct;
    }
    const double K[3] = {pst * f2d(d[0]), pst * f2d(d[1]), pst * f2d(d[2])};
    // CM energies: e1 = (s + m1^2 - m2^2) / (2 sqrt(s)), e2 = sqrt(s) - e1
    constexpr double kDm2 = kMp * kMp - kMn * kMn;
    const double dm2 = like ? 0.0 : (s1 ? kDm2 : -kDm2);
    const double e1 = (s + dm2) * (0.5 * irs), e2 = rs - e1;
    const double PK = dot3(P, K), DPK = D * PK;
    const double f1 = (DPK + e1) * irs, f2 = (e2 - DPK) * irs;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        q1[c] = d2f(K[c] + P[c] * f1);
        q2[c] = d2f(P[c] * f2 - K[c]);
    }
    T1n = (Et * e1 + PK) * irs - m1;
    T2n = (Et * e2 - PK) * irs - m2;
}

template <typename R>
__device__ void collide_lane(int s1, const R *p1, int s2, const R *p2, R ut, R uph, R uf, R *q1, R *q2, double &T1n,
                             double &T2n);
template <>
__device__ void collide_lane<double>(int s1, const double *p1, int s2, const double *p2, double ut, double uph,
                                     double uf, double *q1, double *q2, double &T1n, double &T2n)
{
    collide(s1, p1, s2, p2, ut, uph, uf, q1, q2);
    T1n = kinetic(dot3(q1, q1), nucleon_mass(s1));
    T2n = kinetic(dot3(q2, q2), nucleon_mass(s2));
}
template <>
__device__ void collide_lane<float>(int s1, const float *p1, int s2, const float *p2, float ut, float uph, float uf,
                                    float *q1, float *q2, double &T1n, double &T2n)
{
    collide_mixed(s1, p1, s2, p2, ut, uph, uf, q1, q2, T1n, T2n);
}

// Completes the lane's accepted candidate (§2.3): elastic kinematics, Pauli blocking,
// then the cutoff of each product; the struck nucleon goes on the stack.
template <typename R, bool kCount, bool kSplit>
__device__ void finish_collision(const SimParams &P, const ShellTable<R> &t, const TargetScalars &tab, Lane<R> &L,
                                 Particle<R> *stack, Counters<kCount> &C)
{
    const int s1 = L.s, s2 = L.js, i = L.shell;
    const R ut = L.rng.next(), uph = L.rng.next(), uf = L.rng.next();
    R q1[3], q2[3];
    double T1n, T2n;
    collide_lane<R>(s1, L.p, s2, L.jp, ut, uph, uf, q1, q2, T1n, T2n);
    L.phase = kTransport;
    if (!(T1n > to_d<R>(t.EF[s1][i]) && T2n > to_d<R>(t.EF[s2][i]))) {
        C.add(PNUC_C_PAULI_BLOCKED);
        return;
    }
    C.add(PNUC_C_COLLISIONS);
    ++L.n_coll;
    double cut2 = to_d<R>(t.V[s2][i]) + (s2 == 1 ? to_d<R>(t.EC) : 0.0);
    double cut1 = to_d<R>(t.V[s1][i]) + (s1 == 1 ? to_d<R>(t.EC) : 0.0);
    if (T2n < cut2) {
        C.add(PNUC_C_CAPTURES);
    } else if (L.sp >= kStackCap) {
        L.flags |= PNUC_FLAG_STACK_OVERFLOW;
        C.add(PNUC_C_CAPTURES);
    } else {
        Particle<R> &np = stack[L.sp++];
        np.r[0] = L.r[0];
        np.r[1] = L.r[1];
        np.r[2] = L.r[2];
        np.p[0] = q2[0];
        np.p[1] = q2[1];
        np.p[2] = q2[2];
        np.s = s2;
        np.shell = i;
    }
    L.p[0] = q1[0];
    L.p[1] = q1[1];
    L.p[2] = q1[2];
    if (T1n < cut1) {
        C.add(PNUC_C_CAPTURES);
        next_particle<R, kSplit>(P, tab, L, stack);
    }
}

// ------------------------------------------------------------------ evaporation step
// Rejection sampler of t on [0, x] (four draws per trial); returns -1 after max_trials.
template <typename R>
__device__ R sample_t(Stream<R> &rng, R a, R x, R b, int max_trials, int &trials)
{
    R W1 = x * x / (R(2) * a), W2 = b * x;
    bool small = x < R(2);
    R pmix = small ? W1 * x / (W1 * x + R(2) * W2) : W1 / (W1 + W2);
    for (int k = 0; k < max_trials; ++k) {
        rng.template ensure<true>(6);  // four for this trial, and the two decay angles if it is accepted
        R um = rng.next(), u1 = rng.next(), u2 = rng.next(), ua = rng.next();
        ++trials;
        bool first = um < pmix;
        R t;
        if (small) t = first ? x * (u1 > u2 ? u1 : u2) : x * u1;
        else t = first ? -log(u1 * u2) : -log(u1);
        if (t >= x) continue;
        R h = (t * (R(2) * x - t) / (R(4) * a) + b) * (x - t);
        if (small) h *= exp(-t);
        if (ua * (W1 * t + W2) < h) return t;
    }
    return R(-1);
}

// Reading M26's emission sampler: the daughter's excitation U in [0, Y] with density
// ~ (Y + b - U) rho(U), rho the composite level density. One draw picks the part, the
// constant-temperature one (U < L = min(Y, U_x)) with probability I_ct / I (FP64); then trials
// of four draws as in sample_t(). Constant-temperature part: t = k (L - U) on [0, kL] has
// density ~ (c0 + t) e^-t, c0 = k (Y + b - L): for kL >= 2 the mixture of Exp(1) (weight c0)
// and Gamma(2,1) (weight 1), kept if t < kL; for kL < 2 the mixture of kL u1 (weight c0 kL)
// and kL max(u1, u2) (weight (kL)^2 / 2), kept with probability e^-t. Fermi-gas part:
// sample_t()'s trial on [0, x], kept if t < x - x_x (U above U_x). Returns U, or -1 after
// max_trials.
__device__ double width_integral_ct(const double *T, double a, double Y, double b, double *ct_part);
__device__ double width_integral_ct_f32(const double *T, float a, float Y, float b, float x, double *ct_part);
__device__ __noinline__ double exp_beyond_fixed(float x);

// T: the daughter's row of M26's constant table (SimParams.ct_table)
template <typename R>
__device__ R sample_U_ct(Stream<R> &rng, const double *T, R a, R Y, R b, R x, int max_trials, int &trials)
{
    const R Ux = to_R<R>(__ldg(&T[0])), k = to_R<R>(__ldg(&T[1])), xx = R(2) * sqrt(a * Ux);
    double ict, itot;
    if constexpr (sizeof(R) == 4) itot = width_integral_ct_f32(T, a, Y, b, x, &ict);
    else itot = width_integral_ct(T, a, Y, b, &ict);
    if (to_d<R>(rng.next()) * itot < ict) {
        const R L = Y < Ux ? Y : Ux, kL = k * L, c0 = k * (Y + b - L);
        const bool small = kL < R(2);
        const R pmix = small ? c0 * kL / (c0 * kL + R(0.5) * kL * kL) : c0 / (c0 + R(1));
        for (int n = 0; n < max_trials; ++n) {
            rng.template ensure<true>(6);  // four for this trial, and the two decay angles if it is accepted
            const R um = rng.next(), u1 = rng.next(), u2 = rng.next(), ua = rng.next();
            ++trials;
            const bool first = um < pmix;
            R t;
            if (small) {
                t = first ? kL * u1 : kL * (u1 > u2 ? u1 : u2);
                if (!(ua < exp(-t))) continue;
            } else {
                t = first ? -log(u1) : -log(u1 * u2);
                if (!(t < kL)) continue;
            }
            return L - t / k;
        }
        return R(-1);
    }
    const R W1 = x * x / (R(2) * a), W2 = b * x;
    const bool small = x < R(2);
    const R pmix = small ? W1 * x / (W1 * x + R(2) * W2) : W1 / (W1 + W2);
    const R tmax = x - xx;
    for (int n = 0; n < max_trials; ++n) {
        rng.template ensure<true>(6);
        const R um = rng.next(), u1 = rng.next(), u2 = rng.next(), ua = rng.next();
        ++trials;
        const bool first = um < pmix;
        R t;
        if (small) t = first ? x * (u1 > u2 ? u1 : u2) : x * u1;
        else t = first ? -log(u1 * u2) : -log(u1);
        if (t >= tmax) continue;
        R h = (t * (R(2) * x - t) / (R(4) * a) + b) * (x - t);
        if (small) h *= exp(-t);
        if (ua * (W1 * t + W2) < h) return (x - t) * (x - t) / (R(4) * a);
    }
    return R(-1);
}

// Channel parameters in precision R (the Q-value in FP64).
template <typename R>
struct ChanP {
    double Q;
    R V, b, a, x, w0;  // barrier, offset, level-density parameter, 2 sqrt(aY), g m c A^(2/3)
    R Y;               // X - V: the range of the daughter's excitation
    bool open;
};

template <typename R>
__device__ void channel_params(const SimParams &P, int Z, int A, double Estar, int j, ChanP<R> &c)
{
    c.open = false;
    c.x = R(0);
    const int Zd = Z - cEjZ[j], Ad = A - cEjA[j];
    if (Zd < 1 || Ad - Zd < 1 || Ad < 5) return;
    // (M_d + m_j) - M_parent, tabulated per parent with the context (the same FP64 sum)
    const double Q = __ldg(&P.qval[(size_t)kQStride * (Z * kMassA + A) + j]);
    const R A3 = to_R<R>(__ldg(&P.cbrtA[Ad]));
    R V, b, cj;
    if (cEjZ[j] == 0) {
        R alpha = R(0.76) + R(1.93) / A3;
        R beta = (R(1.66) / (A3 * A3) - R(0.05)) / alpha;
        V = beta < R(0) ? -beta : R(0);
        b = beta > R(0) ? beta : R(0);
        cj = alpha;
    } else {
        V = R(kE2) * cEjZ[j] * Zd / (R(1.5) * (to_R<R>(__ldg(&P.cbrtA[cEjA[j]])) + A3));
        b = R(0);
        cj = R(1);
    }
    const R X = to_R<R>(Estar - Q);
    const R Y = X - V;
    c.Q = Q;
    c.V = V;
    c.b = b;
    c.a = R(Ad) / R(8);
    c.Y = Y;
    if (!(Y > R(0))) return;
    c.x = R(2) * sqrt(c.a * Y);
    c.w0 = ej_G<R>(j) * ej_M<R>(j) * cj * (A3 * A3);
    c.open = true;
}

// F(x) = e^x (x^2 - 3x + 3) + x^2/2 - 3 and G(x) = e^x (x - 1) + 1 (the closed-form width
// integrals), FP64 mode: the exponential reaches e^160; series below x = 1.
__device__ __forceinline__ void width_FG(double x, double &F, double &G)
{
    if (x >= 1.0) {
        const double ex = exp(x);
        F = ex * (x * x - 3.0 * x + 3.0) + 0.5 * x * x - 3.0;
        G = ex * (x - 1.0) + 1.0;
        return;
    }
    double term = x, f = 0.0, g = 0.0;  // term = x^n / n!
#pragma unroll 1
    for (int n = 2; n <= 20; ++n) {
        term *= x / n;
        g += (n - 1) * term;
        if (n >= 4) f += ((n - 1) * (n - 3)) * term;
    }
    F = f;
    G = g;
}

// Reading M26 (the option pnuc_config.level_density = 1): the daughter's level density is
// constant-temperature below U_x = 2.5 + 150/A_d MeV (A_d = 8a) and M20's Fermi gas above,
// joined in value and slope at U_x: exp(sqrt(a U_x) + U / T) with 1/T = sqrt(a / U_x).
// The daughter's row of the constant table (tables.cu, built with the context): U_x, k = 1/T,
// C = e^{sqrt(a U_x)}, e^{k U_x} - 1, e^{k U_x} - 1 - k U_x, G(x_x), H(x_x); a = A_d / 8.
__device__ __forceinline__ const double *ct_row(const double *table, double a)
{
    return table + kCtStride * (int)(8.0 * a + 0.5);
}

// e^z - 1 - z, by series below z = 1/2
__device__ double expm1_minus(double z)
{
    if (z >= 0.5) return expm1(z) - z;
    double term = z, sum = 0.0;  // term = z^n / n!
#pragma unroll 1
    for (int n = 2; n <= 20; ++n) {
        term *= z / n;
        sum += term;
    }
    return sum;
}

// M26's width integral over U in [0, Y] of (Y + b - U) rho(U), FP64: the constant-temperature
// part over [0, L], L = min(Y, U_x), is C [(Y + b - L)(e^{kL} - 1)/k + (e^{kL} - 1 - kL)/k^2]
// (k = 1/T, C = e^{sqrt(a U_x)}); above U_x, M20's integral over [0, Y] less the same
// integrand over [0, U_x], (Y + b) G(x_x)/(2a) - H(x_x)/(8a^2), x_x = 2 sqrt(a U_x),
// H(x) = e^x (x^3 - 3x^2 + 6x - 6) + 6. The constant-temperature part goes to *ct_part. What
// depends only on the daughter comes from its row T of the constant table, so that a width
// takes one exponential at most (e^{kY} below U_x, M20's e^x above).
__device__ double width_integral_ct(const double *T, double a, double Y, double b, double *ct_part)
{
    const double Ux = __ldg(&T[0]), k = __ldg(&T[1]), C = __ldg(&T[2]);
    double ict;
    if (Y < Ux) {
        const double kL = k * Y;
        ict = C * ((Y + b - Y) * expm1(kL) / k + expm1_minus(kL) / (k * k));
    } else {
        ict = C * ((Y + b - Ux) * __ldg(&T[3]) / k + __ldg(&T[4]) / (k * k));
    }
    *ct_part = ict;
    if (!(Y > Ux)) return ict;
    const double below = (Y + b) * __ldg(&T[5]) / (2.0 * a) - __ldg(&T[6]) / (8.0 * a * a);
    double F, G;
    width_FG(2.0 * sqrt(a * Y), F, G);
    return ict + ((F / (4.0 * a * a) + b * G / (2.0 * a)) - below);
}

// M26's width integral in the FP32 mode (a, Y, b and x = 2 sqrt(aY) in FP32): the same closed
// forms as width_integral_ct(), with the daughter's constants as FP64 factors (no division)
// and the exponentials in double precision on the integer pipes (exp_fixed), as M20's widths
// take them: e^{kY} for kY >= 1 (below 1, e^{kY} - 1 and e^{kY} - 1 - kY by their series in
// FP32, as M20's series below x = 1), and e^x above U_x (x >= 2.5 there). The Fermi-gas part
// is M20's integral in its FP32-mode form, e^x A1 + A0 (channel_width_f32_d), less the
// daughter's constant part below U_x.
__device__ double width_integral_ct_f32(const double *T, float a, float Y, float b, float x, double *ct_part)
{
    const float Ux = d2f(__ldg(&T[0])), k = d2f(__ldg(&T[1]));
    double ict;
    if (Y < Ux) {
        const float z = k * Y;
        double em1, emm;  // e^z - 1, e^z - 1 - z
        if (z >= 1.f) {
            em1 = exp_fixed(z) - 1.0;
            emm = em1 - f2d(z);
        } else {
            float term = z, s = 0.f;  // term = z^n / n!, s = the sum from n = 2
#pragma unroll 1
            for (int n = 2; n <= 12; ++n) {
                term *= z / float(n);
                s += term;
            }
            em1 = f2d(z + s);
            emm = f2d(s);
        }
        ict = __ldg(&T[11]) * (f2d(b) * em1) + __ldg(&T[12]) * emm;
    } else {
        ict = __ldg(&T[7]) * f2d(Y + b - Ux) + __ldg(&T[8]);
    }
    *ct_part = ict;
    if (!(Y > Ux)) return ict;
    const double ex = x < 256.f ? exp_fixed(x) : exp_beyond_fixed(x);
    const float ia = 1.f / a, q = 0.25f * ia * ia, h = 0.5f * b * ia;
    const float A1 = (x * x - 3.f * x + 3.f) * q + (x - 1.f) * h;
    const float A0 = (0.5f * x * x - 3.f) * q + h;
    const double below = f2d(Y + b) * __ldg(&T[9]) - __ldg(&T[10]);
    return ict + ((ex * f2d(A1) + f2d(A0)) - below);
}

// The type the six widths of a step are held and drawn in: FP64 (the FP64 mode, and the
// FP32 mode's widths with FP64 exponentials), or FP32 for the scaled FP32 widths (below).
template <typename R, bool kScaled>
struct WidthOf {
    using T = double;
};
template <>
struct WidthOf<float, true> {
    using T = float;
};
template <typename R, bool kScaled>
using width_t = typename WidthOf<R, kScaled>::T;

// a draw or parameter of precision R as a width-type value (float -> double on the integer
// pipes, fpconv.h)
template <typename W, typename R>
__device__ __forceinline__ W as_width(R x)
{
    if constexpr (sizeof(W) == sizeof(R)) return x;
    else return to_d<R>(x);
}

// FP32 mode, widths in FP64: the channel parameters (x, a, b, w0) come in FP32, and so do the
// factors of the closed forms: with F = e^x (x^2 - 3x + 3) + x^2/2 - 3 and G = e^x (x - 1) + 1,
// the width w0 (F/(4a^2) + b G/(2a)) is w0 (e^x A1 + A0) with A1 = (x^2 - 3x + 3)/(4a^2) +
// b (x - 1)/(2a) and A0 = (x^2/2 - 3)/(4a^2) + b/(2a), both FP32; the exponential (up to e^160,
// beyond FP32's range, and computed on the integer pipes, expfixed.h) and the two products
// that carry it are FP64. The series below x = 1 needs no exponential and runs in FP32.
// The series below x = 1 (M20) and e^x beyond exp_fixed's range (x >= 256, which no nucleus
// the library accepts reaches) are rare, and out of line: the evaporation kernel's loop is
// bound partly by instruction fetch, and with this code inlined it ran 4% slower.
__device__ __noinline__ double width_series_f32_d(float x, float a, float b, float w0)
{
    double F, G;
    {
        float term = x, f = 0.f, g = 0.f;  // term = x^n / n!
#pragma unroll 1
        for (int n = 2; n <= 20; ++n) {
            term *= x / float(n);
            g += float(n - 1) * term;
            if (n >= 4) f += float((n - 1) * (n - 3)) * term;
        }
        F = f2d(f);
        G = f2d(g);
    }
    const float ia = 1.f / a;
    return f2d(w0) * (F * f2d(0.25f * ia * ia) + G * f2d(0.5f * b * ia));
}
__device__ __noinline__ double exp_beyond_fixed(float x) { return exp(f2d(x)); }

__device__ __forceinline__ double channel_width_f32_d(const ChanP<float> &c)
{
    const float x = c.x;
    if (!(x >= 1.f)) return width_series_f32_d(x, c.a, c.b, c.w0);
    const double ex = x < 256.f ? exp_fixed(x) : exp_beyond_fixed(x);
    const float ia = 1.f / c.a, q = 0.25f * ia * ia, h = 0.5f * c.b * ia;
    const float A1 = (x * x - 3.f * x + 3.f) * q + (x - 1.f) * h;
    const float A0 = (0.5f * x * x - 3.f) * q + h;
    return f2d(c.w0) * (ex * f2d(A1) + f2d(A0));
}

// The width of one open channel, FP64 in the FP64 mode and in the FP32 mode (the scale
// reference xm is ignored). The channel draw uses only the six widths' ratios, so the scaled
// FP32 variant (kScaled) returns the width times e^-xm, xm the largest x of the parent's open
// channels: the exponential becomes e^(x - xm) <= 1 and the whole width is FP32 arithmetic
// (the unscaled width reaches e^160, beyond FP32's range).
__device__ float channel_width_scaled(const ChanP<float> &c, float xm);

template <typename R, bool kScaled, bool kCT = false>
__device__ width_t<R, kScaled> channel_width(const ChanP<R> &c, R xm, const double *ct_table)
{
    static_assert(!(kScaled && kCT), "the scaled FP32 widths take the Fermi-gas level density");
    if constexpr (kCT) {  // M26: FP64 widths in both modes (the FP32 mode's from FP32 factors)
        if (!c.open) return 0.0;
        double part;
        const double a = to_d<R>(c.a);
        if constexpr (sizeof(R) == 4)
            return f2d(c.w0) * width_integral_ct_f32(ct_row(ct_table, a), c.a, c.Y, c.b, c.x, &part);
        else
            return c.w0 * width_integral_ct(ct_row(ct_table, a), a, c.Y, c.b, &part);
    } else if constexpr (sizeof(R) == 8) {
        if (!c.open) return 0.0;
        double F, G;
        width_FG(c.x, F, G);
        const double a = c.a;
        const double I = F / (4.0 * a * a) + c.b * G / (2.0 * a);
        return c.w0 * I;
    } else if constexpr (kScaled) {
        return channel_width_scaled(c, xm);
    } else {
        if (!c.open) return 0.0;
        return channel_width_f32_d(c);
    }
}

__device__ float channel_width_scaled(const ChanP<float> &c, float xm)
{
    if (!c.open) return 0.f;
    // s = e^-xm is 0 for xm above about 87 (the FP32 kernels flush denormals); the terms it
    // multiplies are then below 2^-24 of the largest width, which the FP32 sum cannot resolve.
    const float x = c.x, s = expf(-xm);
    float F, G;
    if (x >= 1.f) {
        const float ex = expf(x - xm);
        F = ex * (x * x - 3.f * x + 3.f) + (0.5f * x * x - 3.f) * s;
        G = ex * (x - 1.f) + s;
    } else {
        float term = x, f = 0.f, g = 0.f;  // term = x^n / n!
#pragma unroll 1
        for (int n = 2; n <= 20; ++n) {
            term *= x / float(n);
            g += float(n - 1) * term;
            if (n >= 4) f += float((n - 1) * (n - 3)) * term;
        }
        F = f * s;
        G = g * s;
    }
    const float ia = 1.f / c.a;
    return c.w0 * (F * (0.25f * ia * ia) + G * (0.5f * c.b * ia));
}

// The scale reference of a step's widths: the largest x of the open channels (0 if none).
template <typename R>
__device__ __forceinline__ R widths_xm(const ChanP<R> *chans)
{
    R xm = R(0);
#pragma unroll
    for (int j = 0; j < 6; ++j)
        if (chans[j].open && chans[j].x > xm) xm = chans[j].x;
    return xm;
}

// Two-body decay of the parent (invariant mass W) into an ejectile of mass m1 and a
// daughter of mass m2 with kinetic energy release eps, isotropic in the parent's rest frame
// (cos theta = ct, azimuth ph), boosted to the lab with the parent's four-momentum.
// Writes the ejectile's lab momentum pl, energy el, kinetic energy Tl and direction u.
template <typename R>
__device__ void decay_to_lab(double W, double m1, double m2, double eps, R ct, R ph, const Lane<R> &L, double *pl,
                             double &el, double &Tl, float *u);
template <>
__device__ void decay_to_lab<double>(double W, double m1, double m2, double eps, double ct, double ph,
                                     const Lane<double> &L, double *pl, double &el, double &Tl, float *u)
{
    const double pd = sqrt(eps * (W + m1 + m2) * (W - m1 + m2) * (W + m1 - m2)) / (2.0 * W);
    const double sn = sqrt((1.0 - ct) * (1.0 + ct));
    double sph, cph;
    sincos(ph, &sph, &cph);
    const double pv[3] = {pd * sn * cph, pd * sn * sph, pd * ct};
    const double e1 = sqrt(pd * pd + m1 * m1);
    const double Pr[3] = {L.Prx, L.Pry, L.Prz};
    const double Er = L.Er;
    const double Pm = sqrt(dot3(Pr, Pr));
    const double gamma = Er / sqrt((Er - Pm) * (Er + Pm));
    const double beta[3] = {Pr[0] / Er, Pr[1] / Er, Pr[2] / Er};
    boost(beta, gamma, 1.0, e1, pv, pl);
    el = gamma * (e1 + dot3(beta, pv));
    const double pl2 = dot3(pl, pl);
    Tl = kinetic(pl2, m1);
    const double pln = sqrt(pl2);
    u[0] = (float)(pl[0] / pln);
    u[1] = (float)(pl[1] / pln);
    u[2] = (float)(pl[2] / pln);
}
// FP32 mode: the decay and the boost in FP32, the parent's four-momentum bookkeeping in FP64.
// The factors of p^2 are all positive, so there is no cancellation; the parent is a recoiling
// nucleus (|beta| of order 0.01), so gamma - 1 is taken as beta^2 gamma^2 / (gamma + 1) and
// the lab kinetic energy as (gamma - 1) m1 + gamma (T* + beta.p*), with no difference of
// total energies. The release is taken as at least 0: with x in FP32, a draw of t within a
// few 1e-7 of 0 on a channel without barrier (V = 0) can put the daughter's excitation U_d an
// FP32 rounding above E* - Q (about 5e-7 of such emissions, in emulation), which would
// otherwise give a NaN momentum.
template <>
__device__ void decay_to_lab<float>(double W, double m1, double m2, double eps, float ct, float ph,
                                    const Lane<float> &L, double *pl, double &el, double &Tl, float *u)
{
    const float ef = fmaxf(d2f(eps), 0.f), m1f = d2f(m1), m2f = d2f(m2), Wf = d2f(W);
    const float pd2 = ef * (2.f * (m1f + m2f) + ef) * (2.f * m2f + ef) * (2.f * m1f + ef) / (4.f * Wf * Wf);
    const float pd = sqrtf(pd2);
    const float tcm = pd2 / (sqrtf(pd2 + m1f * m1f) + m1f);  // rest-frame kinetic energy
    const float sn = sqrtf((1.f - ct) * (1.f + ct));
    float sph, cph;
    __sincosf(ph, &sph, &cph);
    const float pv[3] = {pd * sn * cph, pd * sn * sph, pd * ct};
    const float iE = 1.f / d2f(L.Er);
    const float beta[3] = {d2f(L.Prx) * iE, d2f(L.Pry) * iE, d2f(L.Prz) * iE};
    const float b2 = beta[0] * beta[0] + beta[1] * beta[1] + beta[2] * beta[2];
    const float g2 = 1.f / (1.f - b2);
    const float g = sqrtf(g2);
    const float bp = beta[0] * pv[0] + beta[1] * pv[1] + beta[2] * pv[2];
    const float f = g2 / (g + 1.f) * bp + g * (m1f + tcm);
    float plf[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        plf[k] = pv[k] + beta[k] * f;
        pl[k] = f2d(plf[k]);
    }
    const float Tf = fmaxf(b2 * g2 / (g + 1.f) * m1f + g * (tcm + bp), 0.f);
    Tl = f2d(Tf);
    el = m1 + Tl;
    const float r = rsqrtf(plf[0] * plf[0] + plf[1] * plf[1] + plf[2] * plf[2]);
    u[0] = plf[0] * r;
    u[1] = plf[1] * r;
    u[2] = plf[2] * r;
}

// The daughter's excitation U_d = (x - t)^2 / (4a) after an emission at t (§2.4): FP64 in the
// FP64 mode (the oracle's operations), FP32 in the FP32 mode.
template <typename R>
__device__ __forceinline__ double daughter_excitation(R x, R t, R a);
template <>
__device__ __forceinline__ double daughter_excitation<double>(double x, double t, double a)
{
    const double xt = x - t;
    return xt * xt / (4.0 * a);
}
template <>
__device__ __forceinline__ double daughter_excitation<float>(float x, float t, float a)
{
    const float xt = x - t;
    return f2d(xt * xt / (4.f * a));
}

// The second half of an evaporation step (§2.4), given the six channel widths G of the
// parent (Z, A, E* in L): the channel draw, the emission energy, and the two-body decay
// isotropic in the parent's rest frame, boosted to the lab.
template <typename R, bool kScaled, bool kCT, bool kCount, typename Em>
__device__ void evap_emit(const SimParams &P, Lane<R> &L, const width_t<R, kScaled> *G,
                          Counters<kCount> &C, Em &em)
{
    using W = width_t<R, kScaled>;
    const int Z = L.Z, A = L.A;
    const double Estar = L.Estar;
    W S = W(0);
#pragma unroll
    for (int j = 0; j < 6; ++j) S += G[j];
    if (!(S > W(0))) {
        L.phase = kFinish;
        return;
    }
    C.add(PNUC_C_EVAP_STEPS);
    W us = as_width<W>(L.rng.next()) * S, cum = W(0);
    int ch = -1;
#pragma unroll 1
    for (int j = 0; j < 6; ++j) {
        cum += G[j];
        if (ch < 0 && us < cum) ch = j;
    }
    if (ch < 0)
        for (int j = 5; j >= 0; --j)
            if (G[j] > W(0)) {
                ch = j;
                break;
            }
    ChanP<R> c;  // the chosen channel's parameters, recomputed (the same function of Z, A, E*)
    channel_params<R>(P, Z, A, Estar, ch, c);
    int trials = 0;
    double Ud;
    if constexpr (kCT) {
        const R u = sample_U_ct<R>(L.rng, ct_row(P.ct_table, to_d<R>(c.a)), c.a, c.Y, c.b, c.x, P.max_evap_trials,
                                   trials);
        Ud = u < R(0) ? -1.0 : to_d<R>(u);
    } else {
        const R tt = sample_t<R>(L.rng, c.a, c.x, c.b, P.max_evap_trials, trials);
        Ud = tt < R(0) ? -1.0 : daughter_excitation<R>(c.x, tt, c.a);
    }
    C.add(PNUC_C_EVAP_TRIALS, trials);
    if (Ud < 0.0) {
        L.flags |= PNUC_FLAG_EVAP_TRIAL_CAP;
        L.phase = kFinish;
        return;
    }
    const double eps = (Estar - c.Q) - Ud;
    const R ctr = R(2) * L.rng.next() - R(1);
    const R phr = R(kTwoPi) * L.rng.next();
    double pl[3], el, Tl;
    float u[3];
    const double Mparent = __ldg(&P.mass[Z * kMassA + A]);
    const double Md = __ldg(&P.mass[(Z - cEjZ[ch]) * kMassA + (A - cEjA[ch])]);
    decay_to_lab(Mparent + Estar, cEjM[ch], Md + Ud, eps, ctr, phr, L, pl, el, Tl, u);
    em.emit(P, L.ev, ch, 1, L.n_index++, Tl, u[0], u[1], u[2], L.flags);
    ++L.n_evap;
    L.Er -= el;
    L.Prx -= pl[0];
    L.Pry -= pl[1];
    L.Prz -= pl[2];
    L.Z = Z - cEjZ[ch];
    L.A = A - cEjA[ch];
    L.Estar = Ud;
}

// One evaporation step of one lane (the plain kernel): widths of the six channels, then
// evap_emit().
template <typename R, bool kScaled, bool kCT, bool kCount>
__device__ void step_evap(const SimParams &P, Lane<R> &L, Counters<kCount> &C)
{
    if (L.n_evap >= P.max_evap_steps) {
        L.flags |= PNUC_FLAG_EVAP_STEP_CAP;
        L.phase = kFinish;
        return;
    }
    C.add(PNUC_C_EVAP_PASSES);
    width_t<R, kScaled> G[6];
    ChanP<R> chans[6];
#pragma unroll 1
    for (int j = 0; j < 6; ++j) {
        channel_params<R>(P, L.Z, L.A, L.Estar, j, chans[j]);
        if (chans[j].open) C.add(chans[j].x >= R(1) ? PNUC_C_EVAP_EXPS : PNUC_C_EVAP_SERIES);
    }
    const R xm = kScaled ? widths_xm<R>(chans) : R(0);
#pragma unroll 1
    for (int j = 0; j < 6; ++j) G[j] = channel_width<R, kScaled, kCT>(chans[j], xm, P.ct_table);
    EmitNow em;
    evap_emit<R, kScaled, kCT, kCount>(P, L, G, C, em);
}

// ------------------------------------------------------------------ warp-wide widths
// One width evaluation: the parameters channel_width() reads, and where its result goes
// (6 x lane + channel in the warp's width array).
template <typename R>
struct WidthJob {
    R x, a, b, w0, Y;
    int tag;
};
constexpr int kWidthSlots = 6 * 32;  // per warp: six channels of every lane

template <typename R, bool kScaled, bool kCT>
__device__ __forceinline__ width_t<R, kScaled> job_width(const WidthJob<R> &jb, R xm, const double *ct_table)
{
    ChanP<R> c;
    c.open = true;
    c.x = jb.x;
    c.a = jb.a;
    c.b = jb.b;
    c.w0 = jb.w0;
    c.Y = jb.Y;
    return channel_width<R, kScaled, kCT>(c, xm, ct_table);
}

// One evaporation step of every lane of the warp with `active` set (the evaporation kernel).
// The widths are evaluated by the whole warp: the (lane, channel) pairs of open channels
// go to a job list in shared memory, those that need the exponential (x >= 1) from the
// front and the series ones (x < 1) from the back, and the 32 lanes work through it. One
// pass then serves up to 32 exponentials, where the per-lane loop issues one pass per channel
// for whichever lanes have it open; each width is channel_width()'s arithmetic, bit for bit.
// Each result goes to its lane's six entries of gw (closed channels are set to 0 by their
// lane), with the lane's scale reference in xms; no per-lane channel records are kept, so
// nothing of the step lives in local memory. Called by all 32 lanes of the warp; jobs and gw
// are the warp's kWidthSlots entries, xms its 32.
template <typename R, bool kScaled, bool kCT, bool kCount, typename Em>
__device__ void step_evap_warp(const SimParams &P, Lane<R> &L, bool active, WidthJob<R> *jobs,
                               width_t<R, kScaled> *gw, R *xms, Counters<kCount> &C, Em &em)
{
    if (active && L.n_evap >= P.max_evap_steps) {
        L.flags |= PNUC_FLAG_EVAP_STEP_CAP;
        L.phase = kFinish;
        active = false;
    }
    const unsigned FULL = 0xffffffffu, lane = threadIdx.x & 31, below = (1u << lane) - 1u;
    width_t<R, kScaled> *G = gw + 6 * lane;
    R xm = R(0);
    int nexp = 0, nser = 0;
#pragma unroll 1
    for (int j = 0; j < 6; ++j) {
        ChanP<R> c;
        if (active) {
            channel_params<R>(P, L.Z, L.A, L.Estar, j, c);
        } else {
            c.open = false;
            c.x = R(0);
        }
        const bool ex = c.open && c.x >= R(1);
        const bool se = c.open && !(c.x >= R(1));
        const unsigned me = __ballot_sync(FULL, ex), ms = __ballot_sync(FULL, se);
        if (ex || se) {
            const int slot = ex ? nexp + __popc(me & below) : kWidthSlots - 1 - (nser + __popc(ms & below));
            jobs[slot] = WidthJob<R>{c.x, c.a, c.b, c.w0, c.Y, (int)(6 * lane) + j};
            if (c.x > xm) xm = c.x;
        } else {
            G[j] = width_t<R, kScaled>(0);
        }
        nexp += __popc(me);
        nser += __popc(ms);
    }
    xms[lane] = xm;
    if (kCount) {
        const unsigned act = __ballot_sync(FULL, active);
        if (lane == 0) {
            C.add(PNUC_C_EVAP_PASSES, __popc(act));
            C.add(PNUC_C_EVAP_EXPS, nexp);
            C.add(PNUC_C_EVAP_SERIES, nser);
        }
    }
    __syncwarp();
    for (int k = lane; k < nexp; k += 32) {
        const WidthJob<R> jb = jobs[k];
        gw[jb.tag] = job_width<R, kScaled, kCT>(jb, xms[jb.tag / 6], P.ct_table);
    }
    for (int k = kWidthSlots - 1 - (int)lane; k >= kWidthSlots - nser; k -= 32) {
        const WidthJob<R> jb = jobs[k];
        gw[jb.tag] = job_width<R, kScaled, kCT>(jb, xms[jb.tag / 6], P.ct_table);
    }
    __syncwarp();
    if (active) evap_emit<R, kScaled, kCT, kCount>(P, L, G, C, em);
    __syncwarp();  // the lists are reused by the next step
}

// Advances lane L by one step of its current phase (no batching: the plain kernel).
template <typename R, bool kScaled, bool kCT, bool kCount>
__device__ __forceinline__ void step(const SimParams &P, const ShellTable<R> *sh, const TargetScalars *tabs, Lane<R> &L,
                                     Particle<R> *stack, Counters<kCount> &C)
{
    if (L.phase == kTransport) {
        EmitNow em;
        step_transport<R, kCount, false>(P, sh[L.tgt], tabs[L.tgt], L, stack, C, em);
    } else if (L.phase == kKinWait) {
        finish_collision<R, kCount, false>(P, sh[L.tgt], tabs[L.tgt], L, stack, C);
    } else if (L.phase == kEntry) {
        step_entry<R, kCount>(P, sh[L.tgt], tabs[L.tgt].R, L, C);
    } else if (L.phase == kEvap) {
        step_evap<R, kScaled, kCT, kCount>(P, L, C);
    }
}

}  // namespace
}  // namespace dev
}  // namespace pnuc
