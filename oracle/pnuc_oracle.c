/*
 * pnuc oracle: a plain, slow, FP64 CPU implementation of the proton-nucleus
 * intranuclear cascade + evaporation model of arXiv:1309.7963 (section 2), one event
 * at a time, in the order the model takes its steps.
 *
 * TEST INFRASTRUCTURE ONLY. The tests, the smoke check and the benchmark's CPU
 * baseline load it; the pnuc library never does. It shares no code, header, table or
 * constant generator with the CUDA path: both are written independently from the same
 * model reading.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared. No fused multiply-add, so the CUDA
 * FP64 mode (built with --fmad=false) differs from it only by libm ulps.
 *
 * Where the paper is silent the reading taken is stated beside the code. Parity of
 * each function is pinned in tests/test_oracle_*.py against library routines,
 * closed forms, measured NN cross sections and angular distributions, and conservation
 * laws. One piece has no such pin: orc_backward_a above p_lab = 0.8 GeV/c (parity
 * unpinned: no measured np backward-to-forward peak ratio is at hand; only its continuity
 * at 0.8 GeV/c and its decrease with momentum are tested).
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <string.h>

/* ------------------------------------------------------------------ constants */
#define HBARC 197.3269804 /* MeV fm */
#define E2 1.44           /* e^2, MeV fm */
#define M_P 938.272       /* MeV */
#define M_N 939.565
#define TWO_PI 6.283185307179586
#define PI 3.141592653589793
#define NSHELL 15

/* ejectiles in channel order n, p, d, t, 3He, alpha (section 2.4: He and lighter) */
static const double EJ_M[6] = {M_N, M_P, 1875.613, 2808.921, 2808.391, 3727.379};
static const int EJ_Z[6] = {0, 1, 1, 1, 2, 2};
static const int EJ_A[6] = {1, 1, 2, 3, 3, 4};
static const double EJ_G[6] = {2, 2, 3, 2, 2, 1};

/* flags */
#define F_BAD_INPUT 1u
#define F_ATTEMPT_CAP 2u
#define F_STEP_CAP 4u
#define F_STACK_OVERFLOW 8u
#define F_BAD_RESIDUAL 16u
#define F_NO_EXCITATION 32u
#define F_EVAP_TRIAL_CAP 64u
#define F_EVAP_STEP_CAP 128u
#define F_OUTPUT_OVERFLOW 256u

/* ------------------------------------------------------------------ types */
typedef struct {
    int32_t Z, A;
    double c, R, EC, ZoverA, M, S[2]; /* S[0] neutron, S[1] proton separation energy */
    double r[NSHELL + 1];
    double rho[NSHELL];
    double rho_s[2][NSHELL], pF[2][NSHELL], EF[2][NSHELL], V[2][NSHELL];
    double vF[NSHELL];
} orc_target;

typedef struct {
    uint32_t event;
    int32_t species, origin, index;
    double T, ux, uy, uz, px, py, pz;
} orc_secondary;

typedef struct {
    int32_t Zc, Ac, Zf, Af, n_casc, n_evap, n_coll, n_attempts;
    uint32_t flags, pad;
    double Estar_c, Estar_f, Pcas[3], Pf[3], Ef;
} orc_residual;

typedef struct {
    uint64_t steps, candidates, kinematics, pauli_blocked, collisions, crossings,
        reflections, escapes, captures, attempts, evap_steps, evap_trials, draws;
    /* E* settlements; six-channel width evaluations; open channels among them with
     * x = 2 sqrt(aY) >= 1 and < 1 (work counts, no effect on the results) */
    uint64_t settled, evap_passes, evap_exps, evap_series;
} orc_counters;

typedef struct {
    int32_t max_steps, max_attempts, stack_cap, max_evap_steps, max_evap_trials;
    int32_t level_density; /* 0: Fermi gas (reading M20); 1: constant temperature below U_x (M26) */
} orc_limits;

/* one trace entry per model decision (for hand-traced events and invariant tests) */
typedef struct {
    uint32_t event;
    int32_t kind, species, shell;
    double T, x, y, z;
} orc_trace;

enum {
    TR_ENTRY = 0, TR_CANDIDATE_NULL = 1, TR_PAULI = 2, TR_COLLISION = 3, TR_REFRACT = 4,
    TR_REFLECT = 5, TR_ESCAPE = 6, TR_CAPTURE = 7, TR_EVAP = 8, TR_PRODUCT = 9
};

/* ------------------------------------------------------------------ Philox4x64-10
 * Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11):
 * ten rounds of two 64x64->128 multiplications; the key is bumped by the Weyl
 * constants between rounds. */
void orc_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4])
{
    uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k0 += 0x9E3779B97F4A7C15ULL;
            k1 += 0xBB67AE8584CAA73BULL;
        }
        unsigned __int128 m0 = (unsigned __int128)0xD2E7470EE14C6C93ULL * c0;
        unsigned __int128 m1 = (unsigned __int128)0xCA5A826395121157ULL * c2;
        uint64_t hi0 = (uint64_t)(m0 >> 64), lo0 = (uint64_t)m0;
        uint64_t hi1 = (uint64_t)(m1 >> 64), lo1 = (uint64_t)m1;
        uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 32-bit half-word -> uniform in (0,1): h plus one half, over 2^32; exact in FP64 */
double orc_uniform(uint32_t h) { return ((double)h + 0.5) * 0x1p-32; }

/* The event's draw stream (reading M7): a Philox block (d/8, event, 0, 0), key (seed, 0),
 * gives 4 words = 8 draws; draw d is half d%2 (0: the high 32 bits, 1: the low) of word
 * (d/2)%4 of block d/8. A test may inject the first n_inject uniforms. */
typedef struct {
    uint64_t seed, event, next, block;
    uint64_t buf[4];
    int have;
    const double *inject;
    int64_t n_inject;
    orc_counters *cnt;
} orc_stream;

static void stream_init(orc_stream *st, uint64_t seed, uint64_t event, const double *inject,
                        int64_t n_inject, orc_counters *cnt)
{
    memset(st, 0, sizeof *st);
    st->seed = seed;
    st->event = event;
    st->inject = inject;
    st->n_inject = n_inject;
    st->cnt = cnt;
}

static double U(orc_stream *st)
{
    uint64_t d = st->next++;
    if (st->cnt) st->cnt->draws++;
    if ((int64_t)d < st->n_inject) return st->inject[d];
    uint64_t blk = d >> 3;
    if (!st->have || st->block != blk) {
        uint64_t ctr[4] = {blk, st->event, 0, 0}, key[2] = {st->seed, 0};
        orc_philox4x64_10(ctr, key, st->buf);
        st->block = blk;
        st->have = 1;
    }
    const uint64_t w = st->buf[(d >> 1) & 3];
    return orc_uniform((d & 1) ? (uint32_t)w : (uint32_t)(w >> 32));
}

/* The first n draws of an event's stream, as the simulation consumes them. */
void orc_stream_draws(uint64_t seed, uint64_t event, int64_t n, double *out)
{
    orc_stream st;
    stream_init(&st, seed, event, NULL, 0, NULL);
    for (int64_t i = 0; i < n; i++) out[i] = U(&st);
}

/* ------------------------------------------------------------------ small vector helpers */
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double mass_of(int s) { return s == 1 ? M_P : M_N; } /* nucleon species: 0 n, 1 p */
/* kinetic energy from |p|^2, without cancellation */
static double kinetic(double p2, double m) { return p2 / (sqrt(p2 + m * m) + m); }

/* ------------------------------------------------------------------ nucleus (section 2.2) */

/* Semi-empirical mass formula, textbook coefficient set; nuclear (not atomic) masses. */
double orc_semf_mass(int Z, int A)
{
    double a = A, z = Z, n = A - Z;
    double a13 = cbrt(a);
    double asym = a - 2.0 * z;
    double B = 15.75 * a - 17.8 * (a13 * a13) - 0.711 * z * (z - 1.0) / a13 - 23.7 * asym * asym / a;
    int zo = Z & 1, no = (A - Z) & 1;
    if (!zo && !no) B += 11.18 / sqrt(a);
    else if (zo && no) B -= 11.18 / sqrt(a);
    return z * M_P + n * M_N - B;
}

/* Eq. 1: Fermi (Woods-Saxon) profile */
static double fermi_profile(double r, double c) { return 1.0 / (1.0 + exp((r - c) / 0.545)); }

/* integral of r^2 f(r) over [a, b]: composite Simpson rule, 4096 panels */
static double shell_integral(double a, double b, double c)
{
    const int n = 4096;
    double h = (b - a) / n, sum = 0.0;
    for (int k = 0; k <= n; k++) {
        double r = a + k * h;
        double w = (k == 0 || k == n) ? 1.0 : ((k & 1) ? 4.0 : 2.0);
        sum += w * r * r * fermi_profile(r, c);
    }
    return sum * h / 3.0;
}

/* Builds the 15-shell table of a target (section 2.2). Returns 0, or 1 if (Z, A) is
 * outside the supported range. */
int orc_target_setup(int Z, int A, orc_target *t)
{
    memset(t, 0, sizeof *t);
    if (A < 6 || A > 250 || Z < 2 || A - Z < 2 || Z > 100) return 1;
    t->Z = Z;
    t->A = A;
    t->c = 1.07 * cbrt((double)A);
    t->R = t->c + 2.5; /* after Chen et al. */
    for (int k = 0; k <= NSHELL; k++) t->r[k] = k * t->R / NSHELL;
    double I[NSHELL], total = 0.0;
    for (int i = 0; i < NSHELL; i++) {
        I[i] = shell_integral(t->r[i], t->r[i + 1], t->c);
        total += I[i];
    }
    t->M = orc_semf_mass(Z, A);
    t->S[0] = orc_semf_mass(Z, A - 1) + M_N - t->M;     /* neutron separation energy */
    t->S[1] = orc_semf_mass(Z - 1, A - 1) + M_P - t->M; /* proton separation energy */
    if (!(t->S[0] > 0.0) || !(t->S[1] > 0.0)) return 1;
    t->EC = E2 * (Z - 1) / t->R;
    t->ZoverA = (double)Z / A;
    for (int i = 0; i < NSHELL; i++) {
        double r0 = t->r[i], r1 = t->r[i + 1];
        t->rho[i] = 3.0 * A * I[i] / (4.0 * PI * (r1 * r1 * r1 - r0 * r0 * r0) * total);
        t->rho_s[1][i] = ((double)Z / A) * t->rho[i];
        t->rho_s[0][i] = ((double)(A - Z) / A) * t->rho[i];
        double vmax = 0.0;
        for (int s = 0; s < 2; s++) {
            double m = mass_of(s);
            double pf = HBARC * cbrt(3.0 * PI * PI * t->rho_s[s][i]);
            t->pF[s][i] = pf;
            t->EF[s][i] = pf * pf / (sqrt(pf * pf + m * m) + m);
            t->V[s][i] = t->EF[s][i] + t->S[s];
            double v = pf / sqrt(pf * pf + m * m);
            if (v > vmax) vmax = v;
        }
        t->vF[i] = vmax;
    }
    return 0;
}

/* ------------------------------------------------------------------ NN cross sections (section 2.3)
 * Cugnon et al. parametrisations as recalled (p in GeV/c, sigma in mb). */
static double clamp_p(double p) { return p < 0.1 ? 0.1 : (p > 2.0 ? 2.0 : p); }

double orc_sigma(int like, double p)
{
    p = clamp_p(p);
    if (like) {
        if (p < 0.44) return 34.0 * pow(p / 0.4, -2.104);
        if (p < 0.8) {
            double d = p - 0.7;
            return 23.5 + 1000.0 * d * d * d * d;
        }
        double d = p - 1.3;
        return 1250.0 / (p + 50.0) - 4.0 * d * d;
    }
    if (p < 0.8) return 33.0 + 196.0 * pow(fabs(p - 0.95), 2.5);
    return 31.0 / sqrt(p);
}

/* slope B of d(sigma)/dt ~ exp(B t), (GeV/c)^-2 */
double orc_slope(int like, double p)
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

/* weight of the backward (u-channel) term for unlike pairs; above 0.8 GeV/c parity unpinned */
double orc_backward_a(double p)
{
    if (p <= 0.8) return 1.0;
    double r = 0.8 / p;
    return r * r;
}

/* Majorant of sigma * v_rel * E1 (GeV mb) over every partner of the shell's Fermi
 * spheres. Since v_rel = m2 p_lab/(E1 E2) <= p_lab/E1, sigma v_rel E1 <= g(p_lab) with
 * g(p) = p sigma(p). The pair momentum lies in [p_lo, p_hi] (partner velocity at most
 * v_F, collinear); g is bounded piecewise: the pp branch below 0.44 GeV/c decreases,
 * g_np < 31 below 0.8 GeV/c and rises above it, sigma_pp <= 28.1 mb above 0.44 GeV/c. */
double orc_g_hat(double p1, double E1, double vF)
{
    double plo = (p1 - vF * E1) * 1e-3;
    if (plo < 0.0) plo = 0.0;
    double phi = (p1 + vF * E1) * 1e-3 / sqrt((1.0 - vF) * (1.0 + vF));
    double pc = clamp_p(plo);
    double glo = pc < 0.44 ? pc * orc_sigma(1, pc) : 0.0;
    double ph = phi > 0.8 ? phi : 0.8;
    double g1 = 28.1 * ph;
    double g2 = 31.0 * ph / sqrt(ph < 2.0 ? ph : 2.0);
    double g = 31.0;
    if (glo > g) g = glo;
    if (g1 > g) g = g1;
    if (g2 > g) g = g2;
    return g;
}

/* cos(theta*) from one uniform: t in [-4p*^2, 0] with density ~ exp(B t) */
double orc_cos_theta(double B, double pstar_gev, double u)
{
    double b = 4.0 * B * pstar_gev * pstar_gev;
    double y = b > 0.0 ? -log1p(u * expm1(-b)) / b : u;
    return 1.0 - 2.0 * y;
}

/* rotate unit vector n by polar angle (ct, st) and azimuth phi */
void orc_rotate(const double n[3], double ct, double st, double phi, double d[3])
{
    double rho = sqrt(n[0] * n[0] + n[1] * n[1]);
    double cp = cos(phi), sp = sin(phi);
    if (rho > 0.0) {
        double e1[3] = {n[0] * n[2] / rho, n[1] * n[2] / rho, -rho};
        double e2[3] = {-n[1] / rho, n[0] / rho, 0.0};
        for (int k = 0; k < 3; k++) d[k] = ct * n[k] + st * (cp * e1[k] + sp * e2[k]);
    } else {
        d[0] = st * cp;
        d[1] = st * sp;
        d[2] = (n[2] >= 0.0 ? 1.0 : -1.0) * ct;
    }
}

/* Lorentz boost of (e, p) by velocity beta with gamma; sign -1 into the moving frame,
 * +1 out of it. */
static void boost(const double beta[3], double gamma, int sign, double e, const double p[3], double *eo, double po[3])
{
    double bp = dot3(beta, p);
    double g2 = gamma * gamma / (gamma + 1.0);
    double f = g2 * bp + sign * gamma * e;
    for (int k = 0; k < 3; k++) po[k] = p[k] + beta[k] * f;
    if (eo) *eo = gamma * (e + sign * bp);
}

/* Elastic NN collision with relativistic two-body kinematics (section 2.3). Species s1 with
 * momentum p1 on s2 with p2; three uniforms (t, phi*, backward flip). Writes the
 * products' momenta. */
void orc_collide(int s1, const double p1[3], int s2, const double p2[3], double ut, double uphi,
                 double uf, double q1[3], double q2[3])
{
    double m1 = mass_of(s1), m2 = mass_of(s2);
    int like = (s1 == s2);
    double pp1 = dot3(p1, p1), pp2 = dot3(p2, p2);
    double E1 = sqrt(pp1 + m1 * m1), E2v = sqrt(pp2 + m2 * m2);
    double T1 = kinetic(pp1, m1), T2 = kinetic(pp2, m2);
    double X = T1 * T2 + T1 * m2 + T2 * m1 - dot3(p1, p2);
    if (X < 0.0) X = 0.0;
    double k = sqrt(X * (X + 2.0 * m1 * m2));
    double plab = k / m2;
    double rs = sqrt((m1 + m2) * (m1 + m2) + 2.0 * X);
    double pst = k / rs;
    double Et = E1 + E2v;
    double beta[3] = {(p1[0] + p2[0]) / Et, (p1[1] + p2[1]) / Et, (p1[2] + p2[2]) / Et};
    double gamma = Et / rs;
    double p1c[3];
    boost(beta, gamma, -1, E1, p1, NULL, p1c);
    double nrm = sqrt(dot3(p1c, p1c));
    double n[3] = {p1c[0] / nrm, p1c[1] / nrm, p1c[2] / nrm};
    double ct = orc_cos_theta(orc_slope(like, plab * 1e-3), pst * 1e-3, ut);
    if (!like) {
        double a = orc_backward_a(plab * 1e-3);
        if (uf < a / (1.0 + a)) ct = -ct;
    }
    double st = sqrt((1.0 - ct) * (1.0 + ct));
    double d[3];
    orc_rotate(n, ct, st, TWO_PI * uphi, d);
    double k1[3] = {pst * d[0], pst * d[1], pst * d[2]};
    double k2[3] = {-k1[0], -k1[1], -k1[2]};
    double e1 = sqrt(pst * pst + m1 * m1), e2 = sqrt(pst * pst + m2 * m2);
    boost(beta, gamma, +1, e1, k1, NULL, q1);
    boost(beta, gamma, +1, e2, k2, NULL, q2);
}

/* Distance along d from r to the boundary of shell i; *dir = -1 inward, +1 outward. */
double orc_boundary_distance(const orc_target *t, int shell, const double r[3], const double d[3], int *dir)
{
    double beta = dot3(r, d), q = dot3(r, r);
    if (shell > 0 && beta < 0.0) {
        double ri = t->r[shell];
        double c = q - ri * ri, D = beta * beta - c;
        if (D > 0.0) {
            *dir = -1;
            double s = c / (-beta + sqrt(D));
            return s > 0.0 ? s : 0.0;
        }
    }
    double ro = t->r[shell + 1];
    double c = q - ro * ro;
    *dir = 1;
    /* moving inward, the particle is on or inside its outer sphere (it was reflected there
     * or came from inside): rounding that puts it outside must not shorten the chord */
    if (beta <= 0.0) return -beta + sqrt(beta * beta - (c > 0.0 ? 0.0 : c));
    double D = beta * beta - c;
    if (D < 0.0) D = 0.0;
    double s = -c / (beta + sqrt(D));
    return s > 0.0 ? s : 0.0;
}

/* Potential step at a shell boundary (section 2.3, after Chen et al.): kinetic energy
 * changes by dT with the tangential momentum kept. Returns 1 if the particle refracts
 * (p updated), 0 if it reflects (normal component reversed). n is the unit normal.
 * Reading M11: the refracted normal component takes the sign of the crossing, dir = +1 for
 * a crossing outward (along n), -1 inward. */
int orc_refract(const double n[3], double p[3], double m, double dT, int dir)
{
    double pp = dot3(p, p);
    double T = kinetic(pp, m), Tn = T + dT;
    double pn = dot3(p, n);
    double q2 = pn * pn + (Tn - T) * (Tn + T + 2.0 * m);
    if (Tn <= 0.0 || q2 <= 0.0) {
        for (int k = 0; k < 3; k++) p[k] -= 2.0 * pn * n[k];
        return 0;
    }
    double pnn = dir * sqrt(q2);
    for (int k = 0; k < 3; k++) p[k] += (pnn - pn) * n[k];
    return 1;
}

/* ------------------------------------------------------------------ evaporation (section 2.4) */

/* F(x) = e^x (x^2 - 3x + 3) + x^2/2 - 3 and G(x) = e^x (x - 1) + 1, by series below x = 1 */
static double width_F(double x)
{
    if (x >= 1.0) return exp(x) * (x * x - 3.0 * x + 3.0) + 0.5 * x * x - 3.0;
    double term = x * x * x / 6.0, sum = 0.0; /* term = x^n / n!, starting at n = 3 */
    for (int n = 4; n <= 20; n++) {
        term *= x / n;
        sum += (double)((n - 1) * (n - 3)) * term;
    }
    return sum;
}
static double width_G(double x)
{
    if (x >= 1.0) return exp(x) * (x - 1.0) + 1.0;
    double term = x, sum = 0.0; /* term = x^n / n!, starting at n = 1 */
    for (int n = 2; n <= 20; n++) {
        term *= x / n;
        sum += (double)(n - 1) * term;
    }
    return sum;
}

/* integral over U in [0, Y] of (Y + b - U) exp(2 sqrt(a U)) dU */
double orc_width_integral(double a, double Y, double b)
{
    double x = 2.0 * sqrt(a * Y);
    return width_F(x) / (4.0 * a * a) + b * width_G(x) / (2.0 * a);
}

/* Reading M26 (an option; M20's Fermi gas stays the default): the level density of GEM's
 * evaporation after Gilbert and Cameron, a constant-temperature form below the matching
 * energy U_x = 2.5 + 150/A_d MeV and the Fermi-gas form above it. Matched to M20's
 * exp(2 sqrt(a U)) in value and in slope at U_x, the constant-temperature part is
 * exp(sqrt(a U_x) + U / T) with 1/T = sqrt(a / U_x). A_d = 8a (a = A_d / 8). */
static double ct_Ux(double a) { return 2.5 + 150.0 / (8.0 * a); }

double orc_level_density(double a, double U, int mode)
{
    if (mode == 1) {
        double Ux = ct_Ux(a);
        if (U < Ux) return exp(sqrt(a * Ux) + U * sqrt(a / Ux));
    }
    return exp(2.0 * sqrt(a * U));
}

/* e^z - 1 - z, by series below z = 1/2 */
static double expm1_minus(double z)
{
    if (z >= 0.5) return expm1(z) - z;
    double term = z, sum = 0.0; /* term = z^n / n!, starting at n = 1 */
    for (int n = 2; n <= 20; n++) {
        term *= z / n;
        sum += term;
    }
    return sum;
}

/* Reading M26's width integral: over U in [0, Y] of (Y + b - U) rho(U) dU with rho the
 * composite density. The constant-temperature part over [0, L], L = min(Y, U_x), is
 * C [(Y + b - L)(e^{kL} - 1)/k + (e^{kL} - 1 - kL)/k^2] with k = 1/T, C = e^{sqrt(a U_x)};
 * above U_x the Fermi-gas part is M20's integral over [0, Y] less the same integrand over
 * [0, U_x], (Y + b)/(2a) G(x_x) - H(x_x)/(8a^2), x_x = 2 sqrt(a U_x), H(x) = e^x (x^3 - 3x^2 +
 * 6x - 6) + 6. Writes the constant-temperature part to *ct_part (if not NULL). */
double orc_width_integral_ct(double a, double Y, double b, double *ct_part)
{
    double Ux = ct_Ux(a), k = sqrt(a / Ux), xx = 2.0 * sqrt(a * Ux);
    double L = Y < Ux ? Y : Ux, kL = k * L;
    double ict = exp(0.5 * xx) * ((Y + b - L) * expm1(kL) / k + expm1_minus(kL) / (k * k));
    if (ct_part) *ct_part = ict;
    if (!(Y > Ux)) return ict;
    double ex = exp(xx);
    double Gx = ex * (xx - 1.0) + 1.0;
    double Hx = ex * (((xx - 3.0) * xx + 6.0) * xx - 6.0) + 6.0;
    double below = (Y + b) * Gx / (2.0 * a) - Hx / (8.0 * a * a);
    return ict + (orc_width_integral(a, Y, b) - below);
}

/* Channel parameters of ejectile j from parent (Z, A) at excitation Estar, with the level
 * density of reading M20 (ld = 0) or M26 (ld = 1). Returns the unnormalised width; writes
 * barrier V, offset b, Q, daughter mass Md, level-density parameter a and x = 2 sqrt(a Y).
 * Closed channels return 0. */
double orc_channel_ld(int Z, int A, double Estar, int j, int ld, double *V_out, double *b_out, double *Q_out,
                      double *Md_out, double *a_out, double *x_out)
{
    int Zd = Z - EJ_Z[j], Ad = A - EJ_A[j];
    *V_out = *b_out = *Q_out = *Md_out = *a_out = *x_out = 0.0;
    if (Zd < 1 || Ad - Zd < 1 || Ad < 5) return 0.0;
    double Md = orc_semf_mass(Zd, Ad);
    double Q = Md + EJ_M[j] - orc_semf_mass(Z, A);
    double A3 = cbrt((double)Ad);
    double V, b, cj;
    if (EJ_Z[j] == 0) {
        /* Dostrovsky inverse cross section for neutrons, GEM constants */
        double alpha = 0.76 + 1.93 / A3;
        double beta = (1.66 / (A3 * A3) - 0.05) / alpha;
        V = beta < 0.0 ? -beta : 0.0;
        b = beta > 0.0 ? beta : 0.0;
        cj = alpha;
    } else {
        /* charged: sigma_g (1 - V/eps) above the Coulomb barrier, r0 = 1.5 fm */
        V = E2 * EJ_Z[j] * Zd / (1.5 * (cbrt((double)EJ_A[j]) + A3));
        b = 0.0;
        cj = 1.0;
    }
    double X = Estar - Q, Y = X - V;
    *V_out = V;
    *b_out = b;
    *Q_out = Q;
    *Md_out = Md;
    double a = Ad / 8.0;
    *a_out = a;
    if (!(Y > 0.0)) return 0.0;
    *x_out = 2.0 * sqrt(a * Y);
    double I = ld == 1 ? orc_width_integral_ct(a, Y, b, NULL) : orc_width_integral(a, Y, b);
    return EJ_G[j] * EJ_M[j] * cj * (A3 * A3) * I;
}

double orc_channel(int Z, int A, double Estar, int j, double *V_out, double *b_out, double *Q_out,
                   double *Md_out, double *a_out, double *x_out)
{
    return orc_channel_ld(Z, A, Estar, j, 0, V_out, b_out, Q_out, Md_out, a_out, x_out);
}

/* Rejection sampler for t in [0, x] with density h(t) ~ [t(2x - t)/(4a) + b](x - t) e^-t.
 * Four uniforms per trial. The envelope is W1 t e^-t + W2 e^-t (W1 = x^2/(2a), W2 = b x):
 * for x >= 2 its two parts are sampled as Gamma(2,1) and Exp(1); for x < 2 the factor
 * e^-t is dropped from the envelope and its parts, W1 t and W2 on [0, x], are sampled as
 * x max(u1, u2) and x u1. Returns t, or -1 after max_trials. */
static double sample_t(orc_stream *st, double a, double x, double b, int max_trials, int *trials)
{
    double W1 = x * x / (2.0 * a), W2 = b * x;
    int small = x < 2.0;
    double pmix = small ? W1 * x / (W1 * x + 2.0 * W2) : W1 / (W1 + W2);
    for (int k = 0; k < max_trials; k++) {
        double um = U(st), u1 = U(st), u2 = U(st), ua = U(st);
        (*trials)++;
        int first = um < pmix;
        double t;
        if (small) t = first ? x * (u1 > u2 ? u1 : u2) : x * u1;
        else t = first ? -log(u1 * u2) : -log(u1);
        if (t >= x) continue;
        double h = (t * (2.0 * x - t) / (4.0 * a) + b) * (x - t);
        if (small) h *= exp(-t);
        if (ua * (W1 * t + W2) < h) return t;
    }
    return -1.0;
}

/* Reading M26's emission sampler: the daughter's excitation U in [0, Y] with density
 * ~ (Y + b - U) rho(U), rho the composite level density. One draw picks the part, the
 * constant-temperature one (U < L = min(Y, U_x)) with probability I_ct / I; then trials of
 * four draws (um, u1, u2, ua) as in sample_t. Constant-temperature part: t = k (L - U) in
 * [0, kL] has density ~ (c0 + t) e^-t, c0 = k (Y + b - L): for kL >= 2 the mixture of
 * Exp(1) (weight c0) and Gamma(2,1) (weight 1), kept if t < kL; for kL < 2 the mixture of
 * kL u1 (weight c0 kL) and kL max(u1, u2) (weight (kL)^2 / 2), kept with probability e^-t.
 * Fermi-gas part: sample_t's trial on [0, x], kept if t < x - x_x (U > U_x). Returns U, or
 * -1 after max_trials. */
static double sample_U_ct(orc_stream *st, double a, double Y, double b, double x, int max_trials, int *trials)
{
    double Ux = ct_Ux(a), k = sqrt(a / Ux), xx = 2.0 * sqrt(a * Ux);
    double ict, itot = orc_width_integral_ct(a, Y, b, &ict);
    double up = U(st);
    if (up * itot < ict) {
        double L = Y < Ux ? Y : Ux, kL = k * L, c0 = k * (Y + b - L);
        int small = kL < 2.0;
        double pmix = small ? c0 * kL / (c0 * kL + 0.5 * kL * kL) : c0 / (c0 + 1.0);
        for (int n = 0; n < max_trials; n++) {
            double um = U(st), u1 = U(st), u2 = U(st), ua = U(st);
            (*trials)++;
            int first = um < pmix;
            double t;
            if (small) {
                t = first ? kL * u1 : kL * (u1 > u2 ? u1 : u2);
                if (!(ua < exp(-t))) continue;
            } else {
                t = first ? -log(u1) : -log(u1 * u2);
                if (!(t < kL)) continue;
            }
            return L - t / k;
        }
        return -1.0;
    }
    double W1 = x * x / (2.0 * a), W2 = b * x;
    int small = x < 2.0;
    double pmix = small ? W1 * x / (W1 * x + 2.0 * W2) : W1 / (W1 + W2);
    double tmax = x - xx;
    for (int n = 0; n < max_trials; n++) {
        double um = U(st), u1 = U(st), u2 = U(st), ua = U(st);
        (*trials)++;
        int first = um < pmix;
        double t;
        if (small) t = first ? x * (u1 > u2 ? u1 : u2) : x * u1;
        else t = first ? -log(u1 * u2) : -log(u1);
        if (t >= tmax) continue;
        double h = (t * (2.0 * x - t) / (4.0 * a) + b) * (x - t);
        if (small) h *= exp(-t);
        if (ua * (W1 * t + W2) < h) return (x - t) * (x - t) / (4.0 * a);
    }
    return -1.0;
}

/* test entry: n samples of M26's emission sampler on a Philox stream (seed, event) */
int64_t orc_sample_U_ct(double a, double Y, double b, uint64_t seed, uint64_t event, int64_t n, double *out)
{
    orc_stream st;
    stream_init(&st, seed, event, NULL, 0, NULL);
    int64_t trials = 0;
    double x = 2.0 * sqrt(a * Y);
    for (int64_t i = 0; i < n; i++) {
        int tr = 0;
        out[i] = sample_U_ct(&st, a, Y, b, x, 1 << 30, &tr);
        trials += tr;
    }
    return trials;
}

/* test entry: the sampler on a Philox stream (seed, event), n samples of U = (x-t)^2/(4a) */
int64_t orc_sample_U(double a, double x, double b, uint64_t seed, uint64_t event, int64_t n, double *out)
{
    orc_stream st;
    stream_init(&st, seed, event, NULL, 0, NULL);
    int64_t trials = 0;
    for (int64_t i = 0; i < n; i++) {
        int tr = 0;
        double t = sample_t(&st, a, x, b, 1 << 30, &tr);
        trials += tr;
        out[i] = (x - t) * (x - t) / (4.0 * a);
    }
    return trials;
}

/* test entry: n partner momenta of the Fermi sphere p_F on a Philox stream */
void orc_sample_fermi(double pF, uint64_t seed, uint64_t event, int64_t n, double *out3)
{
    orc_stream st;
    stream_init(&st, seed, event, NULL, 0, NULL);
    for (int64_t i = 0; i < n; i++) {
        double q = pF * cbrt(U(&st));
        double ct = 2.0 * U(&st) - 1.0;
        double sn = sqrt((1.0 - ct) * (1.0 + ct));
        double ph = TWO_PI * U(&st);
        out3[3 * i] = q * sn * cos(ph);
        out3[3 * i + 1] = q * sn * sin(ph);
        out3[3 * i + 2] = q * ct;
    }
}

/* ------------------------------------------------------------------ one event */
typedef struct {
    int s, shell;
    double r[3], p[3];
} particle;

typedef struct {
    orc_secondary *sec;
    uint64_t cap, count;
    orc_trace *trace;
    uint64_t trace_cap, trace_count;
} sink;

static void trace_put(sink *o, uint32_t ev, int kind, int s, int shell, double T, const double *r)
{
    if (!o->trace) return;
    if (o->trace_count < o->trace_cap) {
        orc_trace *e = &o->trace[o->trace_count];
        e->event = ev;
        e->kind = kind;
        e->species = s;
        e->shell = shell;
        e->T = T;
        e->x = r ? r[0] : 0.0;
        e->y = r ? r[1] : 0.0;
        e->z = r ? r[2] : 0.0;
    }
    o->trace_count++;
}

static int emit(sink *o, uint32_t ev, int species, int origin, int index, double T, const double p[3])
{
    if (o->count < o->cap) {
        orc_secondary *s = &o->sec[o->count];
        double pn = sqrt(dot3(p, p));
        s->event = ev;
        s->species = species;
        s->origin = origin;
        s->index = index;
        s->T = T;
        s->ux = p[0] / pn;
        s->uy = p[1] / pn;
        s->uz = p[2] / pn;
        s->px = p[0];
        s->py = p[1];
        s->pz = p[2];
        o->count++;
        return 1;
    }
    o->count++;
    return 0;
}

/* One event: a nucleon of species proj (1 proton, 0 neutron: the incident particle of a
 * proton- or neutron-induced interaction) at kinetic energy T0 on target t. */
static void run_event(const orc_target *t, int proj, double T0, uint32_t ev, orc_stream *st, const orc_limits *L,
                      sink *o, orc_residual *res, orc_counters *c)
{
    memset(res, 0, sizeof *res);
    res->Zc = res->Zf = t->Z;
    res->Ac = res->Af = t->A;
    if (!(T0 >= 20.0 && T0 <= 250.0)) {
        res->flags |= F_BAD_INPUT;
        return;
    }
    const double mproj = mass_of(proj);
    const double p0 = sqrt(T0 * T0 + 2.0 * T0 * mproj);
    int n_index = 0, n_coll = 0, n_p_esc = 0, n_esc = 0;
    double Esum = 0.0, Psum[3] = {0, 0, 0};
    particle stack[256];
    int cap = L->stack_cap < 256 ? L->stack_cap : 256;
    int64_t steps = 0;
    int attempt = 0, done = 0;

    /* -------- cascade with the non-elastic retry */
    while (!done) {
        if (attempt >= L->max_attempts) {
            res->flags |= F_ATTEMPT_CAP;
            res->n_attempts = attempt;
            return;
        }
        attempt++;
        c->attempts++;
        /* entry on the projected disk of radius R, refracted into the surface shell */
        double b = t->R * sqrt(U(st));
        double phi = TWO_PI * U(st);
        particle cur;
        cur.s = proj;
        cur.shell = NSHELL - 1;
        cur.r[0] = b * cos(phi);
        cur.r[1] = b * sin(phi);
        cur.r[2] = -sqrt(t->R * t->R - b * b);
        cur.p[0] = 0.0;
        cur.p[1] = 0.0;
        cur.p[2] = p0;
        {
            double rr = sqrt(dot3(cur.r, cur.r));
            double n[3] = {cur.r[0] / rr, cur.r[1] / rr, cur.r[2] / rr};
            orc_refract(n, cur.p, mproj, t->V[proj][NSHELL - 1], -1);
        }
        trace_put(o, ev, TR_ENTRY, proj, cur.shell, kinetic(dot3(cur.p, cur.p), mproj), cur.r);
        int sp = 0;      /* stack depth */
        int alive = 1;   /* cur holds a particle */
        while (alive) {
            /* ---- one transport step of cur */
            if (steps >= L->max_steps) {
                res->flags |= F_STEP_CAP;
                alive = 0;
                sp = 0;
                done = 1;
                break;
            }
            steps++;
            c->steps++;
            int s1 = cur.s, i = cur.shell;
            double m1 = mass_of(s1);
            double pp = dot3(cur.p, cur.p), pm = sqrt(pp);
            double E1 = sqrt(pp + m1 * m1);
            double d[3] = {cur.p[0] / pm, cur.p[1] / pm, cur.p[2] / pm};
            int dir;
            double sb = orc_boundary_distance(t, i, cur.r, d, &dir);
            double gh = orc_g_hat(pm, E1, t->vF[i]);
            double Sigma = 0.1 * t->rho[i] * gh / (pm * 1e-3);
            double s = -log(U(st)) / Sigma;
            if (s < sb) {
                /* ---- candidate collision (Metropolis sequence) */
                for (int k = 0; k < 3; k++) cur.r[k] += s * d[k];
                c->candidates++;
                int s2 = (U(st) < t->ZoverA) ? 1 : 0;
                double m2 = mass_of(s2);
                double q = t->pF[s2][i] * cbrt(U(st));
                double ct = 2.0 * U(st) - 1.0;
                double sn = sqrt((1.0 - ct) * (1.0 + ct));
                double ph = TWO_PI * U(st);
                double p2[3] = {q * sn * cos(ph), q * sn * sin(ph), q * ct};
                double T1 = kinetic(pp, m1), T2 = kinetic(q * q, m2);
                double E2v = sqrt(q * q + m2 * m2);
                double X = T1 * T2 + T1 * m2 + T2 * m1 - dot3(cur.p, p2);
                if (X < 0.0) X = 0.0;
                double kk = sqrt(X * (X + 2.0 * m1 * m2));
                double plab = kk / m2;
                double vrel = kk / (E1 * E2v);
                double sig = orc_sigma(s1 == s2, plab * 1e-3);
                double ua = U(st);
                if (!(ua * gh < sig * vrel * E1 * 1e-3)) {
                    trace_put(o, ev, TR_CANDIDATE_NULL, s1, i, T1, cur.r);
                    continue;
                }
                c->kinematics++;
                double ut = U(st), uph = U(st), uf = U(st);
                double q1[3], q2[3];
                orc_collide(s1, cur.p, s2, p2, ut, uph, uf, q1, q2);
                double T1n = kinetic(dot3(q1, q1), m1), T2n = kinetic(dot3(q2, q2), m2);
                if (!(T1n > t->EF[s1][i] && T2n > t->EF[s2][i])) {
                    c->pauli_blocked++;
                    trace_put(o, ev, TR_PAULI, s1, i, T1, cur.r);
                    continue;
                }
                /* accepted collision */
                c->collisions++;
                n_coll++;
                trace_put(o, ev, TR_COLLISION, s1, i, T1, cur.r);
                double cut2 = t->V[s2][i] + (s2 == 1 ? t->EC : 0.0);
                double cut1 = t->V[s1][i] + (s1 == 1 ? t->EC : 0.0);
                trace_put(o, ev, TR_PRODUCT, s1, i, T1n, cur.r);
                trace_put(o, ev, TR_PRODUCT, s2, i, T2n, cur.r);
                if (T2n < cut2) {
                    c->captures++;
                    trace_put(o, ev, TR_CAPTURE, s2, i, T2n, cur.r);
                } else if (sp >= cap) {
                    res->flags |= F_STACK_OVERFLOW;
                    c->captures++;
                    trace_put(o, ev, TR_CAPTURE, s2, i, T2n, cur.r);
                } else {
                    particle *np = &stack[sp++];
                    np->s = s2;
                    np->shell = i;
                    memcpy(np->r, cur.r, sizeof cur.r);
                    memcpy(np->p, q2, sizeof q2);
                }
                memcpy(cur.p, q1, sizeof q1);
                if (T1n < cut1) {
                    c->captures++;
                    trace_put(o, ev, TR_CAPTURE, s1, i, T1n, cur.r);
                    if (sp > 0) cur = stack[--sp];
                    else alive = 0;
                }
                continue;
            }
            /* ---- move to the boundary and cross it */
            for (int k = 0; k < 3; k++) cur.r[k] += sb * d[k];
            c->crossings++;
            int j = i + dir; /* j == NSHELL: outside */
            double dT = -t->V[s1][i] + (j == NSHELL ? 0.0 : t->V[s1][j]);
            double rr = sqrt(dot3(cur.r, cur.r));
            double n[3] = {cur.r[0] / rr, cur.r[1] / rr, cur.r[2] / rr};
            double Tb = kinetic(pp, m1);
            if (!orc_refract(n, cur.p, m1, dT, dir)) {
                c->reflections++;
                trace_put(o, ev, TR_REFLECT, s1, i, Tb, cur.r);
                continue;
            }
            cur.shell = j;
            if (j < NSHELL) {
                trace_put(o, ev, TR_REFRACT, s1, j, Tb + dT, cur.r);
                continue;
            }
            /* escape */
            double Tout = Tb + dT;
            trace_put(o, ev, TR_ESCAPE, s1, i, Tout, cur.r);
            if (n_coll > 0) {
                c->escapes++;
                emit(o, ev, s1, 0, n_index++, Tout, cur.p);
                Esum += Tout + m1;
                for (int k = 0; k < 3; k++) Psum[k] += cur.p[k];
                n_esc++;
                if (s1 == 1) n_p_esc++;
            }
            if (sp > 0) cur = stack[--sp];
            else alive = 0;
        }
        if (n_coll > 0) done = 1;
    }
    res->n_attempts = attempt;
    res->n_coll = n_coll;
    res->n_casc = n_index;

    /* -------- excitation energy through energy conservation (section 2.3, as in
     * Metropolis et al.): the static mean field absorbs the cascade's momentum imbalance
     * but does no work, so E* is the energy balance in the target rest frame and the
     * residual starts the evaporation at rest. */
    int Z = t->Z + proj - n_p_esc, A = t->A + 1 - n_esc;
    c->settled++;
    res->Zc = res->Zf = Z;
    res->Ac = res->Af = A;
    double Er = T0 + mproj + t->M - Esum;
    double Pr[3] = {0.0, 0.0, 0.0};
    res->Pcas[0] = -Psum[0];
    res->Pcas[1] = -Psum[1];
    res->Pcas[2] = p0 - Psum[2];
    res->Ef = Er;
    if (Z < 1 || A - Z < 1) {
        res->flags |= F_BAD_RESIDUAL;
        return;
    }
    double Mc = orc_semf_mass(Z, A);
    double Estar = Er - Mc;
    res->Estar_c = res->Estar_f = Estar;
    if (!(Estar > 0.0)) {
        res->flags |= F_NO_EXCITATION;
        return;
    }
    Er = Mc + Estar; /* the excited residual at rest: its total energy is M + E* */

    /* -------- evaporation (section 2.4) */
    int step;
    for (step = 0; step < L->max_evap_steps; step++) {
        double G[6], V[6], bj[6], Q[6], Md[6], a[6], x[6], S = 0.0;
        c->evap_passes++;
        for (int j = 0; j < 6; j++) {
            G[j] = orc_channel_ld(Z, A, Estar, j, L->level_density, &V[j], &bj[j], &Q[j], &Md[j], &a[j], &x[j]);
            S += G[j];
            if (G[j] > 0.0) {
                if (x[j] >= 1.0) c->evap_exps++;
                else c->evap_series++;
            }
        }
        if (!(S > 0.0)) break;
        c->evap_steps++;
        double us = U(st) * S, cum = 0.0;
        int ch = -1;
        for (int j = 0; j < 6; j++) {
            cum += G[j];
            if (us < cum) {
                ch = j;
                break;
            }
        }
        if (ch < 0)
            for (int j = 5; j >= 0; j--)
                if (G[j] > 0.0) {
                    ch = j;
                    break;
                }
        int trials = 0;
        double X = Estar - Q[ch];
        double Ud;
        if (L->level_density == 1) {
            Ud = sample_U_ct(st, a[ch], X - V[ch], bj[ch], x[ch], L->max_evap_trials, &trials);
        } else {
            double tt = sample_t(st, a[ch], x[ch], bj[ch], L->max_evap_trials, &trials);
            Ud = tt < 0.0 ? -1.0 : (x[ch] - tt) * (x[ch] - tt) / (4.0 * a[ch]);
        }
        c->evap_trials += trials;
        if (Ud < 0.0) {
            res->flags |= F_EVAP_TRIAL_CAP;
            break;
        }
        double eps = X - Ud;
        /* two-body decay, isotropic in the rest frame, boosted to the lab */
        double W = orc_semf_mass(Z, A) + Estar;
        double m1 = EJ_M[ch], m2 = Md[ch] + Ud;
        double pd = sqrt(eps * (W + m1 + m2) * (W - m1 + m2) * (W + m1 - m2)) / (2.0 * W);
        double ct = 2.0 * U(st) - 1.0;
        double ph = TWO_PI * U(st);
        double sn = sqrt((1.0 - ct) * (1.0 + ct));
        double pv[3] = {pd * sn * cos(ph), pd * sn * sin(ph), pd * ct};
        double e1 = sqrt(pd * pd + m1 * m1);
        double Pm2 = sqrt(dot3(Pr, Pr));
        double gamma = Er / sqrt((Er - Pm2) * (Er + Pm2));
        double beta[3] = {Pr[0] / Er, Pr[1] / Er, Pr[2] / Er};
        double pl[3], el;
        boost(beta, gamma, +1, e1, pv, &el, pl);
        double Tl = kinetic(dot3(pl, pl), m1);
        emit(o, ev, ch, 1, n_index++, Tl, pl);
        {
            double info[3] = {V[ch], Q[ch], Estar}; /* barrier, Q-value, parent excitation */
            trace_put(o, ev, TR_EVAP, ch, 1000 * Z + A, eps, info);
        }
        res->n_evap++;
        Er -= el;
        for (int k = 0; k < 3; k++) Pr[k] -= pl[k];
        Z -= EJ_Z[ch];
        A -= EJ_A[ch];
        Estar = Ud;
    }
    if (step == L->max_evap_steps) res->flags |= F_EVAP_STEP_CAP;
    res->Zf = Z;
    res->Af = A;
    res->Estar_f = Estar;
    res->Ef = Er;
    memcpy(res->Pf, Pr, sizeof Pr);
}

/* ------------------------------------------------------------------ batch entry point
 * Simulates events first_event_id + k (k < n): a nucleon of species projectiles[k] (1 proton,
 * 0 neutron; all protons if projectiles is NULL) at energies[k] MeV on targets[tidx[k]].
 * Secondaries are written in event order (at most sec_cap); the return value is the
 * number produced. inject/n_inject, if given, replace the first draws of every event.
 * trace/trace_cap, if given, receive one entry per model decision. */
uint64_t orc_simulate(const orc_target *targets, int32_t n_targets, const double *energies,
                      const int32_t *tidx, const int32_t *projectiles, uint64_t n, uint64_t seed,
                      uint64_t first_event_id,
                      orc_secondary *sec, uint64_t sec_cap, orc_residual *res, orc_counters *cnt,
                      const orc_limits *lim, const double *inject, int64_t n_inject, orc_trace *trace,
                      uint64_t trace_cap, uint64_t *trace_count)
{
    sink o = {sec, sec_cap, 0, trace, trace_cap, 0};
    orc_counters local;
    if (!cnt) {
        memset(&local, 0, sizeof local);
        cnt = &local;
    }
    for (uint64_t k = 0; k < n; k++) {
        int32_t ti = tidx[k];
        const int proj = projectiles ? projectiles[k] : 1;
        uint64_t before = o.count;
        if (ti < 0 || ti >= n_targets || (proj != 0 && proj != 1)) {
            memset(&res[k], 0, sizeof res[k]);
            res[k].flags = F_BAD_INPUT;
            continue;
        }
        orc_stream st;
        stream_init(&st, seed, first_event_id + k, inject, n_inject, cnt);
        run_event(&targets[ti], proj, energies[k], (uint32_t)k, &st, lim, &o, &res[k], cnt);
        if (o.count > sec_cap && before < o.count) res[k].flags |= F_OUTPUT_OVERFLOW;
    }
    if (trace_count) *trace_count = o.trace_count;
    return o.count;
}

/* sizes of the record types, so that the Python side can check its layouts */
int64_t orc_sizeof(int which)
{
    switch (which) {
    case 0: return (int64_t)sizeof(orc_target);
    case 1: return (int64_t)sizeof(orc_secondary);
    case 2: return (int64_t)sizeof(orc_residual);
    case 3: return (int64_t)sizeof(orc_counters);
    case 4: return (int64_t)sizeof(orc_limits);
    case 5: return (int64_t)sizeof(orc_trace);
    }
    return -1;
}
