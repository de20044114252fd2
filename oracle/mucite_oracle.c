/*
 * Oracle for the MuCITE ion-pack time step: plain, slow, FP64 CPU code.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call this file;
 * the tests, the package smoke check and the benchmark's CPU-baseline leg are
 * its only users. It shares no source with the CUDA library.
 *
 * What it follows (Yan, Lengyel, Rosu, Gabelica, "Multiphysics Simulation
 * Framework for Continuous Ion Transport and Energetics in Atmospheric
 * Pressure Interfaces"):
 *   - field evaluation: bilinear interpolation of baked (r,z) grids, Cartesian
 *     projection of E_r (Eq. 3), total field E_DC + E_RF*V/Vref*cos(2 pi f t
 *     + phi) + E_SCE (Eq. 4); gas velocity, temperature and pressure gathered
 *     at the ion (Methods, "Gas field and electrode mask coupling");
 *   - collisions: rate n*sigma*|v_ion - v_gas| (Eq. 6) with the gas partner
 *     drawn from the local Maxwellian about the flow, hard-sphere isotropic
 *     scattering, internal-energy exchange converted to T_eff through the
 *     heat-capacity profile (Methods, "Particle transport, collisions, and
 *     effective internal temperature");
 *   - push: leapfrog kick/drift (the paper uses RK4; the leapfrog reading is
 *     documented with the design);
 *   - terminal classes: electrode hit from the nearest mask node and surface
 *     distance, radial loss, transmitted across the detector plane within the
 *     detector radius, axial exit ("Terminal events" paragraph);
 *   - CIC deposit of q*W onto the axisymmetric PIC grid ("Axisymmetric PIC
 *     space charge update");
 *   - continuous-current source accumulator (Eq. 5) and source sampling
 *     ("Continuous current Gaussian source").
 * Random numbers: Philox4x32-10 written from its published definition
 * (Salmon, Moraes, Dror, Shaw, SC'11), keyed by (seed) with counter
 * (pack id, step, draw block, purpose).
 *
 * Parity status of each function is stated at its definition. Functions that
 * implement the IICT energy partition are "parity unpinned" against the
 * paper (the paper does not print the IICT equations); they are pinned only
 * by invariants (detailed balance, sampler moments).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_E_CHARGE 1.602176634e-19
#define ORC_KB 1.380649e-23
#define ORC_DALTON 1.66053906660e-27
#define ORC_PI 3.14159265358979323846
#define ORC_KMAX 32 /* candidate collisions examined per pack per step */
#define ORC_PLANCK 6.62607015e-34
#define ORC_NA 6.02214076e23

enum { ORC_ACTIVE = 0, ORC_TRANSMITTED = 1, ORC_ELECTRODE = 2, ORC_RADIAL = 3, ORC_AXIAL = 4,
       ORC_EMPTY = 255 };

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon et al. SC'11): 10 rounds of two 32x32->64 products,  */
/* key schedule advanced by the two Weyl constants between rounds.            */
/* Pinned by known answers against an independent open-source Philox4x32-10 */
/* (PyTorch's ATen philox_engine) and by statistical tests.                  */
/* ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 23-bit uniform in (0,1): ((x >> 9) + 1/2) * 2^-23, exact in FP32 and FP64. */
static double u01(uint32_t x) { return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0); }

/* Four uniforms for (pack, step, block, purpose) under key (seed). */
static void draw4(uint64_t seed, uint32_t pack, uint32_t step, uint32_t block, uint32_t purpose,
                  double u[4])
{
    uint32_t ctr[4] = {pack, step, block, purpose};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    orc_philox4x32_10(ctr, key, o);
    for (int i = 0; i < 4; ++i) u[i] = u01(o[i]);
}

void orc_uniforms(uint64_t seed, uint32_t pack, uint32_t step, uint32_t block, uint32_t purpose,
                  double *u)
{
    draw4(seed, pack, step, block, purpose, u);
}

/* ------------------------------------------------------------------------- */
/* Problem description (independent of the CUDA library's structs).          */
/* ------------------------------------------------------------------------- */
typedef struct {
    int nr, nz;
    double R, z0, z1;
    /* node arrays [nz][nr], FP64 */
    const double *er_dc, *ez_dc, *er_rf, *ez_rf;
    const double *gas_p, *gas_T, *gas_ur, *gas_uz;
    const float *dmask; /* -1 at metal nodes, else FP32 surface distance */
    /* optional space-charge field on the PIC grid [pnz][pnr] */
    int pnr, pnz;
    const double *er_sc, *ez_sc;
} orc_fields;

typedef struct {
    double mass_da, charge, ccs_m2, n_atoms, cv_c0, cv_c1, T_init;
    double dH_kJmol, dS_JmolK; /* transition-state parameters; dH <= 0 disables Eq. 7 */
} orc_ion;

typedef struct {
    int profile;
    double z_plane, radius, sigma, T_vel;
    int half_space;
    double prefill_z0, prefill_z1;
} orc_source;

typedef struct {
    double dt, v_rf, f_rf, phi_rf, dc_scale, p_scale, hit_dist, z_exit, r_det, m_gas_da;
    uint64_t seed;
    int langevin;                    /* hybrid Langevin branch on */
    double lv_z0, lv_z1, lv_switch;  /* axial window and lambda*dt threshold */
    int integrator;                  /* 0 leapfrog, 1 RK4 */
    double rf_phase0;                /* RF phase (cycles) at the start of the current dt segment */
    int64_t seg_step0;               /* step count at the start of the current dt segment */
} orc_run;

typedef struct {
    double *x, *y, *z, *vx, *vy, *vz, *eint; /* eint = E_int / k_B [K] */
    uint8_t *status;
    int32_t *t_term;
    int64_t *ncoll;    /* accepted collisions per pack (diagnostic) */
    int64_t *nsteps;   /* active steps advanced per pack */
    int64_t *noverflow;/* steps where the candidate cap was reached */
    double *lnsy;      /* ln of the precursor survival yield SY (Eq. 7) */
    double *tau;       /* optical depth left until the next collision candidate */
} orc_state;

/* ------------------------------------------------------------------------- */
/* Heat-capacity profile Cv/k_B = 3N * min(1, c0 + c1*T): E_int(T) and its   */
/* inverse (T_eff from internal energy). Pinned: inverse(E(T)) == T tests.    */
/* ------------------------------------------------------------------------- */
static double tcap_of(const orc_ion *ion)
{
    return ion->cv_c1 > 0.0 ? (1.0 - ion->cv_c0) / ion->cv_c1 : INFINITY;
}

double orc_eint_of_T(const orc_ion *ion, double T)
{
    double n3 = 3.0 * ion->n_atoms;
    double tc = tcap_of(ion);
    if (T <= tc) return n3 * (ion->cv_c0 * T + 0.5 * ion->cv_c1 * T * T);
    double ec = ion->cv_c0 * tc + 0.5 * ion->cv_c1 * tc * tc;
    return n3 * (ec + (T - tc));
}

double orc_T_of_eint(const orc_ion *ion, double eint)
{
    double n3 = 3.0 * ion->n_atoms;
    double e = eint / n3;
    double tc = tcap_of(ion);
    double ec = isinf(tc) ? INFINITY : ion->cv_c0 * tc + 0.5 * ion->cv_c1 * tc * tc;
    if (e <= ec) return 2.0 * e / (ion->cv_c0 + sqrt(ion->cv_c0 * ion->cv_c0 + 2.0 * ion->cv_c1 * e));
    return tc + (e - ec);
}

double orc_cv_of_T(const orc_ion *ion, double T)
{
    double f = ion->cv_c0 + ion->cv_c1 * T;
    return 3.0 * ion->n_atoms * (f < 1.0 ? f : 1.0);
}

/* Transition-state (Eyring) rate of Eq. 7 at temperature T:
 * k = (k_B T / h) exp(dS/R) exp(-dH/(R T)), R = k_B N_A. Pinned: closed-form
 * survival exp(-k t) at constant T_eff; Arrhenius slope d ln(k/T)/d(1/T). */
double orc_eyring_rate(const orc_ion *ion, double T)
{
    if (!(ion->dH_kJmol > 0.0) || !(T > 0.0)) return 0.0;
    double R = ORC_KB * ORC_NA;
    return ORC_KB * T / ORC_PLANCK * exp(ion->dS_JmolK / R) * exp(-ion->dH_kJmol * 1000.0 / (R * T));
}

/* ------------------------------------------------------------------------- */
/* E from a potential by central differences (field bake; the paper takes E  */
/* from the baked potentials): E = -grad(phi), interior central,              */
/* one-sided at the domain edges, E_r = 0 on the axis.                        */
/* ------------------------------------------------------------------------- */
void orc_efield_from_phi(int nr, int nz, double dr, double dz, const double *phi, double *er,
                         double *ez)
{
    for (int j = 0; j < nz; ++j) {
        for (int i = 0; i < nr; ++i) {
            const double *row = phi + (size_t)j * nr;
            double dpr;
            if (i == 0) dpr = 0.0;
            else if (i == nr - 1) dpr = (row[i] - row[i - 1]) / dr;
            else dpr = (row[i + 1] - row[i - 1]) / (2.0 * dr);
            double dpz;
            if (j == 0) dpz = (phi[(size_t)(j + 1) * nr + i] - phi[(size_t)j * nr + i]) / dz;
            else if (j == nz - 1) dpz = (phi[(size_t)j * nr + i] - phi[(size_t)(j - 1) * nr + i]) / dz;
            else dpz = (phi[(size_t)(j + 1) * nr + i] - phi[(size_t)(j - 1) * nr + i]) / (2.0 * dz);
            er[(size_t)j * nr + i] = -dpr;
            ez[(size_t)j * nr + i] = -dpz;
        }
    }
}

/* Bilinear interpolation of a node array at fractional grid coordinates. */
static double bilin(const double *a, int nr, int i0, int j0, double fr, double fz)
{
    const double *p = a + (size_t)j0 * nr + i0;
    return (1.0 - fr) * (1.0 - fz) * p[0] + fr * (1.0 - fz) * p[1] + (1.0 - fr) * fz * p[nr] +
           fr * fz * p[nr + 1];
}

static void cell_of(double g, int n, int *i0, double *f)
{
    double fl = floor(g);
    int i = (int)fl;
    if (i < 0) { *i0 = 0; *f = 0.0; return; }
    if (i > n - 2) { *i0 = n - 2; *f = 1.0; return; }
    *i0 = i;
    *f = g - fl;
}

/* Local gathered quantities at an ion position (Eq. 3, Eq. 4, gas coupling). */
typedef struct {
    double Edc[3], Erf[3], Esc[3];
    double n, T, u[3];
} orc_local;

static void gather(const orc_fields *F, const orc_run *run, double x, double y, double z,
                   orc_local *L)
{
    double r = sqrt(x * x + y * y);
    double dr = F->R / (F->nr - 1), dz = (F->z1 - F->z0) / (F->nz - 1);
    int i0, j0;
    double fr, fz;
    cell_of(r / dr, F->nr, &i0, &fr);
    cell_of((z - F->z0) / dz, F->nz, &j0, &fz);
    double cx = r > 0.0 ? x / r : 0.0, cy = r > 0.0 ? y / r : 0.0; /* Eq. 3, 0 on axis */
    double er = bilin(F->er_dc, F->nr, i0, j0, fr, fz), ez = bilin(F->ez_dc, F->nr, i0, j0, fr, fz);
    L->Edc[0] = er * cx; L->Edc[1] = er * cy; L->Edc[2] = ez;
    er = bilin(F->er_rf, F->nr, i0, j0, fr, fz); ez = bilin(F->ez_rf, F->nr, i0, j0, fr, fz);
    L->Erf[0] = er * cx; L->Erf[1] = er * cy; L->Erf[2] = ez;
    double p = bilin(F->gas_p, F->nr, i0, j0, fr, fz) * run->p_scale;
    double T = bilin(F->gas_T, F->nr, i0, j0, fr, fz);
    double ur = bilin(F->gas_ur, F->nr, i0, j0, fr, fz), uz = bilin(F->gas_uz, F->nr, i0, j0, fr, fz);
    L->T = T;
    L->n = T > 0.0 ? p / (ORC_KB * T) : 0.0;
    L->u[0] = ur * cx; L->u[1] = ur * cy; L->u[2] = uz;
    L->Esc[0] = L->Esc[1] = L->Esc[2] = 0.0;
    if (F->er_sc) {
        double pdr = F->R / (F->pnr - 1), pdz = (F->z1 - F->z0) / (F->pnz - 1);
        cell_of(r / pdr, F->pnr, &i0, &fr);
        cell_of((z - F->z0) / pdz, F->pnz, &j0, &fz);
        er = bilin(F->er_sc, F->pnr, i0, j0, fr, fz);
        ez = bilin(F->ez_sc, F->pnr, i0, j0, fr, fz);
        L->Esc[0] = er * cx; L->Esc[1] = er * cy; L->Esc[2] = ez;
    }
}

/* Acceleration (q/m) E_tot at a position for a given RF scalar (Eq. 3, Eq. 4). */
static void field_accel(const orc_fields *F, const orc_run *run, double qm, const double p[3], double srf,
                        double a[3])
{
    orc_local L;
    gather(F, run, p[0], p[1], p[2], &L);
    for (int d = 0; d < 3; ++d) a[d] = qm * (run->dc_scale * L.Edc[d] + srf * L.Erf[d] + L.Esc[d]);
}

/* RF scalar V/Vref * cos(2 pi f t_n + phi) with t_n = n dt; the phase is the
 * fractional part of n*dt*f taken in FP64 (Eq. 4, Vref = 1 V). */
double orc_rf_scalar(const orc_run *run, int64_t n)
{
    if (run->v_rf == 0.0 || run->f_rf == 0.0) return 0.0;
    double x = run->rf_phase0 + (double)(n - run->seg_step0) * (run->dt * run->f_rf);
    double frac = x - floor(x);
    return run->v_rf * cos(2.0 * ORC_PI * frac + run->phi_rf);
}

/* RF scalar half a step after step n (RK4 midpoint evaluations). */
double orc_rf_scalar_half(const orc_run *run, int64_t n)
{
    if (run->v_rf == 0.0 || run->f_rf == 0.0) return 0.0;
    double x = run->rf_phase0 + ((double)(n - run->seg_step0) + 0.5) * (run->dt * run->f_rf);
    double frac = x - floor(x);
    return run->v_rf * cos(2.0 * ORC_PI * frac + run->phi_rf);
}

/* ------------------------------------------------------------------------- */
/* Collisions within one step (Eq. 6 and the IICT paragraph).                 */
/*                                                                           */
/* The partner velocity c = u + c' is drawn from the local Maxwellian about    */
/* the flow u. With w = |v - u| and s = sqrt(2kT/m_g), |v - c| <= w + |c'|,   */
/* so candidates are generated at the majorant rate n*sigma*(w + 2s/sqrt(pi)) */
/* with c' drawn from f(c')(w + |c'|) / (w + 2s/sqrt(pi)) (a mixture of the   */
/* Maxwellian and its speed-weighted form) and accepted with probability     */
/* |v - c| / (w + |c'|). Accepted events occur at rate n*sigma*<|v - c|>.     */
/* Candidates form a Poisson process of rate nu = n sigma (w + 2s/sqrt(pi))   */
/* (recomputed after every accepted event and at every step): each pack      */
/* carries the optical depth tau (an Exp(1) variate) left until its next     */
/* candidate; a step of length dt consumes nu (dt - t); when tau runs out     */
/* inside the step a candidate is processed and a fresh tau is drawn.         */
/*                                                                           */
/* Accepted event: isotropic scattering in the centre-of-mass frame, momentum */
/* conserved, internal exchange by the Borgnakke-Larsen rule: the collision  */
/* energy E_c = mu g^2/2 + E_int is split with E_int' = B E_c,               */
/* B ~ Beta(Cv(T_eff)/k_B, 2), sampled as U1^(1/a) U2^(1/(a+1)); 1-B is       */
/* formed with expm1 so that small exchanges keep their precision.           */
/* Uniforms of candidate k of a step: 12 fields of Philox blocks 2k and 2k+1 */
/* (see draw_candidate).                                                     */
/* Pins: collision rate vs n*sigma*gbar(w); equilibrium T_eff -> T_gas;      */
/* Beta moments. IICT itself: parity unpinned.                               */
/* ------------------------------------------------------------------------- */

/* 12 uniforms of one candidate from Philox blocks 2k and 2k+1 of the step
 * (purpose 0): fields 0..7 are ((w_j >> 11) + 1/2) 2^-21 of the eight words,
 * fields 8..11 join the low 11 bits of word pairs (2m, 2m+1) into 22-bit
 * uniforms ((v + 1/2) 2^-22). Exact in FP32 and FP64. */
static void draw_candidate(uint64_t seed, uint32_t pack, uint32_t step, uint32_t k, double f[12])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t c0[4] = {pack, step, 2u * k, 0u}, c1[4] = {pack, step, 2u * k + 1u, 0u};
    uint32_t w[8];
    orc_philox4x32_10(c0, key, w);
    orc_philox4x32_10(c1, key, w + 4);
    for (int j = 0; j < 8; ++j) f[j] = ((double)(w[j] >> 11) + 0.5) * (1.0 / 2097152.0);
    for (int m = 0; m < 4; ++m) {
        uint32_t v = ((w[2 * m] & 0x7FFu) << 11) | (w[2 * m + 1] & 0x7FFu);
        f[8 + m] = ((double)v + 0.5) * (1.0 / 4194304.0);
    }
}

static int collide(const orc_ion *ion, const orc_run *run, const orc_local *L, uint64_t seed,
                   uint32_t pack, uint32_t step, double v[3], double *eint, double *tau, int frozen,
                   int *overflow)
{
    *overflow = 0;
    double sigma = ion->ccs_m2;
    if (!(L->n > 0.0) || !(sigma > 0.0) || !(L->T > 0.0)) return 0;
    double M = ion->mass_da * ORC_DALTON, mg = run->m_gas_da * ORC_DALTON;
    double mu = M * mg / (M + mg);
    double s = sqrt(2.0 * ORC_KB * L->T / mg);
    double cbar = 2.0 * s / sqrt(ORC_PI);
    double t = 0.0;
    int accepted = 0;
    for (int k = 0; k < ORC_KMAX; ++k) {
        double w3[3] = {v[0] - L->u[0], v[1] - L->u[1], v[2] - L->u[2]};
        double w = sqrt(w3[0] * w3[0] + w3[1] * w3[1] + w3[2] * w3[2]);
        double nu = L->n * sigma * (w + cbar);
        double room = nu * (run->dt - t);
        if (*tau >= room) {
            *tau -= room;
            return accepted;
        }
        t += *tau / nu;
        double f[12];
        draw_candidate(seed, pack, step, (uint32_t)k, f);
        *tau = -log(f[11]);
        /* Both partner laws are isotropic with |c'|^2/s^2 ~ Gamma(k, 1):
         * k = 3/2 for the Maxwellian (components of variance s^2/2), k = 2 for
         * its speed-weighted form. Gamma(2) = Exp(1) + Exp(1); Gamma(3/2) =
         * Exp(1) + N^2/2 with N = sqrt(-2 ln u) cos(2 pi u'), so
         * N^2/2 = -ln(u) cos^2(2 pi u'). */
        double fk = 1.0;
        if (f[0] * (w + cbar) < w) {
            double cw = cos(2.0 * ORC_PI * f[2]);
            fk = cw * cw;
        }
        double y = -log(f[3]) - log(f[4]) * fk;
        double cmag = s * sqrt(y), cp[3];
        double pct = 2.0 * f[5] - 1.0, pst = sqrt(fmax(0.0, 1.0 - pct * pct));
        double pph = 2.0 * ORC_PI * f[6];
        cp[0] = cmag * pst * cos(pph);
        cp[1] = cmag * pst * sin(pph);
        cp[2] = cmag * pct;
        double g3[3] = {w3[0] - cp[0], w3[1] - cp[1], w3[2] - cp[2]};
        double g = sqrt(g3[0] * g3[0] + g3[1] * g3[1] + g3[2] * g3[2]);
        if (!(f[1] * (w + cmag) < g)) continue;
        ++accepted;
        if (frozen) continue;
        double Vcm[3];
        for (int d = 0; d < 3; ++d) Vcm[d] = (M * v[d] + mg * (L->u[d] + cp[d])) / (M + mg);
        double etr = 0.5 * mu * g * g / ORC_KB; /* [K] */
        double ec = etr + *eint;
        double Teff = orc_T_of_eint(ion, *eint);
        double acv = orc_cv_of_T(ion, Teff);
        double one_minus_B = -expm1(log(f[9]) / acv + log(f[10]) / (acv + 1.0));
        double etr_new = ec * one_minus_B;
        *eint = *eint + (etr - etr_new);
        double gnew = sqrt(2.0 * etr_new * ORC_KB / mu);
        double ct = 2.0 * f[7] - 1.0, st = sqrt(fmax(0.0, 1.0 - ct * ct));
        double ph = 2.0 * ORC_PI * f[8];
        double nhat[3] = {st * cos(ph), st * sin(ph), ct};
        for (int d = 0; d < 3; ++d) v[d] = Vcm[d] + (mg / (M + mg)) * gnew * nhat[d];
    }
    *overflow = 1;
    return accepted;
}

/* Expected collision rate n sigma <|v - c|> of Eq. 6 with c drawn from the
 * local Maxwellian about the flow: n sigma s [(x + 1/(2x)) erf(x) +
 * exp(-x^2)/sqrt(pi)], x = |v - u|/s, s = sqrt(2kT/m_g) (-> 2s/sqrt(pi) at
 * x = 0). Pinned: frozen-ion rate tests. */
double orc_collision_rate(const orc_ion *ion, const orc_run *run, const orc_local *L, const double v[3])
{
    if (!(L->n > 0.0) || !(ion->ccs_m2 > 0.0) || !(L->T > 0.0)) return 0.0;
    double mg = run->m_gas_da * ORC_DALTON;
    double s = sqrt(2.0 * ORC_KB * L->T / mg);
    double w = sqrt((v[0] - L->u[0]) * (v[0] - L->u[0]) + (v[1] - L->u[1]) * (v[1] - L->u[1]) +
                    (v[2] - L->u[2]) * (v[2] - L->u[2]));
    double x = w / s;
    double gbar = x > 1e-6 ? s * ((x + 0.5 / x) * erf(x) + exp(-x * x) / sqrt(ORC_PI))
                           : 2.0 * s / sqrt(ORC_PI);
    return L->n * ion->ccs_m2 * gbar;
}

/* Hybrid Langevin branch (Methods, Particle transport, collisions, and
 * effective internal temperature: an optional mode that relaxes the velocity
 * toward the gas flow in one lumped step, with a random part set by the gas
 * temperature): exact Ornstein-Uhlenbeck update of the
 * velocity relative to the flow over dt,
 *   v <- u + (v - u) e^{-gamma dt} + sqrt(kT/M (1 - e^{-2 gamma dt})) xi,
 * with the friction gamma = q / (M K) from the low-field Mason-Schamp
 * mobility K = (3q / 16N) sqrt(2 pi / (mu k T)) / sigma. Normals from draw
 * block 128 of the step (Box-Muller). T_eff is not updated. Pinned:
 * stationary Maxwellian, drift K E, explicit-vs-hybrid transmission. */
static void langevin_step(const orc_ion *ion, const orc_run *run, const orc_local *L, uint64_t seed,
                          uint32_t pack, uint32_t step, double v[3])
{
    double M = ion->mass_da * ORC_DALTON, mg = run->m_gas_da * ORC_DALTON;
    double mu = M * mg / (M + mg);
    double q = fabs((double)ion->charge) * ORC_E_CHARGE;
    double K = 3.0 * q / (16.0 * L->n) * sqrt(2.0 * ORC_PI / (mu * ORC_KB * L->T)) / ion->ccs_m2;
    double gamma = q / (M * K);
    double decay = exp(-gamma * run->dt);
    double sd = sqrt(ORC_KB * L->T / M * -expm1(-2.0 * gamma * run->dt));
    double u[4];
    draw4(seed, pack, step, 128u, 0u, u);
    double r01 = sqrt(-2.0 * log(u[0])), r23 = sqrt(-2.0 * log(u[2]));
    double xi[3] = {r01 * cos(2.0 * ORC_PI * u[1]), r01 * sin(2.0 * ORC_PI * u[1]),
                    r23 * cos(2.0 * ORC_PI * u[3])};
    for (int d = 0; d < 3; ++d) v[d] = L->u[d] + (v[d] - L->u[d]) * decay + sd * xi[d];
}

/* Fixed-point lattice used for every discrete decision (classification, mask
 * lookup, deposit, tally bins): x = xq*R*2^-30, y likewise,
 * z = z0 + zq*(z1-z0)*2^-30. FP64 positions are quantised by rint(x*2^30/R). */
static int64_t clamp32(double v)
{
    if (v < -2147483648.0) return -2147483648LL;
    if (v > 2147483647.0) return 2147483647LL;
    return (int64_t)v;
}

void orc_quantize(double R, double z0, double z1, double x, double y, double z, int32_t *xq,
                  int32_t *yq, int32_t *zq)
{
    double sx = 1073741824.0 / R, sz = 1073741824.0 / (z1 - z0);
    *xq = (int32_t)clamp32(rint(x * sx));
    *yq = (int32_t)clamp32(rint(y * sx));
    *zq = (int32_t)clamp32(rint((z - z0) * sz));
}

/* Thresholds of the classification on the lattice. */
typedef struct {
    int64_t zexit_q, rdet_q;
    float hit;
} orc_thr;

static orc_thr thresholds(const orc_fields *F, const orc_run *run)
{
    orc_thr t;
    t.zexit_q = (int64_t)ceil((run->z_exit - F->z0) / (F->z1 - F->z0) * 1073741824.0);
    t.rdet_q = (int64_t)floor(run->r_det / F->R * 1073741824.0);
    t.hit = (float)run->hit_dist;
    return t;
}

/* Terminal classification of one lattice position ("Terminal events"):
 * electrode hit (nearest mask node is metal or within the hit distance) ->
 * radial loss (r >= R) -> plane z >= z_exit crossed (transmitted when
 * r <= r_det, else axial exit) -> z < z0 (axial exit). The nearest node's r
 * index is taken in FP32 from the lattice integers. Pinned: brute-force
 * geometric checks in the tests. */
static int classify_q(const orc_fields *F, const orc_thr *t, int32_t xq, int32_t yq, int32_t zq)
{
    float fx = (float)xq, fy = (float)yq;
    float sr = (float)(F->nr - 1) * (1.0f / 1073741824.0f);
    float rr = sqrtf(fx * fx + fy * fy);
    int ir = (int)(rr * sr + 0.5f);
    if (ir > F->nr - 1) ir = F->nr - 1;
    int64_t zt = (int64_t)zq * (int64_t)(F->nz - 1) + (1LL << 29);
    int64_t iz = zt >> 30;
    if (iz < 0) iz = 0;
    if (iz > F->nz - 1) iz = F->nz - 1;
    float d = F->dmask[(size_t)iz * F->nr + ir];
    if (d <= t->hit) return ORC_ELECTRODE;
    uint64_t r2 = (uint64_t)((int64_t)xq * xq) + (uint64_t)((int64_t)yq * yq);
    if (r2 >= (1ULL << 60)) return ORC_RADIAL;
    if ((int64_t)zq >= t->zexit_q) {
        uint64_t rd2 = (uint64_t)(t->rdet_q * t->rdet_q);
        return r2 <= rd2 ? ORC_TRANSMITTED : ORC_AXIAL;
    }
    if (zq < 0) return ORC_AXIAL;
    return ORC_ACTIVE;
}

void orc_classify_fixed(const orc_fields *F, const orc_run *run, int64_t n, const int32_t *xq,
                        const int32_t *yq, const int32_t *zq, uint8_t *status)
{
    orc_thr t = thresholds(F, run);
    for (int64_t p = 0; p < n; ++p) status[p] = (uint8_t)classify_q(F, &t, xq[p], yq[p], zq[p]);
}

/* ------------------------------------------------------------------------- */
/* Time stepping: for steps n = step0 .. step0+nsteps-1 and every active pack:*/
/*   gather at x_n -> collisions -> kick v += (q/m) E_tot(x_n, t_n) dt ->     */
/*   drift x += v dt -> classify at x_{n+1} (operator order of the Methods).  */
/* Pins: uniform-field parabola, energy conservation, Dehmelt secular         */
/* frequency, Mason-Schamp mobility, collision rate, T_int relaxation.        */
/* ------------------------------------------------------------------------- */
void orc_run_steps(const orc_fields *F, const orc_ion *ion, const orc_run *run, orc_state *S,
                   int64_t n_packs, int64_t step0, int64_t nsteps, int frozen_collisions)
{
    orc_thr thr = thresholds(F, run);
    double qm = ion->charge * ORC_E_CHARGE / (ion->mass_da * ORC_DALTON);
    double *srf = (double *)malloc(sizeof(double) * (size_t)(nsteps > 0 ? nsteps : 1));
    for (int64_t k = 0; k < nsteps; ++k) srf[k] = orc_rf_scalar(run, step0 + k);
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < n_packs; ++p) {
        if (S->status[p] != ORC_ACTIVE) continue;
        double x = S->x[p], y = S->y[p], z = S->z[p];
        double v[3] = {S->vx[p], S->vy[p], S->vz[p]};
        double eint = S->eint[p];
        double lnsy = S->lnsy ? S->lnsy[p] : 0.0;
        double tau = S->tau[p];
        for (int64_t k = 0; k < nsteps; ++k) {
            int64_t n = step0 + k;
            orc_local L;
            gather(F, run, x, y, z, &L);
            int ovf = 0, nc = 0;
            int lv = run->langevin && z >= run->lv_z0 && z <= run->lv_z1 &&
                     orc_collision_rate(ion, run, &L, v) * run->dt >= run->lv_switch;
            if (lv)
                langevin_step(ion, run, &L, run->seed, (uint32_t)p, (uint32_t)n, v);
            else
                nc = collide(ion, run, &L, run->seed, (uint32_t)p, (uint32_t)n, v, &eint, &tau,
                             frozen_collisions, &ovf);
            if (S->ncoll) S->ncoll[p] += nc;
            if (S->noverflow) S->noverflow[p] += ovf;
            if (S->nsteps) S->nsteps[p] += 1;
            /* Eq. 7: the survival yield decays at the rate of the current T_eff
             * (not updated during an aggregated Langevin step) */
            if (ion->dH_kJmol > 0.0 && !lv)
                lnsy -= orc_eyring_rate(ion, orc_T_of_eint(ion, eint)) * run->dt;
            if (run->integrator == 1) {
                /* RK4 under the instantaneous total field (Methods, "Simulation scope and
                 * modular architecture" and "Particle transport, collisions, and
                 * effective internal temperature"): four field
                 * evaluations at t_n, t_n + dt/2 (twice) and t_n + dt */
                double h = run->dt, sh = orc_rf_scalar_half(run, n), s1 = orc_rf_scalar(run, n + 1);
                double p[3] = {x, y, z}, a1[3], a2[3], a3[3], a4[3], v2[3], v3[3], v4[3], q[3];
                field_accel(F, run, qm, p, srf[k], a1);
                for (int d = 0; d < 3; ++d) { q[d] = p[d] + 0.5 * h * v[d]; v2[d] = v[d] + 0.5 * h * a1[d]; }
                field_accel(F, run, qm, q, sh, a2);
                for (int d = 0; d < 3; ++d) { q[d] = p[d] + 0.5 * h * v2[d]; v3[d] = v[d] + 0.5 * h * a2[d]; }
                field_accel(F, run, qm, q, sh, a3);
                for (int d = 0; d < 3; ++d) { q[d] = p[d] + h * v3[d]; v4[d] = v[d] + h * a3[d]; }
                field_accel(F, run, qm, q, s1, a4);
                for (int d = 0; d < 3; ++d) {
                    p[d] += h / 6.0 * (v[d] + 2.0 * v2[d] + 2.0 * v3[d] + v4[d]);
                    v[d] += h / 6.0 * (a1[d] + 2.0 * a2[d] + 2.0 * a3[d] + a4[d]);
                }
                x = p[0]; y = p[1]; z = p[2];
            } else {
                for (int d = 0; d < 3; ++d)
                    v[d] += qm * (run->dc_scale * L.Edc[d] + srf[k] * L.Erf[d] + L.Esc[d]) * run->dt;
                x += v[0] * run->dt;
                y += v[1] * run->dt;
                z += v[2] * run->dt;
            }
            int32_t xq, yq, zq;
            orc_quantize(F->R, F->z0, F->z1, x, y, z, &xq, &yq, &zq);
            int st = classify_q(F, &thr, xq, yq, zq);
            if (st != ORC_ACTIVE) {
                S->status[p] = (uint8_t)st;
                S->t_term[p] = (int32_t)(n + 1);
                break;
            }
        }
        S->x[p] = x; S->y[p] = y; S->z[p] = z;
        S->vx[p] = v[0]; S->vy[p] = v[1]; S->vz[p] = v[2];
        S->eint[p] = eint;
        if (S->lnsy) S->lnsy[p] = lnsy;
        S->tau[p] = tau;
    }
    free(srf);
}

/* Limits of the global micro step of Eq. 1 on the current state:
 * out[0] = 0.05 t_RF, out[1] = 0.1 tau_coll (1 / largest expected collision
 * rate), out[2] = dt_acc = 0.1 min_p max(|v|, v_th) / |a| (velocity change
 * per step at most 10 % of the speed scale; v_th = sqrt(kT/M) of the local
 * gas), out[3] = dt_CFL = 0.5 min(dr, dz) / max|v| (displacement at most half
 * a grid spacing), out[4] = dt_L = 2 ns with the hybrid branch on (Table S2),
 * out[5] = the smallest of them; absent limits are +inf. dt_rem, the time to
 * the next scheduled boundary, is the caller's. */
void orc_dt_limits(const orc_fields *F, const orc_ion *ion, const orc_run *run, const orc_state *S,
                   int64_t n_packs, int64_t step, double out[6])
{
    double qm = ion->charge * ORC_E_CHARGE / (ion->mass_da * ORC_DALTON);
    double M = ion->mass_da * ORC_DALTON;
    double srf = orc_rf_scalar(run, step);
    double lam = 0.0, vmax = 0.0, acc = INFINITY;
    for (int64_t p = 0; p < n_packs; ++p) {
        if (S->status[p] != ORC_ACTIVE) continue;
        double v[3] = {S->vx[p], S->vy[p], S->vz[p]};
        orc_local L;
        gather(F, run, S->x[p], S->y[p], S->z[p], &L);
        double r = orc_collision_rate(ion, run, &L, v);
        if (r > lam) lam = r;
        double vm = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        if (vm > vmax) vmax = vm;
        double a[3];
        for (int d = 0; d < 3; ++d) a[d] = qm * (run->dc_scale * L.Edc[d] + srf * L.Erf[d] + L.Esc[d]);
        double am = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
        double vth = L.T > 0.0 ? sqrt(ORC_KB * L.T / M) : 0.0;
        double vs = vm > vth ? vm : vth;
        if (am > 0.0 && 0.1 * vs / am < acc) acc = 0.1 * vs / am;
    }
    double dr = F->R / (F->nr - 1), dz = (F->z1 - F->z0) / (F->nz - 1);
    out[0] = run->f_rf > 0.0 && run->v_rf != 0.0 ? 0.05 / run->f_rf : INFINITY;
    out[1] = lam > 0.0 ? 0.1 / lam : INFINITY;
    out[2] = acc;
    out[3] = vmax > 0.0 ? 0.5 * (dr < dz ? dr : dz) / vmax : INFINITY;
    out[4] = run->langevin ? 2e-9 : INFINITY;
    double m = out[0];
    for (int i = 1; i < 5; ++i) if (out[i] < m) m = out[i];
    out[5] = m;
}

/* Count accepted collisions in one step of length dt at a fixed ion velocity
 * (the velocity is not updated): used to pin the sampled rate against
 * n*sigma*gbar(w). */
int64_t orc_count_collisions_frozen(const orc_ion *ion, const orc_run *run, double n, double T,
                                    const double u[3], const double v[3], int64_t trials)
{
    orc_local L;
    memset(&L, 0, sizeof L);
    L.n = n; L.T = T;
    L.u[0] = u[0]; L.u[1] = u[1]; L.u[2] = u[2];
    int64_t total = 0;
#pragma omp parallel for reduction(+ : total) schedule(static)
    for (int64_t t = 0; t < trials; ++t) {
        double vv[3] = {v[0], v[1], v[2]};
        double e = 0.0, c[4];
        draw4(run->seed, (uint32_t)t, 0u, 2u, 1u, c);
        double tau = -log(c[0]);
        int ovf;
        total += collide(ion, run, &L, run->seed, (uint32_t)t, (uint32_t)(t >> 32), vv, &e, &tau, 1, &ovf);
    }
    return total;
}

/* Borgnakke-Larsen partition sampler alone: returns 1-B for B ~ Beta(a, 2). */
double orc_one_minus_beta(double a, double u2, double u3)
{
    return -expm1(log(u2) / a + log(u3) / (a + 1.0));
}

/* ------------------------------------------------------------------------- */
/* Source ("Continuous current Gaussian source"): positions uniform over a    */
/* disc (r = a sqrt(u)) or a Gaussian truncated at the hard radius (inverse   */
/* CDF of the truncated Rayleigh law), on the source plane or, for a prefill, */
/* uniform in z; velocity Maxwellian at T_vel, v_z folded to >= 0 when asked; */
/* E_int = E_int(T_init). Purpose 1 of the Philox counter.                   */
/* ------------------------------------------------------------------------- */
void orc_inject(const orc_ion *ion, const orc_source *src, const orc_run *run, orc_state *S,
                int64_t p0, int64_t count)
{
    double M = ion->mass_da * ORC_DALTON;
    double sd = sqrt(ORC_KB * src->T_vel / M);
    double e0 = orc_eint_of_T(ion, ion->T_init);
    for (int64_t p = p0; p < p0 + count; ++p) {
        double a[4], b[4];
        draw4(run->seed, (uint32_t)p, 0u, 0u, 1u, a);
        draw4(run->seed, (uint32_t)p, 0u, 1u, 1u, b);
        double r;
        if (src->profile == 0) {
            r = src->radius * sqrt(a[0]);
        } else {
            double tail = expm1(-src->radius * src->radius / (2.0 * src->sigma * src->sigma));
            r = src->sigma * sqrt(-2.0 * log1p(a[0] * tail));
        }
        double th = 2.0 * ORC_PI * a[1];
        S->x[p] = r * cos(th);
        S->y[p] = r * sin(th);
        if (src->prefill_z1 > src->prefill_z0)
            S->z[p] = src->prefill_z0 + (src->prefill_z1 - src->prefill_z0) * a[2];
        else
            S->z[p] = src->z_plane;
        double r01 = sqrt(-2.0 * log(b[0])), r23 = sqrt(-2.0 * log(b[2]));
        S->vx[p] = sd * r01 * cos(2.0 * ORC_PI * b[1]);
        S->vy[p] = sd * r01 * sin(2.0 * ORC_PI * b[1]);
        double vz = sd * r23 * cos(2.0 * ORC_PI * b[3]);
        S->vz[p] = src->half_space ? fabs(vz) : vz;
        S->eint[p] = e0;
        S->status[p] = ORC_ACTIVE;
        S->t_term[p] = -1;
        if (S->lnsy) S->lnsy[p] = 0.0;
        double c[4];
        draw4(run->seed, (uint32_t)p, 0u, 2u, 1u, c);
        S->tau[p] = -log(c[0]); /* Exp(1) optical depth to the first candidate */
    }
}

/* Source accumulator of Eq. 5: the number of packs released after `nsteps`
 * steps of the source at current I, starting from accumulated real ions acc
 * (updated in place). */
int64_t orc_source_emit(double current_A, double charge, double dt, int64_t weight, int64_t nsteps,
                        double *acc)
{
    double per_step = current_A * dt / (charge * ORC_E_CHARGE);
    int64_t emitted = 0;
    for (int64_t k = 0; k < nsteps; ++k) {
        *acc += per_step;
        while (*acc >= (double)weight) {
            *acc -= (double)weight;
            ++emitted;
        }
    }
    return emitted;
}

/* ------------------------------------------------------------------------- */
/* CIC deposit on the axisymmetric PIC grid, defined on the lattice          */
/* ("Axisymmetric PIC space charge update"): r = floor(sqrt(xq^2+yq^2))       */
/* exactly; cell and 15-bit fractions from integer products; node charge    */
/* Q += (q*W) * w_r * w_z in units of e * 2^-30. Pinned: total charge exact, */
/* brute-force weights on tiny inputs, Green's-function potential.           */
/* ------------------------------------------------------------------------- */
static uint64_t isqrt64(uint64_t v)
{
    uint64_t r = (uint64_t)sqrt((double)v);
    while (r * r > v) --r;
    while ((r + 1) * (r + 1) <= v) ++r;
    return r;
}

void orc_deposit_fixed(int pnr, int pnz, int64_t n, const int32_t *xq, const int32_t *yq,
                       const int32_t *zq, const uint8_t *status, int64_t qw, int64_t *Q)
{
    for (int64_t p = 0; p < n; ++p) {
        if (status[p] != ORC_ACTIVE) continue;
        uint64_t r2 = (uint64_t)((int64_t)xq[p] * xq[p]) + (uint64_t)((int64_t)yq[p] * yq[p]);
        uint64_t r = isqrt64(r2);
        if (r >= (1ULL << 30) || zq[p] < 0 || zq[p] > (1 << 30)) continue;
        uint64_t tr = r * (uint64_t)(pnr - 1);
        uint64_t tz = (uint64_t)zq[p] * (uint64_t)(pnz - 1);
        int64_t i = (int64_t)(tr >> 30), j = (int64_t)(tz >> 30);
        int64_t fr = (int64_t)((tr & ((1ULL << 30) - 1)) >> 15);
        int64_t fz = (int64_t)((tz & ((1ULL << 30) - 1)) >> 15);
        if (i > pnr - 2) { i = pnr - 2; fr = 1 << 15; }
        if (j > pnz - 2) { j = pnz - 2; fz = 1 << 15; }
        int64_t wr0 = (1 << 15) - fr, wr1 = fr, wz0 = (1 << 15) - fz, wz1 = fz;
        Q[(size_t)j * pnr + i] += qw * wr0 * wz0;
        Q[(size_t)j * pnr + i + 1] += qw * wr1 * wz0;
        Q[(size_t)(j + 1) * pnr + i] += qw * wr0 * wz1;
        Q[(size_t)(j + 1) * pnr + i + 1] += qw * wr1 * wz1;
    }
}

/* ------------------------------------------------------------------------- */
/* Observables ("Terminal events, snapshots, and reported observables",      */
/* Eq. 8, conservation of represented weight): a pure function of the state. */
/* FP64 quantities that decide a bin are formed in a fixed operation order    */
/* without fused multiply-add. Pinned: conservation, brute-force recounts.   */
/* ------------------------------------------------------------------------- */
typedef struct {
    int64_t count[8], weight[8];
    double sum_w_ke[8], sum_w_teff[8], sum_w_sy[8];
    int64_t *exit_hist;  /* [n_exit_bins] weight of transmitted packs by exit step */
    int64_t *r_hist;     /* [n_r_bins] transmitted weight by exit radius (r <= r_det) */
    int64_t *ke_hist;    /* [n_ke_bins] transmitted weight by kinetic energy */
    int64_t *teff_hist;  /* [n_teff_bins] transmitted weight by T_eff */
    int64_t *loss_map;   /* [n_loss_z][n_loss_r] electrode-hit weight */
} orc_tally;

typedef struct {
    int exit_bin_steps, n_exit_bins, n_r_bins, n_ke_bins, n_teff_bins, n_loss_r, n_loss_z;
    double ke_max_ev, teff_max;
} orc_tally_spec;

static int64_t clampi(int64_t v, int64_t lo, int64_t hi) { return v < lo ? lo : (v > hi ? hi : v); }

void orc_tally_state(const orc_fields *F, const orc_ion *ion, const orc_run *run,
                     const orc_tally_spec *ts, int64_t n, const int32_t *xq, const int32_t *yq,
                     const int32_t *zq, const double *vx, const double *vy, const double *vz,
                     const double *eint, const double *lnsy, const uint8_t *status,
                     const int32_t *t_term, int64_t weight, orc_tally *T)
{
    double M = ion->mass_da * ORC_DALTON;
    double c_ke = 0.5 * M / ORC_E_CHARGE;
    double ke_scale = (double)ts->n_ke_bins / ts->ke_max_ev;
    double t_scale = (double)ts->n_teff_bins / ts->teff_max;
    float r_scale = (float)((double)ts->n_r_bins / (run->r_det / F->R) / 1073741824.0);
    float lr_scale = (float)((double)ts->n_loss_r / 1073741824.0);
    for (int64_t p = 0; p < n; ++p) {
        int st = status[p];
        if (st == ORC_EMPTY || st > 7) continue;
        T->count[st] += 1;
        T->weight[st] += weight;
        double v2 = vx[p] * vx[p];
        v2 = v2 + vy[p] * vy[p];
        v2 = v2 + vz[p] * vz[p];
        double ke = v2 * c_ke;
        double te = orc_T_of_eint(ion, eint[p]);
        T->sum_w_ke[st] += (double)weight * ke;
        T->sum_w_teff[st] += (double)weight * te;
        T->sum_w_sy[st] += (double)weight * (lnsy ? exp(lnsy[p]) : 1.0);
        float fx = (float)xq[p], fy = (float)yq[p];
        float rr = sqrtf(fx * fx + fy * fy);
        if (st == ORC_TRANSMITTED) {
            int64_t b = clampi((int64_t)t_term[p] / ts->exit_bin_steps, 0, ts->n_exit_bins - 1);
            T->exit_hist[b] += weight;
            b = clampi((int64_t)(rr * r_scale), 0, ts->n_r_bins - 1);
            T->r_hist[b] += weight;
            b = clampi((int64_t)(ke * ke_scale), 0, ts->n_ke_bins - 1);
            T->ke_hist[b] += weight;
            b = clampi((int64_t)(te * t_scale), 0, ts->n_teff_bins - 1);
            T->teff_hist[b] += weight;
        } else if (st == ORC_ELECTRODE) {
            int64_t br = clampi((int64_t)(rr * lr_scale), 0, ts->n_loss_r - 1);
            int64_t bz = clampi(((int64_t)zq[p] * ts->n_loss_z) >> 30, 0, ts->n_loss_z - 1);
            T->loss_map[bz * ts->n_loss_r + br] += weight;
        }
    }
}

/* Host threads of the OpenMP loops over packs: n > 0 sets the count, n <= 0
 * leaves it; returns the count the next loop uses (1 without OpenMP). */
int orc_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
