/*
 * Plain FP64 CPU oracle of one time step of the hybrid pseudopotential
 * phase-change lattice Boltzmann method with conjugate heat transfer
 * (Zhao, Liang, Sun, Cai, Li, arXiv:1911.10747).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of what the GPU path computes.  Only the tests, the smoke check
 * and the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or helper with the CUDA library; the two are written
 * independently from the paper.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no FMA contraction, so the
 * rounding of every product and sum is the one written here).
 *
 * Every function names the passage it follows.  Readings of passages the
 * paper leaves open are marked "reading:".
 *
 * Pinned, without a GPU, by tests/test_oracle_pins.py and
 * tests/test_oracle_step.py against what the paper and the mathematics fix:
 * the transfer matrix and velocities (Eq. 2, 6, printed), moments of the
 * textbook equilibrium and of Guo's force, the BGK limit, the PR EOS (Tc,
 * critical point, acentric factor, Maxwell densities and latent heat against
 * printed values), psi reproducing p_EOS, the counter-based draws, the
 * Eq. 27-28 stencils, RK4 amplification, steady conduction through the
 * heater, Eq. 36 on quadratics, mass conservation, symmetries, the phase
 * viscosities (shear-wave decay), momentum balance, neutral wall adhesion
 * at the heater and at the lid, the nucleate-spot layout, the open top,
 * the sine and noisy bottoms, advection and the phase-change source of
 * Eq. 24, the vapour fraction, flat-interface coexistence, the Laplace law
 * and the initial state.
 * Parity unpinned: the full coupled step as a whole (no closed form exists);
 * the CUDA path is compared with this file, part by part pinned as above.
 *
 * Layout: populations f[i][y][x] (i = 0..8, y = fluid row 0..nf-1, x =
 * 0..nx-1); temperature T[r][x] for rows r = 0..nt-1, nt = ns + nf, where
 * rows 0..ns-1 are the solid heater (row 0 = heater bottom, Dirichlet) and
 * fluid row y is temperature row ns + y.
 *
 * Model A (Fig. 1a, Sec. 4.1: no solid, the temperature given at the bottom
 * surface of the fluid) is flag F_MODEL_A with ns = 1: row 0 is then not a
 * heater row but the Dirichlet row of the heated wall, holding T_b(x, n).
 * reading: it is coupled to the first fluid row like the top ghost row is
 * to the last one -- the link conducts with the fluid's lambda (the mean of
 * lambda_f with itself), so T_b sits one lattice spacing below the first
 * fluid row, half a spacing below the halfway wall of the flow part.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- D2Q9 lattice, Eq. 2 ------------------------------------------------ */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
/* lattice weights w_a of the equilibrium and of Eq. 27-28 */
static const double WL[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
/* interaction weights of Eq. 11: w(1) = 1/3, w(2) = 1/12 */
static const double WF[9] = {0.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0,
                             1.0 / 12.0, 1.0 / 12.0, 1.0 / 12.0, 1.0 / 12.0};
/* transfer matrix M of Eq. 6 */
static const int MM[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},
    {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},
    {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},
    {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},
    {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1}};
/* squared row norms of M: M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4) */
static const double INVN[9] = {1.0 / 9.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 6.0, 1.0 / 12.0,
                               1.0 / 6.0, 1.0 / 12.0, 1.0 / 4.0, 1.0 / 4.0};

enum { F_PERIODIC_Y = 1, F_ISOTHERMAL = 2, F_FROZEN_FLOW = 4, F_MODEL_A = 8 };
enum { TOP_WALL = 0, TOP_OUTFLOW = 1 };
enum { BC_SPOTS = 0, BC_NOISE = 1, BC_SINE = 2 };
enum { ERR_PSI = 1, ERR_NONFINITE = 2 };

typedef struct {
    int nx, nf, ns, liquid_rows;
    int top_mode, flags, bc_mode, n_spots;
    int spot_x[8];
    int spot_half_width;
    int pad0;
    double c_w_base, c_w_top;
    double c_w_spot[8];
    double a, b, R, omega, G;
    double T_sat_over_Tc, T_b_over_Tc;
    double rho_L, rho_V, rho_mean;
    double g, nu_L, nu_V, c_v, cv_chi;
    double lambda_s, rho_c_s;
    double s[9];
    double varpi, sign_eps;
    double init_noise, bc_noise, sine_amp_over_Tc, sine_wavelength;
    long long sine_t0, sine_t1;
    unsigned long long seed;
} orc_params;

typedef struct {
    orc_params p;
    int nt;
    double Tc, kappa, T_sat, T_b, tau_L, tau_V, rho_bar;
    double *f, *fs, *rho, *ux, *uy, *psi, *T;
    double *cw;            /* per column wettability coefficient of the heater surface */
    double *lam, *Tk, *Ta, *h, *acc; /* FD work arrays over rows 0..nt (ghost row nt) */
    double *uxe, *uye, *rhoe;
    long long step;
    unsigned err;
    double diag[4];        /* q_bottom_mean, q_top_mean, vapour fraction, mass */
    double *q_top;         /* nx */
} orc_run;

/* ---- counter-based uniform draws ----------------------------------------
 * splitmix64 (Steele, Lea, Flood 2014; Vigna's reference constants), folded
 * over (seed, tag, step, index) so that a draw depends only on its counters. */
static uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
double orc_uniform(unsigned long long seed, unsigned long long tag,
                   unsigned long long step, unsigned long long idx)
{
    const uint64_t G = 0x9E3779B97F4A7C15ULL;
    uint64_t h = mix64((uint64_t)seed + G);
    h = mix64((h ^ (uint64_t)tag) + G);
    h = mix64((h ^ (uint64_t)step) + G);
    h = mix64((h ^ (uint64_t)idx) + G);
    return (double)(h >> 11) * (1.0 / 9007199254740992.0);
}
#define TAG_INIT 1ULL
#define TAG_BC 2ULL

/* ---- Peng-Robinson EOS, Eq. 13 ------------------------------------------ */
/* T_c from a = 0.45724 R^2 Tc^2 / Pc and b = 0.0778 R Tc / Pc (Eq. 13 text). */
double orc_Tc(double a, double b, double R) { return (0.0778 * a) / ((0.45724 * b) * R); }
double orc_kappa(double omega) { return 0.37464 + 1.54226 * omega - 0.26992 * omega * omega; }

/* p_EOS(rho, T), Eq. 13 */
double orc_pressure(double rho, double T, double a, double b, double R, double kappa, double Tc)
{
    double t1 = sqrt(T / Tc);
    double t2 = 1.0 + kappa * (1.0 - t1);
    double phi = t2 * t2;
    double br = b * rho;
    double p1 = (rho * R * T) / (1.0 - br);
    double den = 1.0 + 2.0 * br - br * br;
    double p2 = (a * phi * rho * rho) / den;
    return p1 - p2;
}

/* (dp_EOS/dT) at constant rho: the derivative in the phase-change source of
 * Eq. 24 ("dp/dt" there is read as d/dT at constant rho), from Eq. 13. */
double orc_dpdT(double rho, double T, double a, double b, double R, double kappa, double Tc)
{
    double t1 = sqrt(T / Tc);
    double t2 = 1.0 + kappa * (1.0 - t1);
    double br = b * rho;
    double den = 1.0 + 2.0 * br - br * br;
    double d1 = (rho * R) / (1.0 - br);
    double d2 = (a * kappa * rho * rho * t2) / (sqrt(T * Tc) * den);
    return d1 + d2;
}

/* psi = sqrt(2 (p_EOS - rho c_s^2) / (G c^2)), Eq. 12 with c = 1, c_s^2 = 1/3.
 * Sets *bad when the radicand is negative (psi is then returned as 0). */
double orc_psi(double rho, double T, double a, double b, double R, double kappa, double Tc,
               double G, int *bad)
{
    double p = orc_pressure(rho, T, a, b, R, kappa, Tc);
    double arg = (2.0 * (p - rho / 3.0)) / G;
    if (!(arg >= 0.0)) {
        if (bad) *bad = 1;
        return 0.0;
    }
    return sqrt(arg);
}

/* ---- MRT pieces, Eq. 6, 7, 9 -------------------------------------------- */
/* m = M f, Eq. 6 (sum over columns in increasing order) */
void orc_moments(const double *f, double *m)
{
    for (int k = 0; k < 9; k++) {
        double s = 0.0;
        for (int j = 0; j < 9; j++)
            if (MM[k][j] != 0) s += (double)MM[k][j] * f[j];
        m[k] = s;
    }
}

/* f = M^-1 m with M^-1 = M^T diag(1 / |row k|^2) */
void orc_inverse_moments(const double *m, double *f)
{
    double d[9];
    for (int k = 0; k < 9; k++) d[k] = m[k] * INVN[k];
    for (int j = 0; j < 9; j++) {
        double s = 0.0;
        for (int k = 0; k < 9; k++)
            if (MM[k][j] != 0) s += (double)MM[k][j] * d[k];
        f[j] = s;
    }
}

/* m_eq(rho, u), Eq. 6 */
void orc_meq(double rho, double ux, double uy, double *meq)
{
    double usq = ux * ux + uy * uy;
    meq[0] = rho;
    meq[1] = rho * (-2.0 + 3.0 * usq);
    meq[2] = rho * (1.0 - 3.0 * usq);
    meq[3] = rho * ux;
    meq[4] = -(rho * ux);
    meq[5] = rho * uy;
    meq[6] = -(rho * uy);
    meq[7] = rho * (ux * ux - uy * uy);
    meq[8] = rho * (ux * uy);
}

/* Forcing term S-bar in moment space, Eq. 9.
 * reading: the last entry is ux Fy + uy Fx (the printed minus contradicts
 * S-bar = M S of the standard discrete force); the epsilon term of entry 2
 * carries the sign `sign_eps` (-1 in the cited scheme). */
void orc_source(double ux, double uy, double Fx, double Fy, double Fmx, double Fmy, double psi,
                double varpi, double tau_e, double tau_s, double sign_eps, double *S)
{
    double uF = ux * Fx + uy * Fy;
    double Fm2 = Fmx * Fmx + Fmy * Fmy;
    double num = (12.0 * varpi) * Fm2;
    double psi2 = psi * psi;
    S[0] = 0.0;
    S[1] = 6.0 * uF + num / (psi2 * (tau_e - 0.5));
    S[2] = -6.0 * uF + sign_eps * (num / (psi2 * (tau_s - 0.5)));
    S[3] = Fx;
    S[4] = -Fx;
    S[5] = Fy;
    S[6] = -Fy;
    S[7] = 2.0 * (ux * Fx - uy * Fy);
    S[8] = ux * Fy + uy * Fx;
}

/* m* = m - Lambda (m - m_eq) + (I - Lambda/2) S-bar, Eq. 7 */
void orc_relax(const double *m, const double *meq, const double *S, const double *s, double *ms)
{
    for (int k = 0; k < 9; k++) ms[k] = (m[k] - s[k] * (m[k] - meq[k])) + (1.0 - 0.5 * s[k]) * S[k];
}

/* ---- run object ---------------------------------------------------------- */
static int wrapx(int x, int nx) { return ((x % nx) + nx) % nx; }

/* Threads for the per-site loops (1 = serial, the checker's setting).  Each
 * loop iteration writes only its own sites and reads values no other
 * iteration of the same loop writes, and the diagnostics sums stay serial,
 * so any thread count gives bit-identical results (built without OpenMP the
 * pragmas are ignored and the count has no effect). */
static int g_threads = 1;
void orc_set_threads(int n) { g_threads = n > 0 ? n : 1; }
int orc_threads(void) { return g_threads; }
#define ORC_PARALLEL_ROWS _Pragma("omp parallel for schedule(static) num_threads(g_threads) if(g_threads > 1)")
#define ORC_PARALLEL_ROWS_ERR _Pragma("omp parallel for schedule(static) num_threads(g_threads) if(g_threads > 1) reduction(|:err)")

void orc_destroy(orc_run *r)
{
    if (!r) return;
    free(r->f); free(r->fs); free(r->rho); free(r->ux); free(r->uy); free(r->psi); free(r->T);
    free(r->cw); free(r->lam); free(r->Tk); free(r->Ta); free(r->h); free(r->acc);
    free(r->uxe); free(r->uye); free(r->rhoe); free(r->q_top);
    free(r);
}

/* Per-column wettability coefficient c_w = G_w psi(rho_w) of Eq. 14 along the
 * heater surface.  reading: nucleate spots (Sec. 4.1) are columns within
 * spot_half_width (periodic distance) of each spot centre. */
static void build_cw(orc_run *r)
{
    const orc_params *p = &r->p;
    for (int x = 0; x < p->nx; x++) {
        double c = p->c_w_base;
        for (int k = 0; k < p->n_spots; k++) {
            int d = x - p->spot_x[k];
            d = wrapx(d, p->nx);
            if (d > p->nx - d) d = p->nx - d;
            if (d <= p->spot_half_width) c = p->c_w_spot[k];
        }
        r->cw[x] = c;
    }
}

orc_run *orc_create(const orc_params *prm)
{
    orc_run *r = (orc_run *)calloc(1, sizeof(orc_run));
    if (!r) return NULL;
    r->p = *prm;
    const orc_params *p = &r->p;
    int nx = p->nx, nf = p->nf;
    r->nt = p->ns + nf;
    size_t nfl = (size_t)nx * nf, ntl = (size_t)nx * (r->nt + 1);
    r->f = (double *)calloc(9 * nfl, sizeof(double));
    r->fs = (double *)calloc(9 * nfl, sizeof(double));
    r->rho = (double *)calloc(nfl, sizeof(double));
    r->ux = (double *)calloc(nfl, sizeof(double));
    r->uy = (double *)calloc(nfl, sizeof(double));
    r->psi = (double *)calloc(nfl, sizeof(double));
    r->T = (double *)calloc((size_t)nx * r->nt, sizeof(double));
    r->cw = (double *)calloc(nx, sizeof(double));
    r->lam = (double *)calloc(ntl, sizeof(double));
    r->Tk = (double *)calloc(ntl, sizeof(double));
    r->Ta = (double *)calloc(ntl, sizeof(double));
    r->h = (double *)calloc(ntl, sizeof(double));
    r->acc = (double *)calloc(ntl, sizeof(double));
    r->uxe = (double *)calloc(ntl, sizeof(double));
    r->uye = (double *)calloc(ntl, sizeof(double));
    r->rhoe = (double *)calloc(ntl, sizeof(double));
    r->q_top = (double *)calloc(nx, sizeof(double));
    if (!r->f || !r->fs || !r->rho || !r->ux || !r->uy || !r->psi || !r->T || !r->cw || !r->lam ||
        !r->Tk || !r->Ta || !r->h || !r->acc || !r->uxe || !r->uye || !r->rhoe || !r->q_top) {
        orc_destroy(r);
        return NULL;
    }
    r->Tc = orc_Tc(p->a, p->b, p->R);
    r->kappa = orc_kappa(p->omega);
    r->T_sat = p->T_sat_over_Tc * r->Tc;
    r->T_b = p->T_b_over_Tc * r->Tc;
    /* Eq. 4: tau = nu / c_s^2 + 0.5 */
    r->tau_L = 3.0 * p->nu_L + 0.5;
    r->tau_V = 3.0 * p->nu_V + 0.5;
    build_cw(r);

    /* Initial state (Sec. 3.1): liquid below, vapour above, at rest, T = T_sat
     * everywhere including the heater; per-site density noise of relative
     * amplitude init_noise; f = equilibrium at rest = w_i rho. */
    for (int y = 0; y < nf; y++)
        for (int x = 0; x < nx; x++) {
            double base = (y < p->liquid_rows) ? p->rho_L : p->rho_V;
            double U = orc_uniform(p->seed, TAG_INIT, 0, (unsigned long long)y * nx + x);
            double rho = base * (1.0 + p->init_noise * (2.0 * U - 1.0));
            for (int i = 0; i < 9; i++) r->f[(size_t)i * nfl + (size_t)y * nx + x] = WL[i] * rho;
            r->rho[(size_t)y * nx + x] = rho;
        }
    for (size_t k = 0; k < (size_t)nx * r->nt; k++) r->T[k] = r->T_sat;
    if (p->rho_mean > 0.0) {
        r->rho_bar = p->rho_mean;
    } else {
        double s = 0.0;
        for (size_t k = 0; k < nfl; k++) s += r->rho[k];
        r->rho_bar = s / (double)nfl;
    }
    r->step = 0;
    return r;
}

/* Bottom temperature of column x at step n (Sec. 3.2, 4.1):
 * SPOTS: constant T_b; NOISE: T_b (1 + A (2U - 1)), U drawn per column and
 * step; SINE: T_b + A_s Tc sin(2 pi (x - l/4) / l) for t0 < n < t1. */
static double bottom_T(const orc_run *r, int x, long long n)
{
    const orc_params *p = &r->p;
    if (p->bc_mode == BC_NOISE) {
        double U = orc_uniform(p->seed, TAG_BC, (unsigned long long)n, (unsigned long long)x);
        return r->T_b * (1.0 + p->bc_noise * (2.0 * U - 1.0));
    }
    if (p->bc_mode == BC_SINE && n > p->sine_t0 && n < p->sine_t1) {
        double wl = p->sine_wavelength;
        double arg = (2.0 * M_PI) * ((double)x - wl / 4.0) / wl;
        return r->T_b + (p->sine_amp_over_Tc * r->Tc) * sin(arg);
    }
    return r->T_b;
}

/* ---- flow half of the step (Eq. 1-15, halfway bounce-back) -------------- */
static void lbm_part(orc_run *r)
{
    const orc_params *p = &r->p;
    const int nx = p->nx, nf = p->nf, ns = p->ns;
    const size_t nfl = (size_t)nx * nf;
    const int py = (p->flags & F_PERIODIC_Y) != 0;
    const double tau_e = 1.0 / p->s[1], tau_s = 1.0 / p->s[2];

    /* 1. density (Eq. 10) and pseudopotential (Eq. 12-13) at every fluid site */
    unsigned err = 0;
    ORC_PARALLEL_ROWS_ERR
    for (int y = 0; y < nf; y++)
        for (int x = 0; x < nx; x++) {
            size_t k = (size_t)y * nx + x;
            double rho = 0.0;
            for (int i = 0; i < 9; i++) rho += r->f[(size_t)i * nfl + k];
            int bad = 0;
            double T = r->T[(size_t)(ns + y) * nx + x];
            r->rho[k] = rho;
            r->psi[k] = orc_psi(rho, T, p->a, p->b, p->R, r->kappa, r->Tc, p->G, &bad);
            if (bad) err |= ERR_PSI;
            if (!isfinite(rho)) err |= ERR_NONFINITE;
        }
    r->err |= err;

    /* 2-4. forces, velocity, relaxation time, MRT collision at every site */
    ORC_PARALLEL_ROWS
    for (int y = 0; y < nf; y++)
        for (int x = 0; x < nx; x++) {
            size_t k = (size_t)y * nx + x;
            double rho = r->rho[k], psi = r->psi[k];
            /* Eq. 11: F_m = -G psi(x) sum_i w(|e_i|^2) psi(x + e_i) e_i over fluid
             * neighbours; Eq. 14 (reading): F_ads = -psi(x) sum over solid
             * neighbours of w c_w e_i, c_w = G_w psi(rho_w) of that wall site. */
            double sx = 0.0, sy = 0.0, ax = 0.0, ay = 0.0;
            for (int i = 1; i < 9; i++) {
                int xn = wrapx(x + EX[i], nx), yn = y + EY[i];
                if (py) yn = wrapx(yn, nf);
                if (yn >= 0 && yn < nf) {
                    double t = WF[i] * r->psi[(size_t)yn * nx + xn];
                    if (EX[i]) sx += EX[i] * t;
                    if (EY[i]) sy += EY[i] * t;
                } else if (yn >= nf && p->top_mode == TOP_OUTFLOW) {
                    /* reading: open top, psi has zero normal gradient */
                    double t = WF[i] * r->psi[(size_t)(nf - 1) * nx + xn];
                    if (EX[i]) sx += EX[i] * t;
                    if (EY[i]) sy += EY[i] * t;
                } else {
                    double cw = (yn < 0) ? r->cw[xn] : p->c_w_top;
                    double t = WF[i] * cw;
                    if (EX[i]) ax += EX[i] * t;
                    if (EY[i]) ay += EY[i] * t;
                }
            }
            double pre = -p->G * psi;
            double Fmx = pre * sx, Fmy = pre * sy;
            double Fax = -psi * ax, Fay = -psi * ay;
            /* Eq. 15: F_g = (rho - rho_bar) (0, -g) */
            double Fgy = -((rho - r->rho_bar) * p->g);
            double Fx = Fmx + Fax;
            double Fy = (Fmy + Fay) + Fgy;

            double f[9], m[9], meq[9], S[9], ms[9], s[9], fo[9];
            for (int i = 0; i < 9; i++) f[i] = r->f[(size_t)i * nfl + k];
            orc_moments(f, m);
            /* Eq. 10: rho v = sum e f + F / 2 */
            double ux = (m[3] + 0.5 * Fx) / rho;
            double uy = (m[5] + 0.5 * Fy) / rho;
            /* Eq. 5 then Eq. 4: s7 = s8 = 1 / tau_nu(rho) */
            double tau = r->tau_V + ((rho - p->rho_V) / (p->rho_L - p->rho_V)) * (r->tau_L - r->tau_V);
            for (int i = 0; i < 9; i++) s[i] = p->s[i];
            s[7] = 1.0 / tau;
            s[8] = s[7];
            orc_meq(rho, ux, uy, meq);
            orc_source(ux, uy, Fx, Fy, Fmx, Fmy, psi, p->varpi, tau_e, tau_s, p->sign_eps, S);
            orc_relax(m, meq, S, s, ms);
            orc_inverse_moments(ms, fo);
            for (int i = 0; i < 9; i++) r->fs[(size_t)i * nfl + k] = fo[i];
            r->ux[k] = ux;
            r->uy[k] = uy;
        }

    /* 5. streaming, Eq. 8, pulled from x - e_i; halfway bounce-back (static
     * walls) when x - e_i is a heater or top-wall site; OUTFLOW top (option):
     * unknown downward populations copied from the row below (zero gradient). */
    ORC_PARALLEL_ROWS
    for (int y = 0; y < nf; y++)
        for (int x = 0; x < nx; x++) {
            size_t k = (size_t)y * nx + x;
            for (int i = 0; i < 9; i++) {
                int xs = wrapx(x - EX[i], nx), ys = y - EY[i];
                if (py) ys = wrapx(ys, nf);
                double v;
                if (ys >= 0 && ys < nf) {
                    v = r->fs[(size_t)i * nfl + (size_t)ys * nx + xs];
                } else if (ys >= nf && p->top_mode == TOP_OUTFLOW) {
                    v = r->fs[(size_t)i * nfl + (size_t)y * nx + xs];
                } else {
                    v = r->fs[(size_t)OPP[i] * nfl + k];
                }
                r->f[(size_t)i * nfl + k] = v;
            }
        }
}

/* ---- heat half of the step (Eq. 24-28, RK4 with frozen rho, u) ---------- */
/* harmonic mean of two conductivities at a link (reading: conservative
 * conduction across the heater/fluid jump) */
static double hmean(double a, double b) { return (2.0 * (a * b)) / (a + b); }

/* Energy equation right-hand side K(T) of Eq. 24 at extended row r, column x,
 * for the stage temperature Tk.  Extended rows: 0..nt-1 physical, nt = top
 * ghost (T_sat, u = 0, lambda copied from row nt-1). */
static double K_site(const orc_run *r, const double *Tk, int row, int x)
{
    const orc_params *p = &r->p;
    const int nx = p->nx, nt = r->nt;
    const int py = (p->flags & F_PERIODIC_Y) != 0;
    size_t k0 = (size_t)row * nx + x;
    double T0 = Tk[k0], l0 = r->lam[k0];
    double sD = 0.0, gx = 0.0, gy = 0.0, dxu = 0.0, dyu = 0.0;
    for (int a = 1; a < 9; a++) {
        int xn = wrapx(x + EX[a], nx), rn = row + EY[a];
        if (py) rn = wrapx(rn, nt);
        size_t kn = (size_t)rn * nx + xn;
        double Ta = Tk[kn];
        /* Eq. 28 with the conductivity inside: 6 sum w_a lambda_face (T_a - T) */
        sD += WL[a] * (hmean(l0, r->lam[kn]) * (Ta - T0));
        /* Eq. 27: 3 sum w_a phi_a e_a */
        double wT = WL[a] * Ta, wux = WL[a] * r->uxe[kn], wuy = WL[a] * r->uye[kn];
        if (EX[a]) { gx += EX[a] * wT; dxu += EX[a] * wux; }
        if (EY[a]) { gy += EY[a] * wT; dyu += EY[a] * wuy; }
    }
    double D = 6.0 * sD;
    if (!py && row < p->ns) return D / p->rho_c_s; /* solid: conduction only */
    gx = 3.0 * gx;
    gy = 3.0 * gy;
    double divu = 3.0 * dxu + 3.0 * dyu;
    double rho = r->rhoe[k0];
    double ux = r->uxe[k0], uy = r->uye[k0];
    double rcv = rho * p->c_v;
    double adv = ux * gx + uy * gy;
    double dp = orc_dpdT(rho, T0, p->a, p->b, p->R, r->kappa, r->Tc);
    return (-adv + D / rcv) - (((T0 / rcv) * dp) * divu);
}

static void fd_part(orc_run *r)
{
    const orc_params *p = &r->p;
    const int nx = p->nx, nf = p->nf, ns = p->ns, nt = r->nt;
    const int py = (p->flags & F_PERIODIC_Y) != 0;
    const int ext = py ? nt : nt + 1; /* rows held in the work arrays */
    /* frozen fields on the extended grid */
    ORC_PARALLEL_ROWS
    for (int row = 0; row < ext; row++)
        for (int x = 0; x < nx; x++) {
            size_t k = (size_t)row * nx + x;
            if (row < ns) {
                /* Model A: the wall row conducts like the first fluid row */
                r->lam[k] = (p->flags & F_MODEL_A) ? p->cv_chi * r->rho[x] : p->lambda_s;
                r->uxe[k] = 0.0; r->uye[k] = 0.0; r->rhoe[k] = 0.0;
            } else if (row < nt) {
                size_t kf = (size_t)(row - ns) * nx + x;
                double rho = r->rho[kf];
                r->lam[k] = p->cv_chi * rho; /* lambda = rho C_V chi (Sec. 3.1) */
                r->uxe[k] = r->ux[kf]; r->uye[k] = r->uy[kf]; r->rhoe[k] = rho;
            } else { /* top ghost */
                r->lam[k] = r->lam[(size_t)(nt - 1) * nx + x];
                r->uxe[k] = 0.0; r->uye[k] = 0.0; r->rhoe[k] = 0.0;
            }
        }
    /* Dirichlet rows: bottom row 0 already holds T_b(x, n); top ghost = T_sat */
    ORC_PARALLEL_ROWS
    for (int row = 0; row < ext; row++)
        for (int x = 0; x < nx; x++) {
            size_t k = (size_t)row * nx + x;
            r->Tk[k] = (row < nt) ? r->T[k] : r->T_sat;
        }
    const int r0 = py ? 0 : 1, r1 = nt; /* evolved rows [r0, r1) */
    /* Eq. 25-26 */
    for (int stage = 0; stage < 4; stage++) {
        ORC_PARALLEL_ROWS
        for (int row = r0; row < r1; row++)
            for (int x = 0; x < nx; x++) r->h[(size_t)row * nx + x] = K_site(r, r->Tk, row, x);
        ORC_PARALLEL_ROWS
        for (int row = r0; row < r1; row++)
            for (int x = 0; x < nx; x++) {
                size_t k = (size_t)row * nx + x;
                double hk = r->h[k], Tn = r->T[k];
                if (stage == 0) {
                    r->acc[k] = hk;
                    r->Ta[k] = Tn + 0.5 * hk;
                } else if (stage == 1) {
                    r->acc[k] = r->acc[k] + 2.0 * hk;
                    r->Ta[k] = Tn + 0.5 * hk;
                } else if (stage == 2) {
                    r->acc[k] = r->acc[k] + 2.0 * hk;
                    r->Ta[k] = Tn + hk;
                } else {
                    r->acc[k] = r->acc[k] + hk;
                }
            }
        if (stage < 3) {
            ORC_PARALLEL_ROWS
            for (int row = r0; row < r1; row++)
                for (int x = 0; x < nx; x++) {
                    size_t k = (size_t)row * nx + x;
                    r->Tk[k] = r->Ta[k];
                }
        }
    }
    unsigned err = 0;
    ORC_PARALLEL_ROWS_ERR
    for (int row = r0; row < r1; row++)
        for (int x = 0; x < nx; x++) {
            size_t k = (size_t)row * nx + x;
            double Tn1 = r->T[k] + r->acc[k] / 6.0;
            if (!isfinite(Tn1)) err |= ERR_NONFINITE;
            r->T[k] = Tn1;
        }
    r->err |= err;
}

/* Diagnostics after the step: Eq. 36/39 heat flux at the heater bottom
 * (lambda_s, rows 0-2), local flux through the heater/fluid interface, vapour
 * fraction (rho below the mean of the coexistence densities), total mass.
 * Model A has no heater: both fluxes are the flux through the heated wall,
 * -lambda_f (T(first fluid row) - T_b). */
static void diagnostics(orc_run *r)
{
    const orc_params *p = &r->p;
    const int nx = p->nx, nf = p->nf, ns = p->ns;
    const int model_a = (p->flags & F_MODEL_A) != 0;
    double qb = 0.0, qt = 0.0, mass = 0.0;
    long long nvap = 0;
    double thr = 0.5 * (p->rho_L + p->rho_V);
    if (ns >= 3 && !model_a && !(p->flags & F_PERIODIC_Y)) {
        for (int x = 0; x < nx; x++) {
            double T0 = r->T[x], T1 = r->T[nx + x], T2 = r->T[2 * nx + x];
            double dTdy = ((4.0 * T1 - T2) - 3.0 * T0) / 2.0;
            qb += -p->lambda_s * dTdy;
        }
        qb = qb / (double)nx;
    }
    if (ns >= 1 && !(p->flags & F_PERIODIC_Y)) {
        for (int x = 0; x < nx; x++) {
            double lw = model_a ? p->cv_chi * r->rho[x] : p->lambda_s;
            double lf = hmean(lw, p->cv_chi * r->rho[x]);
            double q = -lf * (r->T[(size_t)ns * nx + x] - r->T[(size_t)(ns - 1) * nx + x]);
            r->q_top[x] = q;
            qt += q;
        }
        qt = qt / (double)nx;
        if (model_a) qb = qt;
    }
    for (size_t k = 0; k < (size_t)nx * nf; k++) {
        mass += r->rho[k];
        if (r->rho[k] < thr) nvap++;
    }
    r->diag[0] = qb;
    r->diag[1] = qt;
    r->diag[2] = (double)nvap / (double)((size_t)nx * nf);
    r->diag[3] = mass;
}

/* One time step n -> n+1: bottom row := T_b(x, n); flow half (uses T^n);
 * heat half (uses rho^n, u^n of this step, frozen over the four stages). */
void orc_step(orc_run *r, long long nsteps)
{
    const orc_params *p = &r->p;
    for (long long it = 0; it < nsteps; it++) {
        long long n = r->step;
        if (!(p->flags & F_PERIODIC_Y) && p->ns >= 1)
            for (int x = 0; x < p->nx; x++) r->T[x] = bottom_T(r, x, n);
        if (!(p->flags & F_FROZEN_FLOW)) {
            lbm_part(r);
        } else {
            /* frozen flow: rho from the populations, u = 0, populations kept */
            size_t nfl = (size_t)p->nx * p->nf;
            for (size_t k = 0; k < nfl; k++) {
                double rho = 0.0;
                for (int i = 0; i < 9; i++) rho += r->f[(size_t)i * nfl + k];
                r->rho[k] = rho;
                r->ux[k] = 0.0;
                r->uy[k] = 0.0;
            }
        }
        if (!(p->flags & F_ISOTHERMAL)) fd_part(r);
        diagnostics(r);
        r->step = n + 1;
    }
}

/* ---- accessors ----------------------------------------------------------- */
double *orc_f(orc_run *r) { return r->f; }
double *orc_T(orc_run *r) { return r->T; }
double *orc_rho(orc_run *r) { return r->rho; }
double *orc_ux(orc_run *r) { return r->ux; }
double *orc_uy(orc_run *r) { return r->uy; }
double *orc_q_top(orc_run *r) { return r->q_top; }
const double *orc_diag(orc_run *r) { return r->diag; }
long long orc_get_step(orc_run *r) { return r->step; }
void orc_set_step(orc_run *r, long long n) { r->step = n; }
unsigned orc_err(orc_run *r) { return r->err; }
double orc_rho_bar(orc_run *r) { return r->rho_bar; }
double orc_run_Tc(orc_run *r) { return r->Tc; }
void orc_set_rho_bar(orc_run *r, double v) { r->rho_bar = v; }
int orc_params_size(void) { return (int)sizeof(orc_params); }

/* Expose K and the FD operators on an arbitrary field for the tests:
 * gradient (Eq. 27) and Laplacian (Eq. 28) of phi on a periodic nx x ny grid. */
void orc_grad_lap(const double *phi, int nx, int ny, double *gx, double *gy, double *lap)
{
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            double p0 = phi[(size_t)y * nx + x], sx = 0.0, sy = 0.0, sl = 0.0;
            for (int a = 1; a < 9; a++) {
                double pa = phi[(size_t)wrapx(y + EY[a], ny) * nx + wrapx(x + EX[a], nx)];
                double w = WL[a] * pa;
                if (EX[a]) sx += EX[a] * w;
                if (EY[a]) sy += EY[a] * w;
                sl += WL[a] * (pa - p0);
            }
            gx[(size_t)y * nx + x] = 3.0 * sx;
            gy[(size_t)y * nx + x] = 3.0 * sy;
            lap[(size_t)y * nx + x] = 6.0 * sl;
        }
}

/* One collision of a single site, for the moment-space pins. */
void orc_collide_site(const double *f, double Fx, double Fy, double Fmx, double Fmy, double psi,
                      double varpi, const double *s, double sign_eps, double *fo)
{
    double m[9], meq[9], S[9], ms[9];
    orc_moments(f, m);
    double rho = m[0];
    double ux = (m[3] + 0.5 * Fx) / rho, uy = (m[5] + 0.5 * Fy) / rho;
    orc_meq(rho, ux, uy, meq);
    orc_source(ux, uy, Fx, Fy, Fmx, Fmy, psi, varpi, 1.0 / s[1], 1.0 / s[2], sign_eps, S);
    orc_relax(m, meq, S, s, ms);
    orc_inverse_moments(ms, fo);
}

void orc_source_vec(double ux, double uy, double Fx, double Fy, double Fmx, double Fmy, double psi,
                    double varpi, double tau_e, double tau_s, double sign_eps, double *S)
{
    orc_source(ux, uy, Fx, Fy, Fmx, Fmy, psi, varpi, tau_e, tau_s, sign_eps, S);
}

/* The published splitmix64 generator step (state += golden gamma, then the
 * finaliser), exposed so the tests can pin mix64 against its reference
 * output sequence. */
unsigned long long orc_splitmix64_next(unsigned long long *state)
{
    *state += 0x9E3779B97F4A7C15ULL;
    return mix64(*state);
}
