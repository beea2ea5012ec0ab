/*
 * orc_xs.c -- oracle photon cross sections (test infrastructure only).
 *
 * The paper uses the Livermore evaluated photon data (Sec. 2.4.1).  Those data
 * are not available, so the path runs on closed-form synthetic models that
 * have the right structure (textbook formulas, CODATA 2018 constants):
 *   Compton:           Klein-Nishina total cross section per free electron,
 *                      times the electron density.
 *   Photoabsorption:   non-relativistic Born K-shell cross section (Heitler),
 *                      sigma_K = 4 sqrt(2) alpha^4 Z^5 sigma_T (mc^2/E)^(7/2),
 *                      times 5/4 for the outer shells; no absorption edges.
 *   Pair production:   near-threshold leading order
 *                      (2 pi / 3) alpha r_e^2 Z^2 ((k-2)/k)^3 for k > 2.
 * Tables: n_grid log-spaced points; stored rounded to binary32; interpolated
 * linearly in ln E in FP64.
 *
 * Charged particles.  The paper follows the electrons and positrons that
 * photon interactions set in motion with its engine's standard models
 * (Sec. 2.4.1 physics list: bremsstrahlung, multiple scattering).  Their data
 * are not available either; the stand-in here is the continuous-slowing-down
 * approximation (CSDA): a particle of kinetic energy T loses energy at the
 * mass stopping power
 *   S(T) = S_col(T) (1 + Z_r T / 800 MeV),
 * S_col the Bethe formula for electrons in the form of Rohrlich and Carlson
 * (1954) as ICRU Report 37 writes it, without the density-effect term:
 *   S_col = 2 pi r_e^2 mc^2 N_A (Z/A) / beta^2
 *           [ ln(tau^2 (tau + 2) / (2 (I/mc^2)^2)) + F(tau) ],
 *   F(tau) = 1 - beta^2 + (tau^2/8 - (2 tau + 1) ln 2) / (tau + 1)^2,
 *   tau = T / mc^2,
 * and the radiative share S_rad/S_col ~ Z T / 800 MeV (Attix, Introduction to
 * Radiological Physics and Radiation Dosimetry), Z_r = sum n Z^2 / sum n Z
 * over the formula unit; the radiated energy is deposited along the track.
 * Mean excitation energies I (ICRU Report 37): Ge 350 eV, Al 166 eV, Cu
 * 322 eV, water 75 eV.  CSDA range
 *   R(T) = T_min / S(T_min) + integral from T_min to T of dT' / S(T')
 * (g/cm^2; divided by the density for mm), T_min = ORC_E_TMIN, tabulated in FP64
 * on 4096 log-spaced energies by Simpson's rule in ln T per interval,
 * interpolated linearly in ln T; the energy left after a path L is the T' with
 * R(T') = R(T) - L, found by bisection.  mu_pair is zero at and below 2 mc^2 whatever
 * the interpolation gives, so pair production can never take a photon below
 * threshold.  Energies outside the grid use the end intervals clamped (f in [0,1]).
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MEC2   510.99895          /* keV */
#define ORC_RE     2.8179403262e-13   /* cm */
#define ORC_ALPHA  (1.0 / 137.035999084)
#define ORC_NA     6.02214076e23      /* 1/mol */
#define ORC_PI     3.14159265358979323846

/* Klein-Nishina total per electron.  The closed form cancels in FP64 as k -> 0
   (relative error ~1e-16 / k^3): 1e-11 at the 10 keV table floor (k = 0.0196). */
double orc_sigma_kn(double k)
{
    double a = 1.0 + 2.0 * k;
    double l = log(a);
    double t1 = (1.0 + k) / (k * k) * (2.0 * (1.0 + k) / a - l / k);
    double t2 = l / (2.0 * k);
    double t3 = (1.0 + 3.0 * k) / (a * a);
    return 2.0 * ORC_PI * ORC_RE * ORC_RE * (t1 + t2 - t3);
}

/* Klein-Nishina: d sigma / d Omega = (r_e^2/2) P^2 (P + 1/P - sin^2 theta),
   P = E'/E = 1/(1 + k(1-c)); per unit cos(theta) multiply by 2 pi. */
double orc_dsigma_kn_dcos(double k, double c)
{
    double P = 1.0 / (1.0 + k * (1.0 - c));
    double s2 = 1.0 - c * c;
    return ORC_PI * ORC_RE * ORC_RE * P * P * (P + 1.0 / P - s2);
}

double orc_sigma_pe(int Z, double E_keV)
{
    double sigma_T = 8.0 * ORC_PI / 3.0 * ORC_RE * ORC_RE;
    double a4 = ORC_ALPHA * ORC_ALPHA * ORC_ALPHA * ORC_ALPHA;
    double z5 = (double)Z * Z * Z * Z * Z;
    double sK = 4.0 * sqrt(2.0) * a4 * z5 * sigma_T * pow(ORC_MEC2 / E_keV, 3.5);
    return 1.25 * sK;
}

double orc_sigma_pair(int Z, double E_keV)
{
    double k = E_keV / ORC_MEC2;
    if (k <= 2.0) return 0.0;
    double r = (k - 2.0) / k;
    return 2.0 * ORC_PI / 3.0 * ORC_ALPHA * ORC_RE * ORC_RE * (double)Z * Z * r * r * r;
}

/* material composition: elements (Z, A in g/mol, atoms per formula unit), density g/cm^3 */
typedef struct { int n; int Z[2]; double A[2]; double cnt[2]; double rho; } orc_matdef;

static int material_def(int code, orc_matdef *m)
{
    memset(m, 0, sizeof(*m));
    switch (code) {
    case ORC_MAT_GE:    m->n = 1; m->Z[0] = 32; m->A[0] = 72.630; m->cnt[0] = 1; m->rho = 5.323; return 0;
    case ORC_MAT_AL:    m->n = 1; m->Z[0] = 13; m->A[0] = 26.982; m->cnt[0] = 1; m->rho = 2.699; return 0;
    case ORC_MAT_CU:    m->n = 1; m->Z[0] = 29; m->A[0] = 63.546; m->cnt[0] = 1; m->rho = 8.96;  return 0;
    case ORC_MAT_WATER: m->n = 2; m->Z[0] = 1;  m->A[0] = 1.008;  m->cnt[0] = 2;
                        m->Z[1] = 8;  m->A[1] = 15.999; m->cnt[1] = 1; m->rho = 1.0; return 0;
    case ORC_MAT_VACUUM: m->n = 0; return 0;
    default: return -1;
    }
}

int orc_mu(int code, double E_keV, double out[3])
{
    orc_matdef m;
    out[0] = out[1] = out[2] = 0.0;
    if (material_def(code, &m) != 0) return -1;
    if (m.n == 0) return 0;
    double molar = 0.0;
    for (int i = 0; i < m.n; ++i) molar += m.cnt[i] * m.A[i];
    double n_units = m.rho * ORC_NA / molar;       /* formula units per cm^3 */
    double k = E_keV / ORC_MEC2;
    double skn = orc_sigma_kn(k);
    double pe = 0, co = 0, pa = 0;
    for (int i = 0; i < m.n; ++i) {
        double n_at = n_units * m.cnt[i];
        pe += n_at * orc_sigma_pe(m.Z[i], E_keV);
        co += n_at * m.Z[i] * skn;
        pa += n_at * orc_sigma_pair(m.Z[i], E_keV);
    }
    /* cm^-1 -> mm^-1 */
    out[0] = 0.1 * pe; out[1] = 0.1 * co; out[2] = 0.1 * pa;
    return 0;
}

/* ---------------- charged particles (CSDA) ---------------- */

static double mean_excitation_eV(int code)
{
    switch (code) {
    case ORC_MAT_GE:    return 350.0;
    case ORC_MAT_AL:    return 166.0;
    case ORC_MAT_CU:    return 322.0;
    case ORC_MAT_WATER: return 75.0;
    default:            return 0.0;
    }
}

int orc_e_stopping(int code, double T_keV, double *s_col, double *s_tot)
{
    orc_matdef m;
    *s_col = *s_tot = 0.0;
    if (material_def(code, &m) != 0) return -1;
    if (m.n == 0) return 0;
    double z = 0.0, a = 0.0, z2 = 0.0;
    for (int i = 0; i < m.n; ++i) {
        z += m.cnt[i] * m.Z[i];
        a += m.cnt[i] * m.A[i];
        z2 += m.cnt[i] * (double)m.Z[i] * m.Z[i];
    }
    double ZA = z / a, Zr = z2 / z;
    double tau = T_keV / ORC_MEC2, g = tau + 1.0;
    double beta2 = 1.0 - 1.0 / (g * g);
    double i_rel = mean_excitation_eV(code) * 1e-3 / ORC_MEC2;
    double F = 1.0 - beta2 + (tau * tau / 8.0 - (2.0 * tau + 1.0) * log(2.0)) / (g * g);
    double K = 2.0 * ORC_PI * ORC_RE * ORC_RE * (ORC_MEC2 * 1e-3) * ORC_NA;   /* MeV cm^2 / mol */
    double col = K * ZA / beta2 * (log(tau * tau * (tau + 2.0) / (2.0 * i_rel * i_rel)) + F);
    *s_col = col;
    *s_tot = col * (1.0 + Zr * (T_keV * 1e-3) / 800.0);
    return 0;
}

/* dT / S in ln T: T (MeV) / S_tot (MeV cm^2/g), g/cm^2 per unit ln T */
static double range_integrand(int code, double lnT)
{
    double T = exp(lnT), c, tot;
    orc_e_stopping(code, T, &c, &tot);
    return T * 1e-3 / tot;
}

static int build_e_range(orc_tables *t, const int *codes, double E_max)
{
    t->e_n = 4096;
    t->lnT_min = log(ORC_E_TMIN);
    t->lnT_max = log(E_max > 2.0 * ORC_E_TMIN ? E_max : 2.0 * ORC_E_TMIN);
    t->e_range = (double *)malloc((size_t)t->n_mat * t->e_n * sizeof(double));
    if (!t->e_range) return -1;
    double h = (t->lnT_max - t->lnT_min) / (t->e_n - 1);
    for (int m = 0; m < t->n_mat; ++m) {
        double *row = t->e_range + (size_t)m * t->e_n;
        orc_matdef md;
        if (material_def(codes[m], &md) != 0) return -1;
        if (md.n == 0) {
            for (int g = 0; g < t->e_n; ++g) row[g] = INFINITY;
            continue;
        }
        double c, tot;
        orc_e_stopping(codes[m], ORC_E_TMIN, &c, &tot);
        double R = ORC_E_TMIN * 1e-3 / tot;                 /* g/cm^2 */
        row[0] = 10.0 * R / md.rho;                          /* mm */
        for (int g = 1; g < t->e_n; ++g) {
            double a = t->lnT_min + (g - 1) * h, b = a + h;
            R += h / 6.0 * (range_integrand(codes[m], a) + 4.0 * range_integrand(codes[m], 0.5 * (a + b)) +
                            range_integrand(codes[m], b));
            row[g] = 10.0 * R / md.rho;
        }
    }
    return 0;
}

double orc_e_range(const orc_tables *t, int m, double T_keV)
{
    const double *row = t->e_range + (size_t)m * t->e_n;
    if (isinf(row[0])) return INFINITY;
    if (T_keV <= ORC_E_TMIN) return row[0] * T_keV / ORC_E_TMIN;
    double h = (t->lnT_max - t->lnT_min) / (t->e_n - 1);
    double gf = (log(T_keV) - t->lnT_min) / h;
    int k = (int)floor(gf);
    if (k > t->e_n - 2) k = t->e_n - 2;
    double f = gf - k;          /* above the table: the last interval extended */
    return row[k] + f * (row[k + 1] - row[k]);
}

double orc_e_energy_after(const orc_tables *t, int m, double T_keV, double L_mm)
{
    double R = orc_e_range(t, m, T_keV);
    if (isinf(R)) return T_keV;
    double left = R - L_mm;
    if (left <= 0.0) return 0.0;
    const double *row = t->e_range + (size_t)m * t->e_n;
    if (left <= row[0]) return ORC_E_TMIN * left / row[0];
    double lo = t->lnT_min, hi = log(T_keV);
    for (int it = 0; it < 200 && hi - lo > 1e-15; ++it) {
        double mid = 0.5 * (lo + hi);
        if (orc_e_range(t, m, exp(mid)) < left) lo = mid;
        else hi = mid;
    }
    return exp(0.5 * (lo + hi));
}

orc_tables *orc_tables_build(const int *codes, int n_mat, int n_grid, double E_min, double E_max)
{
    if (n_mat <= 0 || n_grid < 2 || !(E_min > 0) || !(E_max > E_min)) return NULL;
    orc_tables *t = (orc_tables *)calloc(1, sizeof(*t));
    t->n_mat = n_mat; t->n_grid = n_grid;
    t->lnE_min = log(E_min); t->lnE_max = log(E_max);
    t->mu = (float *)calloc((size_t)n_mat * 3 * n_grid, sizeof(float));
    double step = (t->lnE_max - t->lnE_min) / (n_grid - 1);
    for (int m = 0; m < n_mat; ++m) {
        for (int g = 0; g < n_grid; ++g) {
            double E = exp(t->lnE_min + g * step);
            double mu[3];
            if (orc_mu(codes[m], E, mu) != 0) { orc_tables_free(t); return NULL; }
            for (int c = 0; c < 3; ++c) t->mu[((size_t)m * 3 + c) * n_grid + g] = (float)mu[c];
        }
    }
    if (build_e_range(t, codes, E_max) != 0) { orc_tables_free(t); return NULL; }
    return t;
}

orc_tables *orc_tables_from_array(int n_mat, int n_grid, double E_min, double E_max, const float *mu)
{
    if (n_mat <= 0 || n_grid < 2 || !(E_min > 0) || !(E_max > E_min)) return NULL;
    orc_tables *t = (orc_tables *)calloc(1, sizeof(*t));
    t->n_mat = n_mat; t->n_grid = n_grid;
    t->lnE_min = log(E_min); t->lnE_max = log(E_max);
    size_t n = (size_t)n_mat * 3 * n_grid;
    t->mu = (float *)malloc(n * sizeof(float));
    memcpy(t->mu, mu, n * sizeof(float));
    return t;
}

void orc_tables_free(orc_tables *t)
{
    if (!t) return;
    free(t->mu);
    free(t->e_range);
    free(t);
}

void orc_tables_eval(const orc_tables *t, int m, double E_keV, double out[3])
{
    double step = (t->lnE_max - t->lnE_min) / (t->n_grid - 1);
    double g = (log(E_keV) - t->lnE_min) / step;
    int k = (int)floor(g);
    if (k < 0) k = 0;
    if (k > t->n_grid - 2) k = t->n_grid - 2;
    double f = g - k;
    if (f < 0) f = 0;
    if (f > 1) f = 1;
    for (int c = 0; c < 3; ++c) {
        const float *row = t->mu + ((size_t)m * 3 + c) * t->n_grid;
        out[c] = (1.0 - f) * (double)row[k] + f * (double)row[k + 1];
    }
    if (E_keV <= 2.0 * ORC_MEC2) out[2] = 0.0;
}
