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
 * linearly in ln E in FP64.  mu_pair is zero at and below 2 mc^2 whatever
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
