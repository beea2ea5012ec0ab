// xs.cpp -- synthetic photon attenuation tables (closed-form models, FP64 -> FP32).
//
// The paper's Gadep takes photoelectric, Compton and pair cross sections from the
// Livermore evaluated data (Sec. 2.4.1).  Those data are not part of this
// library; it tabulates closed-form models with the same structure instead:
//   Compton          Klein-Nishina total cross section per free electron
//                    sigma = 2 pi r_e^2 [ (1+k)/k^2 (2(1+k)/(1+2k) - ln(1+2k)/k)
//                                        + ln(1+2k)/(2k) - (1+3k)/(1+2k)^2 ],
//                    k = E / m_e c^2, times the electron density rho N_A Z / A;
//   photoabsorption  Born-approximation K-shell formula (Heitler)
//                    (32 pi sqrt(2) / 3) r_e^2 alpha^4 Z^5 (m_e c^2 / E)^(7/2),
//                    scaled by 5/4 for the outer shells, per atom;
//   pair production  near-threshold form (2 pi / 3) alpha r_e^2 Z^2 ((k - 2)/k)^3, k > 2.
// Mixtures add atom densities.  CODATA 2018 constants.
//
// gadep_erange_build: CSDA ranges of electrons for the charged-particle model
// (the stand-in for the paper's electron transport): stopping power
//   S(T) = S_col(T) (1 + Z_r T / 800 MeV),
//   S_col = 2 pi r_e^2 m_e c^2 N_A (Z/A) beta^-2
//           [ ln(tau^2 (tau + 2) / (2 (I / m_e c^2)^2)) + F(tau) ],
//   F(tau) = 1 - beta^2 + (tau^2 / 8 - (2 tau + 1) ln 2) / (tau + 1)^2
// (Bethe formula for electrons, Rohrlich-Carlson form as in ICRU Report 37,
// density effect left out; radiative share after Attix), and the range
//   R(T) = T_min / S(T_min) + int_{T_min}^{T} dT' / S(T')
// integrated with 4-point Gauss-Legendre rules in ln T between grid points.
#include <cmath>

#include "gadep_internal.h"

namespace {

constexpr double kMeC2 = 510.99895;            // keV
constexpr double kRe = 2.8179403262e-13;       // cm
constexpr double kAlpha = 7.2973525693e-3;
constexpr double kNA = 6.02214076e23;
constexpr double kPi = 3.14159265358979323846;

struct Element { int Z; double A; double per_unit; };
struct Material { int n; Element e[2]; double rho; };

bool material_of(int code, Material *m)
{
    switch (code) {
    case GADEP_MAT_VACUUM: *m = Material{ 0, {}, 0.0 }; return true;
    case GADEP_MAT_GE: *m = Material{ 1, { { 32, 72.630, 1.0 } }, 5.323 }; return true;
    case GADEP_MAT_AL: *m = Material{ 1, { { 13, 26.982, 1.0 } }, 2.699 }; return true;
    case GADEP_MAT_CU: *m = Material{ 1, { { 29, 63.546, 1.0 } }, 8.96 }; return true;
    case GADEP_MAT_WATER: *m = Material{ 2, { { 1, 1.008, 2.0 }, { 8, 15.999, 1.0 } }, 1.0 }; return true;
    default: return false;
    }
}

double klein_nishina(double k)
{
    const double a = 1.0 + 2.0 * k, la = std::log(a);
    return 2.0 * kPi * kRe * kRe *
           ((1.0 + k) / (k * k) * (2.0 * (1.0 + k) / a - la / k) + la / (2.0 * k) -
            (1.0 + 3.0 * k) / (a * a));
}

double born_photo(int Z, double E)
{
    const double z5 = std::pow((double)Z, 5.0);
    return 1.25 * (32.0 * kPi * std::sqrt(2.0) / 3.0) * kRe * kRe * std::pow(kAlpha, 4.0) * z5 *
           std::pow(kMeC2 / E, 3.5);
}

double pair_threshold(int Z, double E)
{
    const double k = E / kMeC2;
    if (k <= 2.0) return 0.0;
    const double r = (k - 2.0) / k;
    return (2.0 * kPi / 3.0) * kAlpha * kRe * kRe * (double)Z * (double)Z * r * r * r;
}

// Mean excitation energy (eV), ICRU Report 37; 0 for vacuum.
double mean_excitation(int code)
{
    switch (code) {
    case GADEP_MAT_GE: return 350.0;
    case GADEP_MAT_AL: return 166.0;
    case GADEP_MAT_CU: return 322.0;
    case GADEP_MAT_WATER: return 75.0;
    default: return 0.0;
    }
}

// Total mass stopping power (MeV cm^2 / g) of an electron of kinetic energy T (keV).
double electron_stopping(const Material &m, double I_eV, double T)
{
    double zsum = 0.0, asum = 0.0, z2sum = 0.0;
    for (int k = 0; k < m.n; ++k) {
        zsum += m.e[k].per_unit * m.e[k].Z;
        asum += m.e[k].per_unit * m.e[k].A;
        z2sum += m.e[k].per_unit * (double)m.e[k].Z * m.e[k].Z;
    }
    const double tau = T / kMeC2, gam = 1.0 + tau;
    const double b2 = (gam * gam - 1.0) / (gam * gam);
    const double ir = I_eV * 1e-3 / kMeC2;
    const double bracket = std::log(tau * tau * (tau + 2.0) / (2.0 * ir * ir)) + 1.0 - b2 +
                           (0.125 * tau * tau - (2.0 * tau + 1.0) * std::log(2.0)) / (gam * gam);
    const double s_col = 2.0 * kPi * kRe * kRe * (kMeC2 * 1e-3) * kNA * (zsum / asum) / b2 * bracket;
    return s_col * (1.0 + (z2sum / zsum) * T * 1e-3 / 800.0);
}

}  // namespace

extern "C" gadep_status gadep_erange_build(const int32_t *codes, int32_t n_mat, int32_t e_n, double T_min,
                                           double T_max, float *range)
{
    gadep::clear_error();
    if (!codes || !range || n_mat < 1 || n_mat > 1024 || e_n < 2 || e_n > (1 << 20) || !(T_min > 0.0) ||
        !(T_max > T_min) || !std::isfinite(T_max))
        return gadep::fail(GADEP_E_INVAL, "gadep_erange_build: bad arguments");
    // 4-point Gauss-Legendre nodes and weights on [-1, 1]
    const double gx[4] = { -0.8611363115940526, -0.3399810435848563, 0.3399810435848563, 0.8611363115940526 };
    const double gw[4] = { 0.3478548451374538, 0.6521451548625461, 0.6521451548625461, 0.3478548451374538 };
    const double l0 = std::log(T_min), dl = (std::log(T_max) - l0) / (e_n - 1);
    for (int32_t i = 0; i < n_mat; ++i) {
        Material m;
        if (!material_of(codes[i], &m))
            return gadep::fail(GADEP_E_INVAL, "gadep_erange_build: unknown material code %d", codes[i]);
        float *row = range + (size_t)i * e_n;
        if (m.n == 0) {
            for (int32_t g = 0; g < e_n; ++g) row[g] = INFINITY;
            continue;
        }
        const double I = mean_excitation(codes[i]);
        const double mm_per_gcm2 = 10.0 / m.rho;
        double R = T_min * 1e-3 / electron_stopping(m, I, T_min);      // g / cm^2
        row[0] = (float)(R * mm_per_gcm2);
        for (int32_t g = 1; g < e_n; ++g) {
            const double mid = l0 + (g - 0.5) * dl;
            double acc = 0.0;
            for (int q = 0; q < 4; ++q) {
                const double T = std::exp(mid + 0.5 * dl * gx[q]);
                acc += gw[q] * T * 1e-3 / electron_stopping(m, I, T);   // dT / S = T dlnT / S
            }
            R += 0.5 * dl * acc;
            row[g] = (float)(R * mm_per_gcm2);
        }
    }
    return GADEP_OK;
}

extern "C" gadep_status gadep_xs_build(const int32_t *codes, int32_t n_mat, int32_t n_grid,
                                       double E_min, double E_max, float *mu)
{
    gadep::clear_error();
    if (!codes || !mu || n_mat < 1 || n_mat > 1024 || n_grid < 2 || n_grid > (1 << 20) ||
        !(E_min > 0.0) || !(E_max > E_min) || !std::isfinite(E_max))
        return gadep::fail(GADEP_E_INVAL, "gadep_xs_build: bad arguments");
    const double l0 = std::log(E_min), dl = (std::log(E_max) - l0) / (n_grid - 1);
    for (int32_t i = 0; i < n_mat; ++i) {
        Material m;
        if (!material_of(codes[i], &m))
            return gadep::fail(GADEP_E_INVAL, "gadep_xs_build: unknown material code %d", codes[i]);
        double molar = 0.0;
        for (int k = 0; k < m.n; ++k) molar += m.e[k].per_unit * m.e[k].A;
        for (int32_t g = 0; g < n_grid; ++g) {
            const double E = std::exp(l0 + g * dl);
            double pe = 0.0, co = 0.0, pa = 0.0;
            if (m.n > 0) {
                const double units = m.rho * kNA / molar;   // formula units per cm^3
                const double kn = klein_nishina(E / kMeC2);
                for (int k = 0; k < m.n; ++k) {
                    const double atoms = units * m.e[k].per_unit;
                    pe += atoms * born_photo(m.e[k].Z, E);
                    co += atoms * m.e[k].Z * kn;
                    pa += atoms * pair_threshold(m.e[k].Z, E);
                }
            }
            // cm^-1 -> mm^-1
            mu[((size_t)i * 3 + 0) * n_grid + g] = (float)(0.1 * pe);
            mu[((size_t)i * 3 + 1) * n_grid + g] = (float)(0.1 * co);
            mu[((size_t)i * 3 + 2) * n_grid + g] = (float)(0.1 * pa);
        }
    }
    return GADEP_OK;
}
