// Host FP64 scalar tables of the attenuation model (Sec. II-A, II-B).
//
// mu(E) / S = rho_e (Cp Z^m / E^n + KN(E)), with S = n_w * 1 barn (water
// electron density n_w = 3.3428e23 /cm^3, expressed per mm), Cp = 9.8e-24 cm^2
// (9.8 barn keV^n), m = 3.8, n = 3.2 and KN the Klein-Nishina total
// cross-section per electron.  The Z^m unknown is carried as z = Z^m / Z_w^m
// (Z_w = 7.45), so the photoelectric term at energy E is P(E) z with
// P(E) = Cp Z_w^m / E^n.  The rho_e and Z^m surrogate equations (eq. rho_e,
// eq. Z_m) are scaled to unit coefficient at water.
#include <cmath>
#include <vector>

#include "model_tables.h"

namespace recon {

namespace {
constexpr double kCpBarn = 9.8;       // Cp = 9.8e-24 cm^2
constexpr double kM = 3.8;            // exponent of Z
constexpr double kN = 3.2;            // exponent of E
constexpr double kR0Cm = 2.818e-13;   // classical electron radius as printed
constexpr double kMec2 = 510.975;     // keV
constexpr double kNw = 3.3428e23;     // electrons / cm^3 in water
constexpr double kZw = 7.45;
constexpr double kPi = 3.14159265358979323846;
}  // namespace

double water_z() { return kZw; }
double z_exponent() { return kM; }
double scale_per_mm() { return kNw * 1e-24 * 0.1; }

double klein_nishina_barn(double e_kev) {
    // 2 pi r0^2 { (1+g)/g^2 [2(1+g)/(1+2g) - ln(1+2g)/g] + ln(1+2g)/(2g)
    //             - (1+3g)/(1+2g)^2 },   g = E / 510.975 keV
    const double g = e_kev / kMec2;
    const double c0 = 2.0 * kPi * (kR0Cm * 1e12) * (kR0Cm * 1e12);  // r0 in 1e-12 cm -> barn
    const double l = std::log1p(2.0 * g);
    const double one2g = 1.0 + 2.0 * g;
    const double a = (1.0 + g) / (g * g) * (2.0 * (1.0 + g) / one2g - l / g);
    const double b = l / (2.0 * g);
    const double c = (1.0 + 3.0 * g) / (one2g * one2g);
    return c0 * (a + b - c);
}

double photo_per_z(double e_kev) { return kCpBarn * std::pow(kZw, kM) / std::pow(e_kev, kN); }

double mu_norm(double Z, double rhoe, double e_kev) {
    return rhoe * (kCpBarn * std::pow(Z, kM) / std::pow(e_kev, kN) + klein_nishina_barn(e_kev));
}

void spectrum_bins(const recon_spectrum& s, std::vector<double>& e, std::vector<double>& w) {
    e.clear();
    w.clear();
    if (s.kind == 0) {
        e.push_back(s.kev);
        w.push_back(1.0);
        return;
    }
    double sum = 0.0;
    for (double E = 10.0; E < s.kvp; E += 1.0) {
        double phi = (s.kvp - E) / E;
        for (int f = 0; f < s.n_filters && f < RECON_MAX_FILTERS; ++f) {
            const recon_filter& fl = s.filters[f];
            phi *= std::exp(-scale_per_mm() * mu_norm(fl.Z, fl.rhoe, E) * fl.thickness_mm);
        }
        e.push_back(E);
        w.push_back(phi);
        sum += phi;
    }
    for (double& x : w) x /= sum;
}

Tables make_tables(const recon_params& p) {
    Tables t{};
    const recon_spectrum* arms[2] = {&p.low, &p.high};
    std::vector<double> e, w;
    for (int i = 0; i < 2; ++i) {
        spectrum_bins(*arms[i], e, w);
        for (int k = 0; k < 2; ++k) {
            double acc = 0.0;
            for (size_t b = 0; b < e.size(); ++b) acc += w[b] * mu_norm(p.basis_z[k], p.basis_rhoe[k], e[b]);
            t.a[k][i] = acc;
        }
    }
    const double ej[2] = {p.e1_kev, p.e2_kev};
    for (int j = 0; j < 2; ++j) {
        for (int k = 0; k < 2; ++k) t.b[k][j] = mu_norm(p.basis_z[k], p.basis_rhoe[k], ej[j]);
        t.P[j] = photo_per_z(ej[j]);
        t.psi[j] = klein_nishina_barn(ej[j]);
    }
    t.r = std::pow(p.e1_kev / p.e2_kev, kN);
    for (int k = 0; k < 2; ++k)
        t.c_f[k] = t.a[k][0] * t.a[k][0] + t.a[k][1] * t.a[k][1] + t.b[k][0] * t.b[k][0] + t.b[k][1] * t.b[k][1];
    t.c12 = t.a[0][0] * t.a[1][0] + t.a[0][1] * t.a[1][1] + t.b[0][0] * t.b[1][0] + t.b[0][1] * t.b[1][1];
    t.c_rho = t.psi[0] * t.r - t.psi[1];
    const double mw1 = t.P[0] + t.psi[0], mw2 = t.P[1] + t.psi[1];
    t.a_w = mw1 * t.P[1] - mw2 * t.P[0];
    t.det = t.a[0][0] * t.a[1][1] - t.a[0][1] * t.a[1][0];
    t.S = scale_per_mm();
    t.zclip_hi = std::pow(p.z_clip_max / kZw, kM);
    return t;
}

}  // namespace recon
