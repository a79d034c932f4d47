// Host FP64 model tables shared by the solver and the scan simulator.
#pragma once
#include <vector>

#include "recon.h"

namespace recon {

struct Tables {
    double a[2][2];   // a[k][i]: basis k at arm i (E_L, E_H), normalised mu
    double b[2][2];   // b[k][j]: basis k at synthesis energy E_j
    double P[2];      // photoelectric coefficient per unit z at E1, E2
    double psi[2];    // Klein-Nishina at E1, E2 (barn)
    double r;         // (E1/E2)^n
    double c_f[2];    // f-update data coefficients
    double c12;       // cross term of the f data terms
    double c_rho;     // coefficient of eq. rho_e divided by E2^n
    double a_w;       // coefficient of eq. Z_m (normalised) at water
    double det;       // a11 a22 - a12 a21 (Cramer)
    double S;         // 1/mm per barn of water electron density
    double zclip_hi;  // initial z upper clip
};

double klein_nishina_barn(double e_kev);
double photo_per_z(double e_kev);
double mu_norm(double Z, double rhoe, double e_kev);
double scale_per_mm();
double water_z();
double z_exponent();
void spectrum_bins(const recon_spectrum& s, std::vector<double>& e, std::vector<double>& w);
Tables make_tables(const recon_params& p);

}  // namespace recon
