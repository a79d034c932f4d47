"""Attenuation model of Sec. II-A and II-B, in FP64 (oracle; test infrastructure only).

Units.  The paper writes the photoelectric/Compton model (eq. mac_E1_eff,
mac_E2_eff) as a "mass" attenuation equal to rho_e times a per-electron cross
section.  We read every mu/rho of the paper as a linear attenuation expressed
per water electron density (reading R2):

    mu(E) [1/mm] = S * mu_hat(E),     S = n_w * 1e-24 cm^2 * 0.1 = 0.033428 /mm,
    mu_hat(E)    = rho_e * (Cp' Z^m / E^n + KN_b(E))          [barn]

with n_w = 3.3428e23 e/cm^3 (water), Cp' = 9.8 barn keV^n (the paper's
Cp = 9.8e-24 cm^2), m = 3.8, n = 3.2, E in keV, and KN_b the Klein-Nishina
total cross-section in barn.  The Z^m variable is normalised by water,
z = Z^m / Z_w^m with Z_w = 7.45 (reading R3), so that

    mu_hat(E) = rho_e * (P(E) z + psi(E)),   P(E) = Cp' Z_w^m / E^n,  psi = KN_b.

Pins: KN against its Thomson limit and closed-form values, and the exact
recovery of (Z, rho_e) through eq. rho_e / eq. Z_m (tests/test_oracle_model.py).
"""
from __future__ import annotations

import numpy as np

CP_CM2 = 9.8e-24          # photoelectric constant Cp (Sec. II-B)
M_EXP = 3.8               # exponent m of Z (Sec. II-B)
N_EXP = 3.2               # exponent n of E (Sec. II-B)
R0_CM = 2.818e-13         # classical electron radius r0 as printed (Sec. II-B)
MEC2_KEV = 510.975        # electron rest energy in gamma = E / 510.975 keV (Sec. II-B)
BARN_CM2 = 1e-24
N_W = 3.3428e23           # electrons / cm^3 of water (normalisation, not in the paper)
Z_W = 7.45                # effective Z of water (normalisation of Z^m)
S_MM = N_W * BARN_CM2 * 0.1   # 1/mm per barn: mu[1/mm] = S_MM * mu_hat
CP_BARN = CP_CM2 / BARN_CM2   # 9.8 barn keV^n
ZW_M = Z_W ** M_EXP           # Z_w^m = 2061.5...
E1_KEV = 50.0             # synthesis energy E1 (Sec. II-A, photoelectric dominant)
E2_KEV = 200.0            # synthesis energy E2 (Sec. II-A, Compton dominant)


def klein_nishina_barn(E_kev):
    """Total Klein-Nishina cross-section per electron, in barn (Sec. II-B).

    KN(g) = C0 { (1+g)/g^2 [2(1+g)/(1+2g) - ln(1+2g)/g] + ln(1+2g)/(2g)
                 - (1+3g)/(1+2g)^2 },  g = E / 510.975 keV, C0 = 2 pi r0^2.
    """
    g = np.asarray(E_kev, dtype=np.float64) / MEC2_KEV
    c0 = 2.0 * np.pi * R0_CM ** 2 / BARN_CM2
    l = np.log1p(2.0 * g)
    t1 = (1.0 + g) / g ** 2 * (2.0 * (1.0 + g) / (1.0 + 2.0 * g) - l / g)
    t2 = l / (2.0 * g)
    t3 = (1.0 + 3.0 * g) / (1.0 + 2.0 * g) ** 2
    return c0 * (t1 + t2 - t3)


def photo_coeff(E_kev):
    """P(E) = Cp' Z_w^m / E^n [barn]: photoelectric term per unit z = Z^m/Z_w^m."""
    return CP_BARN * ZW_M / np.asarray(E_kev, dtype=np.float64) ** N_EXP


def mu_hat(rhoe, Z, E_kev):
    """Normalised linear attenuation rho_e (Cp' Z^m/E^n + KN(E)) (eq. mac_E1_eff)."""
    Z = np.asarray(Z, dtype=np.float64)
    return np.asarray(rhoe, dtype=np.float64) * (CP_BARN * Z ** M_EXP / np.asarray(E_kev, dtype=np.float64) ** N_EXP
                                                 + klein_nishina_barn(E_kev))


def mu_mm(rhoe, Z, E_kev):
    """Linear attenuation in 1/mm."""
    return S_MM * mu_hat(rhoe, Z, E_kev)


# ----------------------------------------------------------------------------
# Spectra (acquisition model; not in the paper, which works on reconstructed
# images).  Kramers' law for the emitted photon number per keV, filtered by the
# same attenuation model, detected by a photon-counting detector.
# ----------------------------------------------------------------------------

def spectrum_bins(spec) -> tuple[np.ndarray, np.ndarray]:
    """(energies keV, normalised detected weights) of one arm.

    spec.kind == 'mono': a single bin at spec.kev.
    spec.kind == 'kramers': 1 keV bins E = 10, 11, ..., kvp-1 keV, emitted
    Phi(E) proportional to (kvp - E)/E, times exp(-mu(E) t) of each filter.
    """
    if spec.kind == "mono":
        return np.array([float(spec.kev)]), np.array([1.0])
    E = np.arange(10.0, float(spec.kvp), 1.0)
    phi = (spec.kvp - E) / E
    for (_, fz, frho, t_mm) in spec.filters:
        phi = phi * np.exp(-mu_mm(frho, fz, E) * t_mm)
    return E, phi / phi.sum()


def effective(values_per_bin: np.ndarray, weights: np.ndarray) -> float:
    return float(np.sum(values_per_bin * weights))


class Tables:
    """Per-solve scalar tables (Algorithm 1 'Require' line).

    a[k][i]: mu_hat of basis k at the acquisition arm i in {L, H} (spectrum
             weighted for polyenergetic arms);
    b[k][j]: mu_hat of basis k at the synthesis energy E_j, j in {1, 2};
    P[j], psi[j]: photoelectric and Compton coefficients at E_j;
    r: (E1/E2)^n;
    c_f[k]: sum_i a[k][i]^2 + sum_j b[k][j]^2 (the f-update denominators);
    c_rho: psi1 r - psi2 = (psi1 E1^n - psi2 E2^n) / E2^n, the coefficient
           of eq. rho_e;
    a_w: m1 P2 - m2 P1 at water (m_j = P_j + psi_j), the coefficient of
         eq. Z_m at water.
    Reading R3: eq. rho_e is divided by its coefficient and eq. Z_m by its
    water coefficient a_w, so both surrogate data terms have unit weight at
    water, like the f terms (the paper introduces beta~ = tau beta for the
    scale of these substituted equations; with this normalisation tau = 1).
    """

    def __init__(self, low, high, basis=((13.0, 1.7), (7.45, 1.0)), e1=E1_KEV, e2=E2_KEV):
        self.basis = tuple(tuple(map(float, b)) for b in basis)
        self.e1, self.e2 = float(e1), float(e2)
        arms = []
        for spec in (low, high):
            E, w = spectrum_bins(spec)
            arms.append((E, w))
        self.arms = arms
        a = np.zeros((2, 2))
        b = np.zeros((2, 2))
        for k, (zk, rk) in enumerate(self.basis):
            for i, (E, w) in enumerate(arms):
                a[k, i] = effective(mu_hat(rk, zk, E), w)
            for j, Ej in enumerate((self.e1, self.e2)):
                b[k, j] = float(mu_hat(rk, zk, Ej))
        self.a = a
        self.b = b
        self.P = np.array([photo_coeff(self.e1), photo_coeff(self.e2)], dtype=np.float64)
        self.psi = np.array([klein_nishina_barn(self.e1), klein_nishina_barn(self.e2)], dtype=np.float64)
        self.r = (self.e1 / self.e2) ** N_EXP
        self.c_f = np.array([a[0] @ a[0] + b[0] @ b[0], a[1] @ a[1] + b[1] @ b[1]])
        self.c_rho = float(self.psi[0] * self.r - self.psi[1])
        mw1, mw2 = self.P[0] + self.psi[0], self.P[1] + self.psi[1]
        self.a_w = float(mw1 * self.P[1] - mw2 * self.P[0])


def rhoe_closed_form(m1, m2, tab: Tables):
    """eq. rho_e: rho_e = (m1 E1^n - m2 E2^n) / (psi1 E1^n - psi2 E2^n)
    = (m1 r - m2) / (psi1 r - psi2), r = (E1/E2)^n."""
    return (np.asarray(m1) * tab.r - np.asarray(m2)) / tab.c_rho


def z_coefficients(m1, m2, tab: Tables):
    """eq. Z_m in normalised form a z = b (reading R3):
    a = (m1 P2 - m2 P1) / a_w  (m1 P2 - m2 P1 = Cp Z_w^m (m1/E2^n - m2/E1^n)),
    b = (m2 psi1 - m1 psi2) / a_w."""
    m1 = np.asarray(m1, dtype=np.float64)
    m2 = np.asarray(m2, dtype=np.float64)
    a = (m1 * tab.P[1] - m2 * tab.P[0]) / tab.a_w
    b = (m2 * tab.psi[0] - m1 * tab.psi[1]) / tab.a_w
    return a, b


def z_from_ztilde(zt):
    """Z = Z_w z^(1/m) (Z is the m-th root of Z^m, Sec. II-D); Z = 1 where z <= 0
    (reading R10)."""
    zt = np.asarray(zt, dtype=np.float64)
    out = np.ones_like(zt)
    pos = zt > 0
    out[pos] = Z_W * zt[pos] ** (1.0 / M_EXP)
    return out


def ztilde_from_z(Z):
    return (np.asarray(Z, dtype=np.float64) / Z_W) ** M_EXP
