"""Algorithm 1 of Sec. II-D in FP64 (oracle; test infrastructure only).

State: basis fractions f1, f2, relative electron density rho_e and the
normalised photoelectric variable z = Z^m / Z_w^m, each an (ny, nx) array.
Differences are periodic forward differences (reading R6): for a map g,

    dx g(j, i) = g(j, i+1) - g(j, i),     dy g(j, i) = g(j+1, i) - g(j, i)

(indices modulo the grid), and their adjoints dx^T h(j,i) = h(j,i-1) - h(j,i),
dy^T v(j,i) = v(j-1,i) - v(j,i).  With these the FFT diagonalisations of
Sec. II-C/II-D are exact: |F dx|^2 = 4 sin^2(pi kx / nx), and "F(1)" is 1
(reading R4).

One iteration (readings R1, R3, R5):
  1. (h_g, v_g) = threshold of (dx g, dy g) at lambda/beta for all four maps
     (eq. sol_hv; a tie goes to zero, reading R7).
  2. f1, f2 by their FFT-diagonalised closed forms, each using the other's
     iterate-k value and the iterate-k model rho_e (P_j z + psi_j) (Alg. 1).
  3. mu_hat(E_j)^(k+1) = f1 b_1j + f2 b_2j from the NEW fractions f^(k+1)
     (eq. mac_E1/E2; reading R1: the printed superscripts of this line and of
     the rho_e and Z^m lines are read as k+1.  Taking them from iterate k
     instead makes the zero-frequency mode, which the regulariser cannot
     damp, grow by a factor 1.62 per iteration.)
  4. rho_e from eq. obj_sub_rho divided by its coefficient (reading R3):
     min ||rho_e - rho_cf(m)||^2 + beta~ ||d rho_e - (h, v)||^2, with
     rho_cf the closed form of eq. rho_e, FFT-diagonalised.
  5. z from eq. obj_sub_z (divided by its water coefficient, reading R3) as
     the normal equations
     [diag(a^2) + beta~ (dx^T dx + dy^T dy)] z = a b + beta~ (dx^T h + dy^T v)
     solved exactly (sparse LU; dense LU on small grids).
  6. beta <- kappa beta, beta~ = tau beta.

Pins (tests/test_oracle_alg1.py): threshold = brute-force per-pixel minimiser
of E(r); FFT solve = dense solve of the same periodic system; z solve = FFT
solve when a^2 is constant, and = dense solve; every block update is the
minimiser of its own subproblem (eq. obj_sub_f / rho / z) under random
perturbations; a uniform material is a fixed point; noiseless uniform inputs
recover (Z, rho_e) exactly.  The relaxed objective (eq. obj_unconstraint) is
pinned to hand-computed values on 3 x 3 grids, to zero at an exact uniform
material, and its f part to eq. obj_sub_f (tests/test_oracle_objective.py).  The full multi-iteration trajectory on noisy
data has no independent pin beyond these (parity unpinned for whole runs).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import model


# ----------------------------------------------------------------------------
# Difference operators (periodic), reading R6
# ----------------------------------------------------------------------------

def forward_diff(g):
    """(dx g, dy g) with periodic wrap."""
    return np.roll(g, -1, axis=1) - g, np.roll(g, -1, axis=0) - g


def adjoint_diff(h, v):
    """dx^T h + dy^T v (the adjoint of forward_diff)."""
    return (np.roll(h, 1, axis=1) - h) + (np.roll(v, 1, axis=0) - v)


def laplacian(g):
    """(dx^T dx + dy^T dy) g, the periodic 5-point operator."""
    return adjoint_diff(*forward_diff(g))


# ----------------------------------------------------------------------------
# Auxiliary-variable subproblem, eq. sol_hv
# ----------------------------------------------------------------------------

def hard_threshold(g, lam_over_beta, dtype=np.float64):
    """(h, v) = (0, 0) where (dx g)^2 + (dy g)^2 <= lambda/beta, else (dx g, dy g).

    ``dtype`` is the precision in which the keep/zero decision is taken.  The
    definition is FP64; with float32 the differences, squares, their sum and
    the threshold are each rounded to float32 in that order (no fused
    multiply-add), which is how the FP32 kernel takes the same decision.
    """
    if dtype == np.float64:
        dx, dy = forward_diff(np.asarray(g, dtype=np.float64))
        keep = dx * dx + dy * dy > lam_over_beta
        return np.where(keep, dx, 0.0), np.where(keep, dy, 0.0), keep
    g32 = np.asarray(g, dtype=np.float32)
    dx = (np.roll(g32, -1, axis=1) - g32).astype(np.float32)
    dy = (np.roll(g32, -1, axis=0) - g32).astype(np.float32)
    s = (dx * dx).astype(np.float32) + (dy * dy).astype(np.float32)
    keep = s.astype(np.float32) > np.float32(lam_over_beta)
    return (np.where(keep, dx, 0).astype(np.float64), np.where(keep, dy, 0).astype(np.float64), keep)


def count_nonzero_gradients(h, v):
    """C(h, v) = #{r : |h(r)| + |v(r)| != 0} (Sec. II-C)."""
    return int(np.count_nonzero((np.abs(h) + np.abs(v)) != 0))


# ----------------------------------------------------------------------------
# Quadratic subproblems
# ----------------------------------------------------------------------------

def spectral_symbol(ny, nx):
    """|F dx|^2 + |F dy|^2 on the (ny, nx) frequency grid."""
    kx = np.arange(nx)
    ky = np.arange(ny)
    sx = 4.0 * np.sin(np.pi * kx / nx) ** 2
    sy = 4.0 * np.sin(np.pi * ky / ny) ** 2
    return sy[:, None] + sx[None, :]


def fft_solve(rhs, c, beta):
    """g = F^-1[ F(rhs) / (c + beta (|F dx|^2 + |F dy|^2)) ] (Sec. II-C, II-D).

    ``rhs`` already holds the data part plus beta (dx^T h + dy^T v); this is
    the closed form of the f1, f2 and rho_e updates of Algorithm 1 with F
    linear.  Requires c > 0 (or c = 0 with a zero-mean right-hand side).
    """
    ny, nx = rhs.shape
    den = c + beta * spectral_symbol(ny, nx)
    return np.real(np.fft.ifft2(np.fft.fft2(rhs) / den))


def periodic_diff_matrices(ny, nx):
    """Sparse Dx, Dy (row-major pixel index j*nx + i) built from cyclic shifts."""
    def d1(n):
        rows = np.arange(n)
        shift = sp.csr_matrix((np.ones(n), (rows, (rows + 1) % n)), shape=(n, n))
        return shift - sp.identity(n, format="csr")
    Dx = sp.kron(sp.identity(ny), d1(nx), format="csr")
    Dy = sp.kron(d1(ny), sp.identity(nx), format="csr")
    return Dx, Dy


def z_system(a2, beta_t):
    """Sparse matrix diag(a^2) + beta~ (Dx^T Dx + Dy^T Dy) (reading R5)."""
    ny, nx = a2.shape
    Dx, Dy = periodic_diff_matrices(ny, nx)
    L = (Dx.T @ Dx + Dy.T @ Dy)
    return (sp.diags(a2.ravel()) + beta_t * L).tocsc()


def z_solve(a2, rhs, beta_t, method="sparse"):
    """Exact solution of [diag(a^2) + beta~ L] z = rhs (Alg. 1, Z^m step)."""
    ny, nx = a2.shape
    M = z_system(a2, beta_t)
    if method == "dense":
        return np.linalg.solve(M.toarray(), rhs.ravel()).reshape(ny, nx)
    return spla.spsolve(M, rhs.ravel()).reshape(ny, nx)


# ----------------------------------------------------------------------------
# Algorithm 1
# ----------------------------------------------------------------------------

@dataclass
class Params:
    """Parameters of Algorithm 1 (none are printed in the paper; reading R8)."""

    lam: float = 1e-2
    beta0: float = 2e-2
    beta_max: float = 1e5
    tau: float = 1.0
    iters: int = 50
    kappa: float | None = None      # default: (beta_max/beta0)^(1/iters)
    order: str = "jacobi"          # reading R1; 'gauss-seidel' is the variant
    z_clip: tuple = (0.0, 30.0)    # Z range of the initial z (reading R16)
    rho_air: float = 0.1           # initial z = 1 (water) where rho_e^(0) < rho_air (R16)
    z_method: str = "sparse"
    decision_dtype: type = np.float64

    def kappa_value(self):
        if self.kappa is not None:
            return float(self.kappa)
        return float((self.beta_max / self.beta0) ** (1.0 / self.iters))


def synthesize(f1, f2, tab):
    """mu_hat(E_j) = f1 b_1j + f2 b_2j, j = 1, 2 (eq. mac_E1, mac_E2)."""
    return f1 * tab.b[0, 0] + f2 * tab.b[1, 0], f1 * tab.b[0, 1] + f2 * tab.b[1, 1]


def model_eval(rhoe, zt, tab):
    """rho_e (P_j z + psi_j), j = 1, 2 (eq. mac_E1_eff, mac_E2_eff)."""
    return rhoe * (tab.P[0] * zt + tab.psi[0]), rhoe * (tab.P[1] * zt + tab.psi[1])


def init_state(muL, muH, tab, z_clip=(0.0, 30.0), rho_air=0.1):
    """Initialisation of Algorithm 1 from normalised images mu_hat(E_L), mu_hat(E_H).

    f by Cramer's rule on eq. lac_EL/EH; mu_hat(E_j) by eq. mac_E1/E2; rho_e
    and z by eq. rho_e / eq. Z_m.  Reading R16: z = b/a is clipped to the Z
    range ``z_clip``, and set to 1 (water) where a = 0 or rho_e^(0) < rho_air:
    in air b/a is a ratio of two noise values, and a large z there makes the
    photoelectric term dominate the model and destabilises the iteration.
    """
    a = tab.a
    det = a[0, 0] * a[1, 1] - a[0, 1] * a[1, 0]
    f1 = (a[1, 1] * muL - a[1, 0] * muH) / det
    f2 = (a[0, 0] * muH - a[0, 1] * muL) / det
    m1, m2 = synthesize(f1, f2, tab)
    rhoe = model.rhoe_closed_form(m1, m2, tab)
    ca, cb = model.z_coefficients(m1, m2, tab)
    zt = cb / np.where(ca != 0.0, ca, 1.0)
    zt = np.clip(zt, model.ztilde_from_z(z_clip[0]) if z_clip[0] > 0 else 0.0,
                 model.ztilde_from_z(z_clip[1]))
    zt = np.where((ca != 0.0) & (rhoe >= rho_air), zt, 1.0)
    return dict(f1=f1, f2=f2, rhoe=rhoe, zt=zt)


def rhs_f(which, st, hv, beta, muL, muH, tab):
    """Right-hand side of the f_which update (Alg. 1) in the pixel domain:

    sum_i mu_k(E_i)(mu(E_i) - f_o mu_o(E_i))
      + sum_j b_kj (rho_e (P_j z + psi_j) - f_o b_oj) + beta (dx^T h + dy^T v),
    with k = which and o the other basis.
    """
    k, o = (0, 1) if which == 0 else (1, 0)
    fo = st["f2"] if which == 0 else st["f1"]
    M1, M2 = model_eval(st["rhoe"], st["zt"], tab)
    data = (tab.a[k, 0] * (muL - fo * tab.a[o, 0]) + tab.a[k, 1] * (muH - fo * tab.a[o, 1])
            + tab.b[k, 0] * (M1 - fo * tab.b[o, 0]) + tab.b[k, 1] * (M2 - fo * tab.b[o, 1]))
    h, v = hv
    return data + beta * adjoint_diff(h, v)


def rhs_rho(m1, m2, hv, beta_t, tab):
    """rho_cf(m) + beta~ (dx^T h + dy^T v) (eq. obj_sub_rho, reading R3)."""
    h, v = hv
    return model.rhoe_closed_form(m1, m2, tab) + beta_t * adjoint_diff(h, v)


def z_terms(m1, m2, hv, beta_t, tab):
    """(a^2, a b + beta~ (dx^T h + dy^T v)) of the Z^m step (reading R5)."""
    a, b = model.z_coefficients(m1, m2, tab)
    h, v = hv
    return a * a, a * b + beta_t * adjoint_diff(h, v)


def thresholds(st, lam_over_beta, dtype=np.float64):
    out = {}
    for g in ("f1", "f2", "rhoe", "zt"):
        h, v, keep = hard_threshold(st[g], lam_over_beta, dtype)
        out[g] = (h, v)
    return out


def iterate(st, beta, beta_t, lam, muL, muH, tab, order="jacobi", z_method="sparse",
            decision_dtype=np.float64):
    """One pass of the repeat-body of Algorithm 1; returns (new state, hv)."""
    hv = thresholds(st, lam / beta, decision_dtype)
    f1 = fft_solve(rhs_f(0, st, hv["f1"], beta, muL, muH, tab), tab.c_f[0], beta)
    st_f2 = dict(st, f1=f1) if order == "gauss-seidel" else st
    f2 = fft_solve(rhs_f(1, st_f2, hv["f2"], beta, muL, muH, tab), tab.c_f[1], beta)
    m1, m2 = synthesize(f1, f2, tab)
    rhoe = fft_solve(rhs_rho(m1, m2, hv["rhoe"], beta_t, tab), 1.0, beta_t)
    a2, rz = z_terms(m1, m2, hv["zt"], beta_t, tab)
    zt = z_solve(a2, rz, beta_t, z_method)
    return dict(f1=f1, f2=f2, rhoe=rhoe, zt=zt), hv


def objective(st, hv, beta, lam, muL, muH, tab):
    """Relaxed objective eq. obj_unconstraint, term by term (FP64)."""
    f1, f2 = st["f1"], st["f2"]
    dL = f1 * tab.a[0, 0] + f2 * tab.a[1, 0] - muL
    dH = f1 * tab.a[0, 1] + f2 * tab.a[1, 1] - muH
    M1, M2 = model_eval(st["rhoe"], st["zt"], tab)
    m1, m2 = synthesize(f1, f2, tab)
    rel = 0.0
    nnz = 0
    for g in ("f1", "f2", "rhoe", "zt"):
        dx, dy = forward_diff(st[g])
        h, v = hv[g]
        rel += np.sum((dx - h) ** 2) + np.sum((dy - v) ** 2)
        nnz += count_nonzero_gradients(h, v)
    terms = dict(fid_L=float(np.sum(dL ** 2)), fid_H=float(np.sum(dH ** 2)),
                 mod_1=float(np.sum((M1 - m1) ** 2)), mod_2=float(np.sum((M2 - m2) ** 2)),
                 relax=float(beta * rel), l0=float(lam * nnz), nnz=nnz)
    terms["total"] = (terms["fid_L"] + terms["fid_H"] + terms["mod_1"] + terms["mod_2"]
                      + terms["relax"] + terms["l0"])
    return terms


def solve(muL, muH, tab, prm: Params, trace=False):
    """Algorithm 1: initialise, then ``prm.iters`` iterations (reading R8:
    kappa = (beta_max/beta0)^(1/iters) so that beta reaches beta_max exactly at
    the last iteration).  Inputs are normalised images mu / S."""
    st = init_state(muL, muH, tab, prm.z_clip, prm.rho_air)
    beta = prm.beta0
    kappa = prm.kappa_value()
    tr = []
    for k in range(prm.iters):
        beta_t = prm.tau * beta
        st_new, hv = iterate(st, beta, beta_t, prm.lam, muL, muH, tab, prm.order, prm.z_method,
                             prm.decision_dtype)
        if trace:
            tr.append(dict(k=k, beta=beta, **objective(st_new, hv, beta, prm.lam, muL, muH, tab)))
        st = st_new
        beta = kappa * beta
    st["Z"] = model.z_from_ztilde(st["zt"])
    if trace:
        st["trace"] = tr
    return st


def solve_mm(muL_mm, muH_mm, tab, prm: Params, trace=False):
    """Algorithm 1 on images in 1/mm (divides by S, reading R2)."""
    return solve(np.asarray(muL_mm, np.float64) / model.S_MM, np.asarray(muH_mm, np.float64) / model.S_MM,
                 tab, prm, trace)


# ----------------------------------------------------------------------------
# Subproblem objectives as printed (used to pin the block updates)
# ----------------------------------------------------------------------------

def sub_objective_f(f1, f2, st, hv_f1, hv_f2, beta, muL, muH, tab):
    """eq. obj_sub_f with rho_e, z held at st's values."""
    M1, M2 = model_eval(st["rhoe"], st["zt"], tab)
    m1, m2 = synthesize(f1, f2, tab)
    J = (np.sum((f1 * tab.a[0, 0] + f2 * tab.a[1, 0] - muL) ** 2)
         + np.sum((f1 * tab.a[0, 1] + f2 * tab.a[1, 1] - muH) ** 2)
         + np.sum((m1 - M1) ** 2) + np.sum((m2 - M2) ** 2))
    for g, (h, v) in ((f1, hv_f1), (f2, hv_f2)):
        dx, dy = forward_diff(g)
        J += beta * (np.sum((dx - h) ** 2) + np.sum((dy - v) ** 2))
    return float(J)


def sub_objective_rho(rhoe, m1, m2, hv, beta_t, tab):
    """eq. obj_sub_rho divided by (psi1 E1^n - psi2 E2^n) (reading R3)."""
    dx, dy = forward_diff(rhoe)
    h, v = hv
    cE = tab.c_rho
    return float(np.sum(((cE * rhoe - (m1 * tab.r - m2)) / cE) ** 2)
                 + beta_t * (np.sum((dx - h) ** 2) + np.sum((dy - v) ** 2)))


def sub_objective_z(zt, m1, m2, hv, beta_t, tab):
    """eq. obj_sub_z in the normalised variable z (reading R3)."""
    a, b = model.z_coefficients(m1, m2, tab)
    dx, dy = forward_diff(zt)
    h, v = hv
    return float(np.sum((a * zt - b) ** 2) + beta_t * (np.sum((dx - h) ** 2) + np.sum((dy - v) ** 2)))
