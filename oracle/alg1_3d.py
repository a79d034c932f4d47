"""Algorithm 1 of Sec. II-D with 3-D multi-domain regularisation, in FP64
(oracle; test infrastructure only).

The paper regularises each slice in 2-D: the gradient of a map is (dx g, dy g)
and the L0 term counts the pixels where the auxiliary pair (h, v) is nonzero
(Sec. II-C, eq. sol_hv).  A volume of slices adds the difference across
slices.  This module is that extension, with the readings:

  R22  dz is the periodic forward difference across the slices of the volume,
       dz g(k, j, i) = g(k+1, j, i) - g(k, j, i) (k modulo the slice count), of
       unit weight like dx and dy.  Periodic for the same reason as reading
       R6: it makes the FFT diagonalisation of the f and rho_e updates exact
       (|F dz|^2 = 4 sin^2(pi kz / nz)).  A single slice has dz = 0, so the
       volume form reduces to the 2-D algorithm slice by slice.
  R23  The auxiliary variable of a map is the triple (h, v, w) for
       (dx g, dy g, dz g), kept or zeroed as a whole: the L0 term counts the
       voxels where any of the three is nonzero, and the minimiser of
       beta |grad g - (h, v, w)|^2 + lambda [(h, v, w) != 0] keeps the triple
       where |grad g|^2 > lambda / beta (a tie goes to zero, reading R7).

Everything pointwise (the model tables, the initialisation, the data terms of
each block) is the 2-D oracle's, applied to (nz, ny, nx) arrays.  One
iteration, in the order of Algorithm 1:
  1. (h, v, w) of the four maps by the 3-D threshold at lambda / beta;
  2. f1, f2 by F^-1[F(rhs) / (c + beta (|F dx|^2 + |F dy|^2 + |F dz|^2))],
     rhs = data + beta (dx^T h + dy^T v + dz^T w);
  3. mu_hat(E_j)^(k+1) from the new f (reading R1);
  4. rho_e by the same closed form with c = 1 and beta~;
  5. z from [diag(a^2) + beta~ (dx^T dx + dy^T dy + dz^T dz)] z
     = a b + beta~ (dx^T h + dy^T v + dz^T w), solved exactly;
  6. beta <- kappa beta.

Pins (tests/test_oracle_alg1_3d.py): one slice equals the 2-D oracle; a
volume of identical slices gives the 2-D solution on every slice; the
threshold equals a brute-force minimiser of its per-voxel energy; the FFT
solve equals a dense solve of a Kronecker-assembled system; the sparse Z^m
matrix equals diag(a^2) plus a roll-based 7-point stencil and its solve a
dense solve; each block update minimises its own subproblem under
perturbations; a uniform material is a fixed point.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import alg1, model


# ----------------------------------------------------------------------------
# Difference operators (periodic in x, y and across slices), readings R6, R22
# ----------------------------------------------------------------------------

def forward_diff3(g):
    """(dx g, dy g, dz g) of an (nz, ny, nx) array with periodic wrap."""
    return np.roll(g, -1, axis=2) - g, np.roll(g, -1, axis=1) - g, np.roll(g, -1, axis=0) - g


def adjoint_diff3(h, v, w):
    """dx^T h + dy^T v + dz^T w (the adjoint of forward_diff3)."""
    return (np.roll(h, 1, axis=2) - h) + (np.roll(v, 1, axis=1) - v) + (np.roll(w, 1, axis=0) - w)


def laplacian3(g):
    """(dx^T dx + dy^T dy + dz^T dz) g, the periodic 7-point operator."""
    return adjoint_diff3(*forward_diff3(g))


# ----------------------------------------------------------------------------
# Auxiliary-variable subproblem, eq. sol_hv with a third component (R23)
# ----------------------------------------------------------------------------

def hard_threshold3(g, lam_over_beta):
    """(h, v, w) = grad g where |grad g|^2 > lambda/beta, else (0, 0, 0)."""
    dx, dy, dz = forward_diff3(np.asarray(g, dtype=np.float64))
    keep = dx * dx + dy * dy + dz * dz > lam_over_beta
    return np.where(keep, dx, 0.0), np.where(keep, dy, 0.0), np.where(keep, dz, 0.0), keep


def count_nonzero_gradients3(h, v, w):
    """C(h, v, w) = #{r : |h(r)| + |v(r)| + |w(r)| != 0}."""
    return int(np.count_nonzero((np.abs(h) + np.abs(v) + np.abs(w)) != 0))


# ----------------------------------------------------------------------------
# Quadratic subproblems
# ----------------------------------------------------------------------------

def spectral_symbol3(nz, ny, nx):
    """|F dx|^2 + |F dy|^2 + |F dz|^2 on the (nz, ny, nx) frequency grid."""
    sx = 4.0 * np.sin(np.pi * np.arange(nx) / nx) ** 2
    sy = 4.0 * np.sin(np.pi * np.arange(ny) / ny) ** 2
    sz = 4.0 * np.sin(np.pi * np.arange(nz) / nz) ** 2
    return sz[:, None, None] + sy[None, :, None] + sx[None, None, :]


def fft_solve3(rhs, c, beta):
    """g = F^-1[F(rhs) / (c + beta (|F dx|^2 + |F dy|^2 + |F dz|^2))], the
    closed form of the f1, f2 and rho_e updates over a volume (F the 3-D
    DFT).  Requires c > 0 (or c = 0 with a zero-mean right-hand side)."""
    nz, ny, nx = rhs.shape
    den = c + beta * spectral_symbol3(nz, ny, nx)
    return np.real(np.fft.ifftn(np.fft.fftn(rhs) / den))


def periodic_diff_matrices3(nz, ny, nx):
    """Sparse Dx, Dy, Dz (voxel index (k ny + j) nx + i) from cyclic shifts."""
    def d1(n):
        rows = np.arange(n)
        shift = sp.csr_matrix((np.ones(n), (rows, (rows + 1) % n)), shape=(n, n))
        return shift - sp.identity(n, format="csr")
    Iz, Iy, Ix = sp.identity(nz), sp.identity(ny), sp.identity(nx)
    Dx = sp.kron(sp.kron(Iz, Iy), d1(nx), format="csr")
    Dy = sp.kron(sp.kron(Iz, d1(ny)), Ix, format="csr")
    Dz = sp.kron(sp.kron(d1(nz), Iy), Ix, format="csr")
    return Dx, Dy, Dz


def z_system3(a2, beta_t):
    """Sparse diag(a^2) + beta~ (Dx^T Dx + Dy^T Dy + Dz^T Dz)."""
    nz, ny, nx = a2.shape
    Dx, Dy, Dz = periodic_diff_matrices3(nz, ny, nx)
    L = Dx.T @ Dx + Dy.T @ Dy + Dz.T @ Dz
    return (sp.diags(a2.ravel()) + beta_t * L).tocsc()


def z_solve3(a2, rhs, beta_t, method="sparse"):
    """Exact solution of [diag(a^2) + beta~ L3] z = rhs (the Z^m step over a volume)."""
    M = z_system3(a2, beta_t)
    if method == "dense":
        return np.linalg.solve(M.toarray(), rhs.ravel()).reshape(a2.shape)
    return spla.spsolve(M, rhs.ravel()).reshape(a2.shape)


# ----------------------------------------------------------------------------
# Algorithm 1 over a volume
# ----------------------------------------------------------------------------

def thresholds3(st, lam_over_beta):
    out = {}
    for g in ("f1", "f2", "rhoe", "zt"):
        h, v, w, _ = hard_threshold3(st[g], lam_over_beta)
        out[g] = (h, v, w)
    return out


def rhs_f3(which, st, hvw, beta, muL, muH, tab):
    """Right-hand side of the f_which update: the 2-D oracle's data part
    (pointwise) plus beta (dx^T h + dy^T v + dz^T w)."""
    zero = np.zeros_like(muL)
    data = alg1.rhs_f(which, st, (zero, zero), beta, muL, muH, tab)
    return data + beta * adjoint_diff3(*hvw)


def rhs_rho3(m1, m2, hvw, beta_t, tab):
    """rho_cf(m) + beta~ (dx^T h + dy^T v + dz^T w)."""
    return model.rhoe_closed_form(m1, m2, tab) + beta_t * adjoint_diff3(*hvw)


def z_terms3(m1, m2, hvw, beta_t, tab):
    """(a^2, a b + beta~ (dx^T h + dy^T v + dz^T w)) of the Z^m step."""
    a, b = model.z_coefficients(m1, m2, tab)
    return a * a, a * b + beta_t * adjoint_diff3(*hvw)


def iterate3(st, beta, beta_t, lam, muL, muH, tab, order="jacobi", z_method="sparse"):
    """One pass of the repeat-body of Algorithm 1 over a volume; returns (new state, hvw)."""
    hvw = thresholds3(st, lam / beta)
    f1 = fft_solve3(rhs_f3(0, st, hvw["f1"], beta, muL, muH, tab), tab.c_f[0], beta)
    st_f2 = dict(st, f1=f1) if order == "gauss-seidel" else st
    f2 = fft_solve3(rhs_f3(1, st_f2, hvw["f2"], beta, muL, muH, tab), tab.c_f[1], beta)
    m1, m2 = alg1.synthesize(f1, f2, tab)
    rhoe = fft_solve3(rhs_rho3(m1, m2, hvw["rhoe"], beta_t, tab), 1.0, beta_t)
    a2, rz = z_terms3(m1, m2, hvw["zt"], beta_t, tab)
    zt = z_solve3(a2, rz, beta_t, z_method)
    return dict(f1=f1, f2=f2, rhoe=rhoe, zt=zt), hvw


def objective3(st, hvw, beta, lam, muL, muH, tab):
    """eq. obj_unconstraint over a volume: the data terms of the 2-D oracle
    plus beta |grad g - (h, v, w)|^2 and lambda C(h, v, w) for the four maps."""
    zero = np.zeros_like(muL)
    base = alg1.objective(st, {g: (zero, zero) for g in ("f1", "f2", "rhoe", "zt")}, beta, lam, muL, muH, tab)
    rel = 0.0
    nnz = 0
    for g in ("f1", "f2", "rhoe", "zt"):
        dx, dy, dz = forward_diff3(st[g])
        h, v, w = hvw[g]
        rel += np.sum((dx - h) ** 2) + np.sum((dy - v) ** 2) + np.sum((dz - w) ** 2)
        nnz += count_nonzero_gradients3(h, v, w)
    terms = dict(fid_L=base["fid_L"], fid_H=base["fid_H"], mod_1=base["mod_1"], mod_2=base["mod_2"],
                 relax=float(beta * rel), l0=float(lam * nnz), nnz=nnz)
    terms["total"] = (terms["fid_L"] + terms["fid_H"] + terms["mod_1"] + terms["mod_2"]
                      + terms["relax"] + terms["l0"])
    return terms


def solve3(muL, muH, tab, prm: alg1.Params):
    """Algorithm 1 over a volume of normalised images (nz, ny, nx): the 2-D
    initialisation (pointwise), then ``prm.iters`` iterations of iterate3 with
    the beta schedule of reading R8."""
    st = alg1.init_state(muL, muH, tab, prm.z_clip, prm.rho_air)
    beta = prm.beta0
    kappa = prm.kappa_value()
    for _ in range(prm.iters):
        st, _ = iterate3(st, beta, prm.tau * beta, prm.lam, muL, muH, tab, prm.order, prm.z_method)
        beta = kappa * beta
    st["Z"] = model.z_from_ztilde(st["zt"])
    return st


# ----------------------------------------------------------------------------
# Subproblem objectives (used to pin the block updates)
# ----------------------------------------------------------------------------

def sub_objective_f3(f1, f2, st, hvw_f1, hvw_f2, beta, muL, muH, tab):
    """eq. obj_sub_f over a volume with rho_e, z held at st's values."""
    zero = np.zeros_like(muL)
    J = alg1.sub_objective_f(f1, f2, st, (zero, zero), (zero, zero), 0.0, muL, muH, tab)
    for g, (h, v, w) in ((f1, hvw_f1), (f2, hvw_f2)):
        dx, dy, dz = forward_diff3(g)
        J += beta * (np.sum((dx - h) ** 2) + np.sum((dy - v) ** 2) + np.sum((dz - w) ** 2))
    return float(J)


def sub_objective_rho3(rhoe, m1, m2, hvw, beta_t, tab):
    """eq. obj_sub_rho over a volume, divided by its coefficient (reading R3)."""
    zero = np.zeros_like(rhoe)
    J = alg1.sub_objective_rho(rhoe, m1, m2, (zero, zero), 0.0, tab)
    dx, dy, dz = forward_diff3(rhoe)
    h, v, w = hvw
    return float(J + beta_t * (np.sum((dx - h) ** 2) + np.sum((dy - v) ** 2) + np.sum((dz - w) ** 2)))


def sub_objective_z3(zt, m1, m2, hvw, beta_t, tab):
    """eq. obj_sub_z over a volume in the normalised variable z (reading R3)."""
    a, b = model.z_coefficients(m1, m2, tab)
    dx, dy, dz = forward_diff3(zt)
    h, v, w = hvw
    return float(np.sum((a * zt - b) ** 2)
                 + beta_t * (np.sum((dx - h) ** 2) + np.sum((dy - v) ** 2) + np.sum((dz - w) ** 2)))
