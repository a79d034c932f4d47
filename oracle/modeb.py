"""Sinogram-domain data fidelity for the f-updates of Algorithm 1 (FP64 oracle;
test infrastructure only).

The paper fits its maps to reconstructed image pairs (Sec. III).  With the
sinograms s_L, s_H themselves as data, the basis-fidelity terms of eq.
obj_unconstraint become, for each acquired arm i in {L, H},

    (1 / gamma) || A (f1 a_1i + f2 a_2i) - s_i / S ||^2,

with A the ray-driven projector of oracle/ct.py (line integrals in mm),
S the water electron density in 1/mm (reading R2), so that s_i / S is in the
units of mu_hat, and gamma = ||A 1||^2 / n_pixels (reading R17: the data term
then weighs a constant image as the image-domain term does).  The
model-consistency terms at E1, E2, the L0 relaxation and the rho_e and Z^m
steps are unchanged.  The f_k update (Jacobi, reading R1: f_o at iterate k)
minimises

    sum_i (1/gamma) ||A(f_k a_ki + f_o a_oi) - s_i/S||^2
      + sum_j ||f_k b_kj + f_o b_oj - rho_e (P_j z + psi_j)||^2
      + beta ||grad f_k - (h, v)_k||^2,

whose normal equations are

    [alpha_k A^T A / gamma + c'_k + beta (dx^T dx + dy^T dy)] f_k
        = t_k - (sum_i a_ki a_oi / gamma) A^T A f_o
          + sum_j b_kj (rho_e (P_j z + psi_j) - f_o b_oj) + beta (dx^T h + dy^T v),

alpha_k = sum_i a_ki^2, c'_k = sum_j b_kj^2, t_k = A^T (sum_i a_ki s_i / S) / gamma.
The oracle solves them by conjugate gradients, preconditioned by the FFT
solve (alpha_k + c'_k + beta K)^-1, to a relative residual of 1e-12 (dense
solve on tiny grids in the tests).  A and A^T are applied as one sparse
matrix per geometry holding the Joseph weights of oracle/ct.py.  The solve
starts from the FBP image pair as in the image-domain mode.

Pins (tests/test_oracle_modeb.py): the sparse matrix reproduces ct.project
and ct.backproject; the normal operator is symmetric positive
definite (adjoint identity of A); the CG solve equals a dense solve of the
same system and minimises the f_k sub-objective under random perturbations;
a uniform material with consistent noiseless data is a fixed point of a
whole iteration.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import alg1, ct, model

_matrices = {}


def matrix(geom):
    """A as a sparse (rays x pixels) matrix of the Joseph weights of
    oracle/ct.py (repeated (ray, pixel) pairs summed), cached per geometry."""
    key = tuple(sorted((k, float(v)) for k, v in geom.items()))
    if key not in _matrices:
        rows, cols, vals = [], [], []
        for ray, pix, w in ct._joseph_samples(geom):
            rows.append(ray)
            cols.append(pix)
            vals.append(w)
        shape = (geom["n_views"] * geom["n_bins"], geom["nx"] * geom["ny"])
        A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=shape)
        A.sum_duplicates()
        _matrices[key] = A
    return _matrices[key]


def project(x, geom):
    return (matrix(geom) @ np.asarray(x, np.float64).ravel()).reshape(geom["n_views"], geom["n_bins"])


def backproject(y, geom):
    return (matrix(geom).T @ np.asarray(y, np.float64).ravel()).reshape(geom["ny"], geom["nx"])


def gamma(geom):
    """||A 1||^2 / n_pixels (reading R17)."""
    ones = np.ones((geom["ny"], geom["nx"]))
    p = project(ones, geom)
    return float(np.sum(p * p) / ones.size)


def data_images(sL, sH, geom, tab, g):
    """t_k = A^T (sum_i a_ki s_i / S) / gamma, k = 0, 1."""
    hL = np.asarray(sL, np.float64) / model.S_MM
    hH = np.asarray(sH, np.float64) / model.S_MM
    return [backproject(tab.a[k, 0] * hL + tab.a[k, 1] * hH, geom) / g for k in (0, 1)]


def coefficients(k, tab):
    """(alpha_k, c'_k, cross) of the f_k normal equations."""
    alpha = tab.a[k, 0] ** 2 + tab.a[k, 1] ** 2
    cp = tab.b[k, 0] ** 2 + tab.b[k, 1] ** 2
    cross = tab.a[0, 0] * tab.a[1, 0] + tab.a[0, 1] * tab.a[1, 1]
    return alpha, cp, cross


def normal_op(x, k, beta, geom, tab, g):
    """[alpha_k A^T A / gamma + c'_k + beta (dx^T dx + dy^T dy)] x."""
    alpha, cp, _ = coefficients(k, tab)
    return alpha * backproject(project(x, geom), geom) / g + cp * x + beta * alg1.laplacian(x)


def rhs(k, st, hv, beta, t, geom, tab, g):
    """Right-hand side of the f_k normal equations (f_o, rho_e, z at iterate k)."""
    o = 1 - k
    fo = st["f2"] if k == 0 else st["f1"]
    cross = tab.a[k, 0] * tab.a[o, 0] + tab.a[k, 1] * tab.a[o, 1]
    M1, M2 = alg1.model_eval(st["rhoe"], st["zt"], tab)
    mod = tab.b[k, 0] * (M1 - fo * tab.b[o, 0]) + tab.b[k, 1] * (M2 - fo * tab.b[o, 1])
    h, v = hv
    return t[k] - cross * backproject(project(fo, geom), geom) / g + mod + beta * alg1.adjoint_diff(h, v)


def f_solve(b, k, beta, geom, tab, g, x0, tol=1e-12, max_iter=2000):
    """Preconditioned conjugate gradients on the f_k normal equations from
    x0, preconditioner (alpha_k + c'_k + beta K)^-1 by FFT, stopping at
    ||r|| <= tol ||b||."""
    alpha, cp, _ = coefficients(k, tab)
    x = np.array(x0, dtype=np.float64)
    r = b - normal_op(x, k, beta, geom, tab, g)
    bb = float(np.sum(b * b))
    if bb == 0.0:
        return np.zeros_like(x)
    y = alg1.fft_solve(r, alpha + cp, beta)
    p = y.copy()
    ry = float(np.sum(r * y))
    for _ in range(max_iter):
        if float(np.sum(r * r)) <= tol * tol * bb:
            break
        q = normal_op(p, k, beta, geom, tab, g)
        a = ry / float(np.sum(p * q))
        x += a * p
        r -= a * q
        y = alg1.fft_solve(r, alpha + cp, beta)
        ry_new = float(np.sum(r * y))
        p = y + (ry_new / ry) * p
        ry = ry_new
    return x


def iterate(st, beta, beta_t, lam, t, geom, tab, g, z_method="sparse", decision_dtype=np.float64):
    """One pass of Algorithm 1 with the sinogram-domain f-updates."""
    hv = alg1.thresholds(st, lam / beta, decision_dtype)
    f1 = f_solve(rhs(0, st, hv["f1"], beta, t, geom, tab, g), 0, beta, geom, tab, g, st["f1"])
    f2 = f_solve(rhs(1, st, hv["f2"], beta, t, geom, tab, g), 1, beta, geom, tab, g, st["f2"])
    m1, m2 = alg1.synthesize(f1, f2, tab)
    rhoe = alg1.fft_solve(alg1.rhs_rho(m1, m2, hv["rhoe"], beta_t, tab), 1.0, beta_t)
    a2, rz = alg1.z_terms(m1, m2, hv["zt"], beta_t, tab)
    zt = alg1.z_solve(a2, rz, beta_t, z_method)
    return dict(f1=f1, f2=f2, rhoe=rhoe, zt=zt), hv


def solve(sL, sH, geom, tab, prm: alg1.Params, st0=None):
    """Algorithm 1 with sinogram-domain f-updates.  Starts from the FBP image
    pair (or from ``st0``); returns the final state with Z."""
    g = gamma(geom)
    t = data_images(sL, sH, geom, tab, g)
    if st0 is None:
        muL = ct.fbp(sL, geom) / model.S_MM
        muH = ct.fbp(sH, geom) / model.S_MM
        st = alg1.init_state(muL, muH, tab, prm.z_clip, prm.rho_air)
    else:
        st = dict(st0)
    beta = prm.beta0
    kappa = prm.kappa_value()
    for _ in range(prm.iters):
        st, _hv = iterate(st, beta, prm.tau * beta, prm.lam, t, geom, tab, g, prm.z_method, prm.decision_dtype)
        beta = kappa * beta
    st["Z"] = model.z_from_ztilde(st["zt"])
    return st


def sub_objective(fk, k, st, hv_k, beta, sL, sH, geom, tab, g):
    """The f_k sub-objective as written in the module docstring."""
    o = 1 - k
    fo = st["f2"] if k == 0 else st["f1"]
    val = 0.0
    for i, s in enumerate((sL, sH)):
        d = ct.project(fk * tab.a[k, i] + fo * tab.a[o, i], geom) - np.asarray(s, np.float64) / model.S_MM
        val += float(np.sum(d * d)) / g
    M = alg1.model_eval(st["rhoe"], st["zt"], tab)
    for j in (0, 1):
        d = fk * tab.b[k, j] + fo * tab.b[o, j] - M[j]
        val += float(np.sum(d * d))
    dx, dy = alg1.forward_diff(fk)
    h, v = hv_k
    return val + beta * float(np.sum((dx - h) ** 2) + np.sum((dy - v) ** 2))
