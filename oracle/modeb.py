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


def normal_op(x, k, beta, geom, tab, g, W=None):
    """[alpha_k A^T A / gamma + c'_k + beta (dx^T dx + dy^T dy)] x; with
    per-ray weights W (the Gauss-Newton mode) A^T diag(W) A / gamma in place
    of alpha_k A^T A / gamma."""
    alpha, cp, _ = coefficients(k, tab)
    if W is None:
        data = alpha * backproject(project(x, geom), geom) / g
    else:
        data = backproject(W * project(x, geom), geom) / g
    return data + cp * x + beta * alg1.laplacian(x)


def rhs(k, st, hv, beta, t, geom, tab, g):
    """Right-hand side of the f_k normal equations (f_o, rho_e, z at iterate k)."""
    o = 1 - k
    fo = st["f2"] if k == 0 else st["f1"]
    cross = tab.a[k, 0] * tab.a[o, 0] + tab.a[k, 1] * tab.a[o, 1]
    M1, M2 = alg1.model_eval(st["rhoe"], st["zt"], tab)
    mod = tab.b[k, 0] * (M1 - fo * tab.b[o, 0]) + tab.b[k, 1] * (M2 - fo * tab.b[o, 1])
    h, v = hv
    return t[k] - cross * backproject(project(fo, geom), geom) / g + mod + beta * alg1.adjoint_diff(h, v)


def f_solve(b, k, beta, geom, tab, g, x0, tol=1e-12, max_iter=2000, W=None):
    """Preconditioned conjugate gradients on the f_k normal equations from
    x0, preconditioner (alpha_k + c'_k + beta K)^-1 by FFT, stopping at
    ||r|| <= tol ||b||.  W: per-ray weights of the Gauss-Newton mode."""
    alpha, cp, _ = coefficients(k, tab)
    x = np.array(x0, dtype=np.float64)
    r = b - normal_op(x, k, beta, geom, tab, g, W)
    bb = float(np.sum(b * b))
    if bb == 0.0:
        return np.zeros_like(x)
    y = alg1.fft_solve(r, alpha + cp, beta)
    p = y.copy()
    ry = float(np.sum(r * y))
    for _ in range(max_iter):
        if float(np.sum(r * r)) <= tol * tol * bb:
            break
        q = normal_op(p, k, beta, geom, tab, g, W)
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


# ----------------------------------------------------------------------------
# Polyenergetic sinogram-domain fidelity, linearised by Gauss-Newton
# ----------------------------------------------------------------------------
#
# With polyenergetic arms the -log sinogram of a ray is a nonlinear function
# of the two basis line integrals l_k = A f_k (the photoelectric / Compton
# model is spanned by the two basis materials at every energy, Sec. II-B):
#
#     h_i(l1, l2) = s_i / S = -ln sum_b w_ib exp(-S (mu_1(E_b) l1 + mu_2(E_b) l2)) / S,
#
# w_ib the normalised detected spectrum of arm i (reading R15).  The data term
# of the f updates becomes (1 / gamma) sum_i || h_i(A f1, A f2) - s_i / S ||^2.
# At the iterate k (Jacobi, reading R1) it is linearised around l^k = A f^k:
#
#     h_i(l) ~ h_i(l^k) + J_i1 (l1 - l1^k) + J_i2 (l2 - l2^k),
#     J_ik = dh_i / dl_k = sum_b om_ib mu_k(E_b),  om_ib = w_ib e_ib / sum_b w_ib e_ib,
#
# (the spectrum reweighted by the attenuation along the ray), so the f_k normal
# equations keep the form of the linear mode with per-ray weights:
#
#     [A^T diag(W_kk) A / gamma + c'_k + beta L] f_k
#         = A^T v_k / gamma + sum_j b_kj (rho_e (P_j z + psi_j) - f_o b_oj) + beta (dx^T h + dy^T v),
#     W_kl = sum_i J_ik J_il,  v_k = sum_i J_ik d_i - W_ko l_o^k,
#     d_i = s_i / S - h_i(l^k) + J_i1 l1^k + J_i2 l2^k.
#
# With monoenergetic arms J_ik = a_ki and these are exactly the linear mode's
# equations.  Pins (tests/test_oracle_modeb.py): J against finite differences
# of h; the monoenergetic reduction; the solve equals a dense solve of the
# same system and minimises the linearised f_k sub-objective; a uniform
# material under noiseless polyenergetic data is a fixed point of a whole
# iteration.


def spectrum_rows(tab):
    """Per arm: (w_b, mu_hat_1(E_b), mu_hat_2(E_b)) over the detected spectrum's bins."""
    (z1, r1), (z2, r2) = tab.basis
    return [(np.asarray(w, np.float64), model.mu_hat(r1, z1, E), model.mu_hat(r2, z2, E)) for (E, w) in tab.arms]


def poly_log(l1, l2, arm):
    """(h, J1, J2) of one arm for line integrals l1, l2 (any shape), in the
    normalised units: h = -ln sum_b w_b exp(-S t_b) / S, t_b = mu_1b l1 +
    mu_2b l2, evaluated from the smallest t_b so that no term underflows."""
    w, m1, m2 = arm
    l1 = np.asarray(l1, np.float64)[..., None]
    l2 = np.asarray(l2, np.float64)[..., None]
    t = m1 * l1 + m2 * l2
    tmin = t.min(axis=-1, keepdims=True)
    e = w * np.exp(-model.S_MM * (t - tmin))
    se = e.sum(axis=-1)
    h = tmin[..., 0] - np.log(se) / model.S_MM
    om = e / se[..., None]
    return h, (om * m1).sum(axis=-1), (om * m2).sum(axis=-1)


def gn_terms(l1, l2, sL, sH, tab):
    """Per ray (W11, W22, W12, v1, v2) of the Gauss-Newton normal equations at
    l^k = (l1, l2) for measured -log sinograms sL, sH."""
    W11 = W22 = W12 = u1 = u2 = 0.0
    for s, arm in zip((sL, sH), spectrum_rows(tab)):
        h, J1, J2 = poly_log(l1, l2, arm)
        d = np.asarray(s, np.float64) / model.S_MM - h + J1 * l1 + J2 * l2
        W11 = W11 + J1 * J1
        W22 = W22 + J2 * J2
        W12 = W12 + J1 * J2
        u1 = u1 + J1 * d
        u2 = u2 + J2 * d
    return W11, W22, W12, u1 - W12 * l2, u2 - W12 * l1


def rhs_gn(k, st, hv, beta, v, geom, tab, g):
    """Right-hand side of the Gauss-Newton f_k normal equations (v: v_k)."""
    o = 1 - k
    fo = st["f2"] if k == 0 else st["f1"]
    M1, M2 = alg1.model_eval(st["rhoe"], st["zt"], tab)
    mod = tab.b[k, 0] * (M1 - fo * tab.b[o, 0]) + tab.b[k, 1] * (M2 - fo * tab.b[o, 1])
    h, vv = hv
    return backproject(v, geom) / g + mod + beta * alg1.adjoint_diff(h, vv)


def iterate_gn(st, beta, beta_t, lam, sL, sH, geom, tab, g, z_method="sparse", decision_dtype=np.float64):
    """One pass of Algorithm 1 with the Gauss-Newton polyenergetic f-updates."""
    hv = alg1.thresholds(st, lam / beta, decision_dtype)
    l1, l2 = project(st["f1"], geom), project(st["f2"], geom)
    W11, W22, W12, v1, v2 = gn_terms(l1, l2, sL, sH, tab)
    f1 = f_solve(rhs_gn(0, st, hv["f1"], beta, v1, geom, tab, g), 0, beta, geom, tab, g, st["f1"], W=W11)
    f2 = f_solve(rhs_gn(1, st, hv["f2"], beta, v2, geom, tab, g), 1, beta, geom, tab, g, st["f2"], W=W22)
    m1, m2 = alg1.synthesize(f1, f2, tab)
    rhoe = alg1.fft_solve(alg1.rhs_rho(m1, m2, hv["rhoe"], beta_t, tab), 1.0, beta_t)
    a2, rz = alg1.z_terms(m1, m2, hv["zt"], beta_t, tab)
    zt = alg1.z_solve(a2, rz, beta_t, z_method)
    return dict(f1=f1, f2=f2, rhoe=rhoe, zt=zt), hv


def solve_gn(sL, sH, geom, tab, prm: alg1.Params, st0=None):
    """Algorithm 1 with the Gauss-Newton polyenergetic f-updates, from the FBP
    image pair (or ``st0``); returns the final state with Z."""
    g = gamma(geom)
    if st0 is None:
        st = alg1.init_state(ct.fbp(sL, geom) / model.S_MM, ct.fbp(sH, geom) / model.S_MM, tab, prm.z_clip,
                             prm.rho_air)
    else:
        st = dict(st0)
    beta = prm.beta0
    kappa = prm.kappa_value()
    for _ in range(prm.iters):
        st, _hv = iterate_gn(st, beta, prm.tau * beta, prm.lam, sL, sH, geom, tab, g, prm.z_method,
                             prm.decision_dtype)
        beta = kappa * beta
    st["Z"] = model.z_from_ztilde(st["zt"])
    return st


def sub_objective_gn(fk, k, st, hv_k, beta, l1, l2, sL, sH, geom, tab, g):
    """The linearised f_k sub-objective of the Gauss-Newton mode at l^k."""
    o = 1 - k
    fo = st["f2"] if k == 0 else st["f1"]
    lk = ct.project(fk, geom)
    lo = l2 if k == 0 else l1
    val = 0.0
    for s, arm in zip((sL, sH), spectrum_rows(tab)):
        h, J1, J2 = poly_log(l1, l2, arm)
        d = np.asarray(s, np.float64) / model.S_MM - h + J1 * l1 + J2 * l2
        Jk, Jo = (J1, J2) if k == 0 else (J2, J1)
        r = Jk * lk + Jo * lo - d
        val += float(np.sum(r * r)) / g
    M = alg1.model_eval(st["rhoe"], st["zt"], tab)
    for j in (0, 1):
        dd = fk * tab.b[k, j] + fo * tab.b[o, j] - M[j]
        val += float(np.sum(dd * dd))
    dx, dy = alg1.forward_diff(fk)
    h, v = hv_k
    return val + beta * float(np.sum((dx - h) ** 2) + np.sum((dy - v) ** 2))
