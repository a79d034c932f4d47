"""Pins of the oracle's relaxed objective (eq. obj_unconstraint, Sec. II-D).

``alg1.objective`` sums, for the state (f1, f2, rho_e, z) and auxiliary
gradients (h, v) of all four maps:

    fid_L + fid_H   = sum (f1 a_1L + f2 a_2L - mu_L)^2 + sum (f1 a_1H + f2 a_2H - mu_H)^2
    mod_1 + mod_2   = sum (rho_e (P_j z + psi_j) - (f1 b_1j + f2 b_2j))^2,  j = 1, 2
    relax           = beta sum_g sum ((dx g - h_g)^2 + (dy g - v_g)^2)
    l0              = lambda sum_g C(h_g, v_g)

The values below are worked out by hand on 3 x 3 grids with small integer
tables, so that a dropped term, a transposed table index, a wrong difference
direction or a miscounted C(h, v) each changes the total.  The derivations
are in the comments next to each expected number."""
import numpy as np
import pytest

from oracle import alg1, model
from synthetic import phantoms as ph


class _Tab:
    """Hand-picked tables: a[k][i] basis k at arm i, b[k][j] basis k at E_j."""
    a = np.array([[2.0, 1.0], [0.0, 1.0]])     # a_1L = 2, a_1H = 1, a_2L = 0, a_2H = 1
    b = np.array([[1.0, 0.5], [0.25, 1.0]])    # b_11 = 1, b_12 = 0.5, b_21 = 0.25, b_22 = 1
    P = np.array([1.0, 0.5])
    psi = np.array([0.5, 1.0])


def _zero_hv(n=3):
    z = np.zeros((n, n))
    return {g: (z.copy(), z.copy()) for g in ("f1", "f2", "rhoe", "zt")}


def _base_state():
    """f1 = 1, f2 = 2, rho_e = 1 everywhere.  mu_L = 2 except mu_L[0,0] = 5,
    mu_H = 3 except mu_H[2,1] = 1.

    dL = 2 f1 + 0 f2 - mu_L = 0 except -3 at (0,0)      -> fid_L = 9
    dH = 1 f1 + 1 f2 - mu_H = 0 except  2 at (2,1)      -> fid_H = 4
    m1 = f1 b_11 + f2 b_21 = 1 + 0.5 = 1.5;  m2 = f1 b_12 + f2 b_22 = 0.5 + 2 = 2.5
    """
    st = dict(f1=np.ones((3, 3)), f2=np.full((3, 3), 2.0), rhoe=np.ones((3, 3)))
    muL = np.full((3, 3), 2.0)
    muL[0, 0] = 5.0
    muH = np.full((3, 3), 3.0)
    muH[2, 1] = 1.0
    return st, muL, muH


def _x_step_state():
    """z = 1 in columns 0 and 1, 2 in column 2.

    M1 = rho (z + 0.5) = 1.5, 1.5, 2.5 -> M1 - m1 = 0, 0, 1 per row        -> mod_1 = 3
    M2 = rho (0.5 z + 1) = 1.5, 1.5, 2 -> M2 - m2 = -1, -1, -0.5 per row   -> mod_2 = 3 (1 + 1 + 0.25) = 6.75
    dx z (periodic, forward) per row: 1-1 = 0, 2-1 = 1, 1-2 = -1; dy z = 0
    """
    st, muL, muH = _base_state()
    zt = np.ones((3, 3))
    zt[:, 2] = 2.0
    st["zt"] = zt
    return st, muL, muH


def test_objective_hand_value_all_gradients_zeroed():
    st, muL, muH = _x_step_state()
    t = alg1.objective(st, _zero_hv(), 0.5, 0.25, muL, muH, _Tab)
    # relax = beta * sum dx z^2 = 0.5 * 3 rows * (0 + 1 + 1) = 3; no kept gradient -> l0 = 0
    assert t["fid_L"] == 9.0 and t["fid_H"] == 4.0
    assert t["mod_1"] == 3.0 and t["mod_2"] == 6.75
    assert t["relax"] == 3.0 and t["nnz"] == 0 and t["l0"] == 0.0
    assert t["total"] == 9.0 + 4.0 + 3.0 + 6.75 + 3.0


def test_objective_hand_value_gradients_kept():
    st, muL, muH = _x_step_state()
    hv = _zero_hv()
    h = np.zeros((3, 3))
    h[:, 1], h[:, 2] = 1.0, -1.0        # h = dx z exactly
    hv["zt"] = (h, np.zeros((3, 3)))
    t = alg1.objective(st, hv, 0.5, 0.25, muL, muH, _Tab)
    # relax = 0; C(h, v) = 2 kept pixels per row * 3 rows = 6 -> l0 = 0.25 * 6 = 1.5
    assert t["relax"] == 0.0 and t["nnz"] == 6 and t["l0"] == 1.5
    assert t["total"] == 9.0 + 4.0 + 3.0 + 6.75 + 1.5


def test_objective_hand_value_mixed_maps():
    st, muL, muH = _x_step_state()
    hv = _zero_hv()
    h = np.zeros((3, 3))
    h[:, 1] = 1.0                        # keeps only the +1 step of z
    hv["zt"] = (h, np.zeros((3, 3)))
    hf, vf = np.zeros((3, 3)), np.zeros((3, 3))
    hf[1, 1], vf[0, 2] = 0.5, -1.0       # on f1, whose differences are all zero
    hv["f1"] = (hf, vf)
    t = alg1.objective(st, hv, 0.5, 0.25, muL, muH, _Tab)
    # z: (dx - h)^2 = 0 at column 1, (-1 - 0)^2 = 1 at column 2, 3 rows -> 3
    # f1: (0 - 0.5)^2 + (0 - (-1))^2 = 1.25
    # relax = 0.5 * (3 + 1.25) = 2.125; C = 3 (z) + 2 (f1) = 5 -> l0 = 1.25
    assert t["relax"] == 2.125 and t["nnz"] == 5 and t["l0"] == 1.25
    assert t["total"] == 9.0 + 4.0 + 3.0 + 6.75 + 2.125 + 1.25


def test_objective_hand_value_y_step():
    st, muL, muH = _base_state()
    zt = np.ones((3, 3))
    zt[2, :] = 3.0
    st["zt"] = zt
    t = alg1.objective(st, _zero_hv(), 0.5, 0.25, muL, muH, _Tab)
    # M1 = z + 0.5 = 1.5, 1.5, 3.5 by row -> (M1 - 1.5)^2 = 4 on row 2: 3 * 4  -> mod_1 = 12
    # M2 = 0.5 z + 1 = 1.5, 1.5, 2.5 by row -> (M2 - 2.5)^2 = 1 on rows 0, 1  -> mod_2 = 6
    # dy z per column: 1-1 = 0, 3-1 = 2, 1-3 = -2 -> 3 columns * 8 = 24; relax = 0.5 * 24 = 12
    assert t["mod_1"] == 12.0 and t["mod_2"] == 6.0 and t["relax"] == 12.0
    assert t["total"] == 9.0 + 4.0 + 12.0 + 6.0 + 12.0


def test_objective_vanishes_at_exact_uniform_material():
    """Noiseless uniform water with the real tables: the basis-2 material is
    water, so f = (0, 1) reproduces mu_L, mu_H, the model at (rho_e, z) =
    (1, 1) equals the synthesis, and every difference is zero."""
    acq = ph.acquisition("small")
    tab = model.Tables(acq.low, acq.high)
    shape = (4, 5)
    muL = np.full(shape, tab.a[1, 0])
    muH = np.full(shape, tab.a[1, 1])
    st = dict(f1=np.zeros(shape), f2=np.ones(shape), rhoe=np.ones(shape), zt=np.ones(shape))
    hv = alg1.thresholds(st, 1e-3)
    t = alg1.objective(st, hv, 3.0, 1e-2, muL, muH, tab)
    scale = tab.b[1, 0] ** 2 * muL.size
    for k in ("fid_L", "fid_H", "mod_1", "mod_2"):
        assert t[k] <= 1e-24 * scale, (k, t[k])
    assert t["relax"] == 0.0 and t["nnz"] == 0 and t["l0"] == 0.0


def test_objective_f_part_equals_f_subproblem():
    """The f-dependent terms of the relaxed objective are eq. obj_sub_f (with
    rho_e and z held): fid + mod + beta (relax of f1, f2) = sub_objective_f."""
    rng = np.random.default_rng(3)
    acq = ph.acquisition("small")
    tab = model.Tables(acq.low, acq.high)
    shape = (6, 7)
    st = dict(f1=rng.random(shape), f2=rng.random(shape) + 0.5, rhoe=rng.random(shape) + 0.5,
              zt=rng.random(shape) + 0.5)
    muL, muH = rng.random(shape) * 20, rng.random(shape) * 15
    hv = alg1.thresholds(st, 0.05)
    beta = 0.7
    t = alg1.objective(st, hv, beta, 1e-2, muL, muH, tab)
    # relax of rho_e and z alone: the same state with f1 = f2 = 0 and their (h, v) zero
    t_rz = alg1.objective(dict(st, f1=np.zeros(shape), f2=np.zeros(shape)),
                          dict(hv, f1=(np.zeros(shape),) * 2, f2=(np.zeros(shape),) * 2),
                          beta, 1e-2, muL, muH, tab)
    relax_f = t["relax"] - t_rz["relax"]
    sub = alg1.sub_objective_f(st["f1"], st["f2"], st, hv["f1"], hv["f2"], beta, muL, muH, tab)
    lhs = t["fid_L"] + t["fid_H"] + t["mod_1"] + t["mod_2"] + relax_f
    assert abs(lhs - sub) <= 1e-12 * abs(sub)
