"""Pins of the sinogram-domain f-updates of the oracle (oracle/modeb.py)."""
import numpy as np

from oracle import alg1, ct, model, modeb
from synthetic import phantoms as ph


def tiny():
    acq = ph.acquisition("small", n=16)
    geom = dict(nx=16, ny=12, pixel_mm=1.0, n_views=24, n_bins=28, sid_mm=200.0, sdd_mm=300.0,
                bin_mm=1.0, start_rad=0.05, arc_rad=2 * np.pi)
    tab = model.Tables(acq.low, acq.high)
    return geom, tab


def random_state(shape, seed):
    rng = np.random.default_rng(seed)
    st = dict(f1=0.2 * rng.standard_normal(shape), f2=1.0 + 0.2 * rng.standard_normal(shape),
              rhoe=1.0 + 0.1 * rng.standard_normal(shape), zt=1.0 + 0.1 * rng.standard_normal(shape))
    hv = (0.05 * rng.standard_normal(shape), 0.05 * rng.standard_normal(shape))
    return st, hv


def test_sparse_matrix_reproduces_projector():
    geom, _ = tiny()
    rng = np.random.default_rng(2)
    x = rng.standard_normal((geom["ny"], geom["nx"]))
    y = rng.standard_normal((geom["n_views"], geom["n_bins"]))
    px, bx = ct.project(x, geom), ct.backproject(y, geom)
    assert np.max(np.abs(modeb.project(x, geom) - px)) <= 1e-12 * np.max(np.abs(px))
    assert np.max(np.abs(modeb.backproject(y, geom) - bx)) <= 1e-12 * np.max(np.abs(bx))


def test_gamma_is_dc_gain():
    geom, _ = tiny()
    g = modeb.gamma(geom)
    ones = np.ones((geom["ny"], geom["nx"]))
    assert np.isclose(np.sum(ones * ct.backproject(ct.project(ones, geom), geom)) / ones.size, g, rtol=1e-12)


def test_normal_operator_symmetric_positive_definite():
    geom, tab = tiny()
    g = modeb.gamma(geom)
    rng = np.random.default_rng(3)
    shape = (geom["ny"], geom["nx"])
    for k in (0, 1):
        x, y = rng.standard_normal(shape), rng.standard_normal(shape)
        qx, qy = modeb.normal_op(x, k, 0.7, geom, tab, g), modeb.normal_op(y, k, 0.7, geom, tab, g)
        assert abs(np.sum(qx * y) - np.sum(x * qy)) <= 1e-12 * np.sum(np.abs(qx * y))
        assert np.sum(qx * x) > 0


def test_cg_equals_dense_solve():
    geom, tab = tiny()
    g = modeb.gamma(geom)
    shape = (geom["ny"], geom["nx"])
    n = shape[0] * shape[1]
    rng = np.random.default_rng(4)
    for k in (0, 1):
        Q = np.empty((n, n))
        for c in range(n):
            e = np.zeros(n)
            e[c] = 1.0
            Q[:, c] = modeb.normal_op(e.reshape(shape), k, 0.3, geom, tab, g).ravel()
        b = rng.standard_normal(shape)
        ref = np.linalg.solve(Q, b.ravel()).reshape(shape)
        got = modeb.f_solve(b, k, 0.3, geom, tab, g, np.zeros(shape))
        assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref))


def test_f_update_is_the_exact_minimiser_of_its_sub_objective():
    """E(f* + d) - E(f*) = d^T Q d for the quadratic sub-objective written
    from the data term itself; a missing term or sign in the normal
    equations breaks the identity."""
    geom, tab = tiny()
    g = modeb.gamma(geom)
    shape = (geom["ny"], geom["nx"])
    st, hv = random_state(shape, 5)
    rng = np.random.default_rng(6)
    sL = rng.uniform(0.0, 3.0, (geom["n_views"], geom["n_bins"]))
    sH = rng.uniform(0.0, 2.5, (geom["n_views"], geom["n_bins"]))
    t = modeb.data_images(sL, sH, geom, tab, g)
    beta = 0.4
    for k in (0, 1):
        fk = modeb.f_solve(modeb.rhs(k, st, hv, beta, t, geom, tab, g), k, beta, geom, tab, g, np.zeros(shape))
        e0 = modeb.sub_objective(fk, k, st, hv, beta, sL, sH, geom, tab, g)
        for s in range(3):
            d = 1e-2 * rng.standard_normal(shape)
            e1 = modeb.sub_objective(fk + d, k, st, hv, beta, sL, sH, geom, tab, g)
            dqd = float(np.sum(d * modeb.normal_op(d, k, beta, geom, tab, g)))
            assert e1 > e0
            assert abs((e1 - e0) - dqd) <= 1e-7 * dqd


def test_uniform_water_is_a_fixed_point():
    """Consistent noiseless mono sinograms of uniform water: the state
    f = (0, 1), rho_e = 1, z = 1 is kept by a whole iteration."""
    acq = ph.acquisition("small", n=16)
    geom = ct.geometry(acq)
    tab = model.Tables(acq.low, acq.high)
    shape = (acq.ny, acq.nx)
    Z = np.full(shape, 7.45)
    rho = np.ones(shape)
    sL, sH = ct.simulate(Z, rho, acq, seed=None)
    g = modeb.gamma(geom)
    t = modeb.data_images(sL, sH, geom, tab, g)
    st = dict(f1=np.zeros(shape), f2=np.ones(shape), rhoe=np.ones(shape), zt=np.ones(shape))
    new, _ = modeb.iterate(st, 0.5, 0.5, 1e-2, t, geom, tab, g, z_method="dense")
    for key in ("f1", "f2", "rhoe", "zt"):
        assert np.max(np.abs(new[key] - st[key])) <= 1e-8, key


# --- polyenergetic fidelity linearised by Gauss-Newton ----------------------

def tiny_poly():
    geom, _ = tiny()
    acq = ph.acquisition("clinical", n=16)
    return geom, model.Tables(acq.low, acq.high)


def test_poly_jacobian_matches_finite_differences():
    _, tab = tiny_poly()
    rng = np.random.default_rng(7)
    l1 = rng.uniform(0.0, 40.0, 9)
    l2 = rng.uniform(0.0, 300.0, 9)
    for arm in modeb.spectrum_rows(tab):
        h, J1, J2 = modeb.poly_log(l1, l2, arm)
        eps = 1e-4
        d1 = (modeb.poly_log(l1 + eps, l2, arm)[0] - modeb.poly_log(l1 - eps, l2, arm)[0]) / (2 * eps)
        d2 = (modeb.poly_log(l1, l2 + eps, arm)[0] - modeb.poly_log(l1, l2 - eps, arm)[0]) / (2 * eps)
        assert np.allclose(J1, d1, rtol=1e-7) and np.allclose(J2, d2, rtol=1e-7)
        # h is the -log of the spectrum-weighted transmission, written out bin by bin
        w, m1, m2 = arm
        ref = np.array([-np.log(np.sum(w * np.exp(-model.S_MM * (m1 * a + m2 * b)))) / model.S_MM
                        for a, b in zip(l1, l2)])
        assert np.allclose(h, ref, rtol=1e-12)


def test_gauss_newton_reduces_to_the_linear_mode_for_mono_arms():
    """Monoenergetic arms: J_ik = a_ki, so W_kk = alpha_k, W_12 = cross and
    A^T v_k / gamma + the cross term of the linear mode agree."""
    geom, tab = tiny()
    g = modeb.gamma(geom)
    rng = np.random.default_rng(8)
    shape = (geom["ny"], geom["nx"])
    st, hv = random_state(shape, 9)
    sL = rng.uniform(0.0, 3.0, (geom["n_views"], geom["n_bins"]))
    sH = rng.uniform(0.0, 2.5, (geom["n_views"], geom["n_bins"]))
    l1, l2 = modeb.project(st["f1"], geom), modeb.project(st["f2"], geom)
    W11, W22, W12, v1, v2 = modeb.gn_terms(l1, l2, sL, sH, tab)
    for k, W in ((0, W11), (1, W22)):
        alpha, _, cross = modeb.coefficients(k, tab)
        assert np.allclose(W, alpha, rtol=1e-13)
        assert np.allclose(W12, cross, rtol=1e-12)
    t = modeb.data_images(sL, sH, geom, tab, g)
    for k, v in ((0, v1), (1, v2)):
        lin = modeb.rhs(k, st, hv, 0.4, t, geom, tab, g)
        gn = modeb.rhs_gn(k, st, hv, 0.4, v, geom, tab, g)
        assert np.allclose(gn, lin, rtol=1e-10, atol=1e-10 * np.abs(lin).max())


def test_gauss_newton_solve_is_dense_solve_and_minimiser():
    geom, tab = tiny_poly()
    g = modeb.gamma(geom)
    shape = (geom["ny"], geom["nx"])
    n = shape[0] * shape[1]
    st, hv = random_state(shape, 10)
    rng = np.random.default_rng(11)
    sL = rng.uniform(0.5, 3.0, (geom["n_views"], geom["n_bins"]))
    sH = rng.uniform(0.4, 2.5, (geom["n_views"], geom["n_bins"]))
    l1, l2 = modeb.project(st["f1"], geom), modeb.project(st["f2"], geom)
    W11, W22, W12, v1, v2 = modeb.gn_terms(l1, l2, sL, sH, tab)
    beta = 0.3
    for k, W, v in ((0, W11, v1), (1, W22, v2)):
        # dense A^T diag(W) A / gamma + c' + beta L from the projector's columns
        Q = np.empty((n, n))
        for c in range(n):
            e = np.zeros(n)
            e[c] = 1.0
            Q[:, c] = modeb.normal_op(e.reshape(shape), k, beta, geom, tab, g, W).ravel()
        b = modeb.rhs_gn(k, st, hv, beta, v, geom, tab, g)
        ref = np.linalg.solve(Q, b.ravel()).reshape(shape)
        got = modeb.f_solve(b, k, beta, geom, tab, g, np.zeros(shape), W=W)
        assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref))
        e0 = modeb.sub_objective_gn(got, k, st, hv, beta, l1, l2, sL, sH, geom, tab, g)
        for s in range(3):
            d = 1e-2 * rng.standard_normal(shape)
            e1 = modeb.sub_objective_gn(got + d, k, st, hv, beta, l1, l2, sL, sH, geom, tab, g)
            dqd = float(np.sum(d * modeb.normal_op(d, k, beta, geom, tab, g, W)))
            assert e1 > e0 and abs((e1 - e0) - dqd) <= 1e-7 * dqd


def test_uniform_material_is_a_gauss_newton_fixed_point():
    """Noiseless polyenergetic sinograms (Kramers 80 / 140 kVp, Al, Sn) of a
    uniform bone-like material: the exact state is kept by a whole iteration
    of the Gauss-Newton mode (the linear mode would move it: beam hardening)."""
    acq = ph.acquisition("clinical", n=16)
    geom = ct.geometry(acq)
    tab = model.Tables(acq.low, acq.high)
    shape = (acq.ny, acq.nx)
    Zv, rv = 11.0, 1.4
    sL, sH = ct.simulate(np.full(shape, Zv), np.full(shape, rv), acq, seed=None)
    st = alg1.init_state(np.full(shape, model.effective(model.mu_hat(rv, Zv, tab.arms[0][0]), tab.arms[0][1])),
                         np.full(shape, model.effective(model.mu_hat(rv, Zv, tab.arms[1][0]), tab.arms[1][1])), tab)
    assert np.allclose(model.z_from_ztilde(st["zt"]), Zv, rtol=1e-10)
    g = modeb.gamma(geom)
    new, _ = modeb.iterate_gn(st, 0.5, 0.5, 1e-2, sL, sH, geom, tab, g, z_method="dense")
    for key in ("f1", "f2", "rhoe", "zt"):
        assert np.max(np.abs(new[key] - st[key])) <= 1e-7 * max(1.0, np.abs(st[key]).max()), key
    lin, _ = modeb.iterate(st, 0.5, 0.5, 1e-2, modeb.data_images(sL, sH, geom, tab, g), geom, tab, g,
                           z_method="dense")
    assert np.max(np.abs(lin["f1"] - st["f1"])) > 1e-3
