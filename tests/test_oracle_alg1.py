"""Pins of the oracle's Algorithm 1 building blocks (Sec. II-C, II-D)."""
import numpy as np
import pytest

from oracle import alg1, l0, model
from synthetic import phantoms as ph


def graph_laplacian_dense(ny, nx):
    """Periodic 5-point graph Laplacian built by accumulating the four
    neighbour couplings of each pixel (independent of the roll-based code)."""
    n = ny * nx
    L = np.zeros((n, n))
    for j in range(ny):
        for i in range(nx):
            p = j * nx + i
            for dj, di in ((0, 1), (0, -1), (1, 0), (-1, 0)):
                q = ((j + dj) % ny) * nx + (i + di) % nx
                L[p, p] += 1.0
                L[p, q] -= 1.0
    return L


@pytest.mark.parametrize("shape", [(8, 8), (6, 10), (5, 7), (1, 6), (2, 3)])
def test_laplacian_matches_graph_laplacian(shape):
    ny, nx = shape
    g = ph.random_field(shape, 1)
    assert np.allclose(alg1.laplacian(g).ravel(), graph_laplacian_dense(ny, nx) @ g.ravel(), atol=1e-12)


def test_adjoint_diff_is_adjoint():
    g = ph.random_field((7, 9), 2)
    h = ph.random_field((7, 9), 3)
    v = ph.random_field((7, 9), 4)
    dx, dy = alg1.forward_diff(g)
    assert abs(np.sum(dx * h) + np.sum(dy * v) - np.sum(g * alg1.adjoint_diff(h, v))) < 1e-12


def test_threshold_is_brute_force_minimiser():
    """eq. sol_hv: per pixel, the returned (h, v) minimises
    E(r) = (h - dx)^2 + (v - dy)^2 + (lambda/beta) H(|h| + |v|) over a dense
    grid of candidate pairs that includes (0, 0) and (dx, dy)."""
    g = ph.random_field((6, 6), 5, 0, 1)
    thr = 0.15
    h, v, _ = alg1.hard_threshold(g, thr)
    dx, dy = alg1.forward_diff(g)
    cand = np.linspace(-1.5, 1.5, 61)
    for j in range(6):
        for i in range(6):
            def E(hh, vv):
                return (hh - dx[j, i]) ** 2 + (vv - dy[j, i]) ** 2 + thr * ((abs(hh) + abs(vv)) != 0)
            best = min(min(E(a, b) for a in cand for b in cand), E(0.0, 0.0), E(dx[j, i], dy[j, i]))
            assert E(h[j, i], v[j, i]) <= best + 1e-15


def test_threshold_tie_goes_to_zero():
    g = np.zeros((3, 3))
    g[1, 2] = 0.5          # dx at (1,1) = 0.5, dy = 0 -> squared 0.25
    h, v, keep = alg1.hard_threshold(g, 0.25)
    assert h[1, 1] == 0.0 and not keep[1, 1]
    h, v, keep = alg1.hard_threshold(g, 0.2499999)
    assert h[1, 1] == 0.5


@pytest.mark.parametrize("shape", [(8, 8), (6, 10), (5, 7), (1, 9)])
def test_fft_solve_equals_dense_solve(shape):
    ny, nx = shape
    rhs = ph.random_field(shape, 7)
    c, beta = 1.3, 0.7
    dense = np.linalg.solve(c * np.eye(ny * nx) + beta * graph_laplacian_dense(ny, nx), rhs.ravel())
    assert np.allclose(alg1.fft_solve(rhs, c, beta).ravel(), dense, rtol=1e-11, atol=1e-12)


def test_z_solve_equals_dense_and_fft():
    ny, nx = 9, 8
    a2 = ph.random_field((ny, nx), 8, 0.1, 2.0)
    rhs = ph.random_field((ny, nx), 9)
    bt = 0.37
    dense = np.linalg.solve(np.diag(a2.ravel()) + bt * graph_laplacian_dense(ny, nx), rhs.ravel())
    assert np.allclose(alg1.z_solve(a2, rhs, bt).ravel(), dense, rtol=1e-10, atol=1e-12)
    assert np.allclose(alg1.z_solve(a2, rhs, bt, "dense").ravel(), dense, rtol=1e-10, atol=1e-12)
    const = np.full((ny, nx), 0.8)
    assert np.allclose(alg1.z_solve(const, rhs, bt), alg1.fft_solve(rhs, 0.8, bt), rtol=1e-10, atol=1e-12)


def _noisy_state(seed=11, n=12):
    acq = ph.acquisition("small")
    tab = model.Tables(acq.low, acq.high)
    rng = np.random.default_rng(seed)
    Z = 7.45 + 5 * (rng.random((n, n)) > 0.7)
    rho = 1.0 + 0.5 * (rng.random((n, n)) > 0.8)
    muL = model.mu_hat(rho, Z, 60.0) * (1 + 0.02 * rng.standard_normal((n, n)))
    muH = model.mu_hat(rho, Z, 90.0) * (1 + 0.02 * rng.standard_normal((n, n)))
    st = alg1.init_state(muL, muH, tab)
    return st, muL, muH, tab


def _is_minimiser(J, x, seed, eps=1e-4, trials=6):
    rng = np.random.default_rng(seed)
    J0 = J(x)
    for _ in range(trials):
        d = rng.standard_normal(x.shape)
        jp, jm = J(x + eps * d), J(x - eps * d)
        curv = jp + jm - 2 * J0
        assert curv > 0
        # first-order term vanishes at the minimiser
        assert abs(jp - jm) < 1e-5 * curv + 1e-10 * abs(J0)


def test_block_updates_minimise_their_subproblems():
    """Each update of Algorithm 1 minimises its own printed subproblem
    (eq. obj_sub_f over f1 with f2 fixed and vice versa, eq. obj_sub_rho,
    eq. obj_sub_z), checked by random two-sided perturbations."""
    st, muL, muH, tab = _noisy_state()
    beta, lam = 0.05, 0.01
    new, hv = alg1.iterate(st, beta, beta, lam, muL, muH, tab)
    _is_minimiser(lambda f1: alg1.sub_objective_f(f1, st["f2"], st, hv["f1"], hv["f2"], beta, muL, muH, tab),
                  new["f1"], 1)
    _is_minimiser(lambda f2: alg1.sub_objective_f(st["f1"], f2, st, hv["f1"], hv["f2"], beta, muL, muH, tab),
                  new["f2"], 2)
    m1, m2 = alg1.synthesize(new["f1"], new["f2"], tab)
    _is_minimiser(lambda r: alg1.sub_objective_rho(r, m1, m2, hv["rhoe"], beta, tab), new["rhoe"], 3)
    _is_minimiser(lambda z: alg1.sub_objective_z(z, m1, m2, hv["zt"], beta, tab), new["zt"], 4)


def test_gauss_seidel_variant_minimises_f2_with_new_f1():
    st, muL, muH, tab = _noisy_state(12)
    beta, lam = 0.05, 0.01
    new, hv = alg1.iterate(st, beta, beta, lam, muL, muH, tab, order="gauss-seidel")
    _is_minimiser(lambda f2: alg1.sub_objective_f(new["f1"], f2, st, hv["f1"], hv["f2"], beta, muL, muH, tab),
                  new["f2"], 5)


@pytest.mark.parametrize("order", ["jacobi", "gauss-seidel"])
def test_uniform_material_is_fixed_point(order):
    acq = ph.acquisition("small")
    tab = model.Tables(acq.low, acq.high)
    muL = np.full((10, 12), model.mu_hat(1.3, 9.0, 60.0))
    muH = np.full((10, 12), model.mu_hat(1.3, 9.0, 90.0))
    st = alg1.solve(muL, muH, tab, alg1.Params(iters=50, order=order))
    assert np.allclose(st["rhoe"], 1.3, rtol=1e-10)
    assert np.allclose(st["Z"], 9.0, rtol=1e-10)


def test_l0_piecewise_constant_fixed_point():
    """Jumps with jump^2 > lambda/beta0 are all kept, then eq. L0_sub_g returns g~."""
    g = ph.piecewise_constant(16, 12, 3, n_levels=3)
    g = np.round(g * 3) * 1.0   # levels on a grid of 1.0: every jump >= 1
    out = l0.l0_smooth(g, lam=0.2)
    assert np.allclose(out, g, atol=1e-11)


def test_l0_fixed_beta_monotone():
    g0 = ph.piecewise_constant(20, 20, 4) + 0.1 * ph.normal_field((20, 20), 5)
    lam, beta = 0.05, 0.4
    g = g0.copy()
    vals = []
    for _ in range(15):
        g, h, v = l0.l0_step(g, g0, beta, lam)
        vals.append(l0.relaxed_objective(g, g0, h, v, beta, lam))
    assert all(b <= a + 1e-12 for a, b in zip(vals, vals[1:]))


def test_l0_reduces_noise():
    clean = ph.piecewise_constant(32, 32, 6)
    noisy = clean + 0.05 * ph.normal_field((32, 32), 7)
    out = l0.l0_smooth(noisy, lam=0.02)
    assert np.mean((out - clean) ** 2) < 0.5 * np.mean((noisy - clean) ** 2)


def test_parameters_schedule():
    prm = alg1.Params(iters=50)
    assert abs(prm.beta0 * prm.kappa_value() ** 50 - prm.beta_max) < 1e-6 * prm.beta_max


def test_init_air_reading():
    acq = ph.acquisition("small")
    tab = model.Tables(acq.low, acq.high)
    muL = np.array([[0.0, 1e-3, model.mu_hat(1.0, 7.45, 60.0)]])
    muH = np.array([[0.0, -1e-3, model.mu_hat(1.0, 7.45, 90.0)]])
    st = alg1.init_state(muL, muH, tab)
    assert st["zt"][0, 0] == 1.0 and st["zt"][0, 1] == 1.0
    assert abs(st["zt"][0, 2] - 1.0) < 1e-12
