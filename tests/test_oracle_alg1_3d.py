"""Pins of the volume form of Algorithm 1 (3-D multi-domain regularisation,
readings R22, R23): each check is against something other than the 3-D code
itself — the 2-D oracle, a dense or Kronecker-assembled system, a brute-force
minimiser, or a fixed point."""
import numpy as np
import pytest

from oracle import alg1, alg1_3d, model
from synthetic import phantoms as ph


def graph_laplacian3_dense(nz, ny, nx):
    """Periodic 7-point graph Laplacian from the six neighbour couplings of each
    voxel, accumulated one by one (independent of the roll- and kron-based code)."""
    n = nz * ny * nx
    L = np.zeros((n, n))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                p = (k * ny + j) * nx + i
                for dk, dj, di in ((0, 0, 1), (0, 0, -1), (0, 1, 0), (0, -1, 0), (1, 0, 0), (-1, 0, 0)):
                    q = (((k + dk) % nz) * ny + (j + dj) % ny) * nx + (i + di) % nx
                    L[p, p] += 1.0
                    L[p, q] -= 1.0
    return L


@pytest.mark.parametrize("shape", [(3, 4, 5), (2, 3, 3), (4, 2, 6), (1, 5, 4)])
def test_laplacian3_matches_graph_laplacian(shape):
    g = ph.random_field(shape, 1)
    L = graph_laplacian3_dense(*shape)
    assert np.allclose(alg1_3d.laplacian3(g).ravel(), L @ g.ravel(), atol=1e-12)
    # the sparse Z^m matrix is diag(a^2) plus beta~ times the same operator
    a2 = ph.random_field(shape, 2, 0.1, 1.0)
    M = alg1_3d.z_system3(a2, 0.7).toarray()
    assert np.allclose(M, np.diag(a2.ravel()) + 0.7 * L, atol=1e-12)


def test_adjoint_diff3_is_adjoint():
    g, h, v, w = (ph.random_field((3, 5, 4), s) for s in (3, 4, 5, 6))
    dx, dy, dz = alg1_3d.forward_diff3(g)
    lhs = np.sum(dx * h) + np.sum(dy * v) + np.sum(dz * w)
    assert abs(lhs - np.sum(g * alg1_3d.adjoint_diff3(h, v, w))) < 1e-12


def test_threshold3_is_brute_force_miniser():
    """Per voxel the returned triple minimises (h - dx)^2 + (v - dy)^2 + (w - dz)^2
    + (lambda/beta) [(h, v, w) != 0] over a grid of candidates that includes
    (0, 0, 0) and the gradient itself."""
    g = ph.random_field((3, 4, 4), 7, 0, 1)
    thr = 0.2
    h, v, w, _ = alg1_3d.hard_threshold3(g, thr)
    dx, dy, dz = alg1_3d.forward_diff3(g)
    cand = np.linspace(-1.2, 1.2, 13)
    for k in range(3):
        for j in range(4):
            for i in range(4):
                gx, gy, gz = dx[k, j, i], dy[k, j, i], dz[k, j, i]

                def E(a, b, c):
                    return (a - gx) ** 2 + (b - gy) ** 2 + (c - gz) ** 2 + thr * ((abs(a) + abs(b) + abs(c)) != 0)
                best = min(min(E(a, b, c) for a in cand for b in cand for c in cand), E(0, 0, 0), E(gx, gy, gz))
                assert E(h[k, j, i], v[k, j, i], w[k, j, i]) <= best + 1e-15


def test_threshold3_tie_goes_to_zero():
    g = np.zeros((2, 3, 3))
    g[1, 1, 1] = 0.5       # dz at (0, 1, 1) = 0.5, dx = dy = 0 -> squared 0.25
    h, v, w, keep = alg1_3d.hard_threshold3(g, 0.25)
    assert w[0, 1, 1] == 0.0 and not keep[0, 1, 1]
    h, v, w, keep = alg1_3d.hard_threshold3(g, 0.2499)
    assert w[0, 1, 1] == 0.5 and keep[0, 1, 1]


@pytest.mark.parametrize("shape", [(3, 4, 5), (4, 3, 2), (1, 6, 4)])
def test_fft_solve3_is_dense_solve(shape):
    """(c I + beta L3) g = rhs, L3 assembled as the Kronecker sum of the 1-D
    periodic second differences."""
    nz, ny, nx = shape

    def lap1(n):
        D = np.roll(np.eye(n), 1, axis=1) - np.eye(n)
        return D.T @ D
    I = np.eye
    L3 = (np.kron(np.kron(I(nz), I(ny)), lap1(nx)) + np.kron(np.kron(I(nz), lap1(ny)), I(nx))
          + np.kron(np.kron(lap1(nz), I(ny)), I(nx)))
    rhs = ph.random_field(shape, 8)
    c, beta = 0.6, 1.7
    dense = np.linalg.solve(c * np.eye(nz * ny * nx) + beta * L3, rhs.ravel())
    assert np.allclose(alg1_3d.fft_solve3(rhs, c, beta).ravel(), dense, rtol=1e-10, atol=1e-12)


def test_z_solve3_is_dense_solve():
    shape = (3, 4, 4)
    a2 = ph.random_field(shape, 9, 0.05, 2.0)
    rhs = ph.random_field(shape, 10)
    bt = 0.9
    M = np.diag(a2.ravel()) + bt * graph_laplacian3_dense(*shape)
    dense = np.linalg.solve(M, rhs.ravel())
    assert np.allclose(alg1_3d.z_solve3(a2, rhs, bt).ravel(), dense, rtol=1e-10, atol=1e-12)
    assert np.allclose(alg1_3d.z_solve3(a2, rhs, bt, "dense").ravel(), dense, rtol=1e-10, atol=1e-12)


def _noisy_volume(seed=21, nz=3, n=8):
    acq = ph.acquisition("small")
    tab = model.Tables(acq.low, acq.high)
    rng = np.random.default_rng(seed)
    Z = 7.45 + 5 * (rng.random((nz, n, n)) > 0.7)
    rho = 1.0 + 0.5 * (rng.random((nz, n, n)) > 0.8)
    muL = model.mu_hat(rho, Z, 60.0) * (1 + 0.02 * rng.standard_normal((nz, n, n)))
    muH = model.mu_hat(rho, Z, 90.0) * (1 + 0.02 * rng.standard_normal((nz, n, n)))
    return muL, muH, tab


def test_one_slice_equals_2d_oracle():
    """A volume of one slice: dz = 0, so every step and the whole solve equal
    the 2-D oracle's."""
    muL, muH, tab = _noisy_volume(nz=1, n=10)
    prm = alg1.Params(iters=8)
    a = alg1_3d.solve3(muL, muH, tab, prm)
    b = alg1.solve(muL[0], muH[0], tab, prm)
    for key in ("f1", "f2", "rhoe", "zt"):
        assert np.allclose(a[key][0], b[key], rtol=1e-9, atol=1e-11), key


def test_identical_slices_give_the_2d_solution_on_each():
    """A volume whose slices are all the same image: dz of every iterate is 0
    (the updates are shift-invariant across slices), so each slice equals the
    2-D solution of that image."""
    muL, muH, tab = _noisy_volume(nz=1, n=10, seed=22)
    vL, vH = np.repeat(muL, 4, axis=0), np.repeat(muH, 4, axis=0)
    prm = alg1.Params(iters=6)
    a = alg1_3d.solve3(vL, vH, tab, prm)
    b = alg1.solve(muL[0], muH[0], tab, prm)
    for key in ("f1", "f2", "rhoe", "zt"):
        for k in range(4):
            assert np.allclose(a[key][k], b[key], rtol=1e-9, atol=1e-11), (key, k)


def test_slices_couple_through_dz():
    """Two different slices: with the 3-D regulariser the solution of a slice
    depends on its neighbour (the 2-D solve of each slice alone differs)."""
    muL, muH, tab = _noisy_volume(nz=2, n=8, seed=23)
    prm = alg1.Params(iters=4)
    a = alg1_3d.solve3(muL, muH, tab, prm)
    b0 = alg1.solve(muL[0], muH[0], tab, prm)
    assert not np.allclose(a["f1"][0], b0["f1"], rtol=1e-6, atol=1e-9)


def _is_minimiser(J, x, seed, eps=1e-4, trials=6):
    rng = np.random.default_rng(seed)
    J0 = J(x)
    for _ in range(trials):
        d = rng.standard_normal(x.shape)
        jp, jm = J(x + eps * d), J(x - eps * d)
        curv = jp + jm - 2 * J0
        assert curv > 0
        assert abs(jp - jm) < 1e-5 * curv + 1e-10 * abs(J0)


def test_block_updates_minimise_their_subproblems():
    """Each update of iterate3 minimises its own subproblem over the volume
    (eq. obj_sub_f, obj_sub_rho, obj_sub_z with the third difference), by
    random two-sided perturbations."""
    muL, muH, tab = _noisy_volume()
    st = alg1.init_state(muL, muH, tab)
    beta, lam = 0.05, 0.01
    new, hvw = alg1_3d.iterate3(st, beta, beta, lam, muL, muH, tab)
    _is_minimiser(lambda f1: alg1_3d.sub_objective_f3(f1, st["f2"], st, hvw["f1"], hvw["f2"], beta, muL, muH, tab),
                  new["f1"], 1)
    _is_minimiser(lambda f2: alg1_3d.sub_objective_f3(st["f1"], f2, st, hvw["f1"], hvw["f2"], beta, muL, muH, tab),
                  new["f2"], 2)
    m1, m2 = alg1.synthesize(new["f1"], new["f2"], tab)
    _is_minimiser(lambda r: alg1_3d.sub_objective_rho3(r, m1, m2, hvw["rhoe"], beta, tab), new["rhoe"], 3)
    _is_minimiser(lambda z: alg1_3d.sub_objective_z3(z, m1, m2, hvw["zt"], beta, tab), new["zt"], 4)


def test_uniform_material_is_fixed_point():
    acq = ph.acquisition("small")
    tab = model.Tables(acq.low, acq.high)
    muL = np.full((3, 6, 8), model.mu_hat(1.3, 9.0, 60.0))
    muH = np.full((3, 6, 8), model.mu_hat(1.3, 9.0, 90.0))
    st = alg1_3d.solve3(muL, muH, tab, alg1.Params(iters=30))
    assert np.allclose(st["rhoe"], 1.3, rtol=1e-10)
    assert np.allclose(st["Z"], 9.0, rtol=1e-10)


def test_objective3_terms():
    """The relaxed objective over a volume: zero relaxation and L0 terms with
    the triples taken as the gradients of an all-kept state's maps give
    lambda times the voxels with a nonzero gradient; the data terms equal the
    2-D oracle's slice by slice."""
    muL, muH, tab = _noisy_volume(nz=2, n=6, seed=24)
    st = alg1.init_state(muL, muH, tab)
    hvw = {g: alg1_3d.hard_threshold3(st[g], 0.0)[:3] for g in ("f1", "f2", "rhoe", "zt")}
    t = alg1_3d.objective3(st, hvw, 0.3, 0.01, muL, muH, tab)
    assert t["relax"] == 0.0
    nnz = sum(int(np.count_nonzero(sum(np.abs(x) for x in alg1_3d.forward_diff3(st[g])) != 0))
              for g in ("f1", "f2", "rhoe", "zt"))
    assert t["nnz"] == nnz and abs(t["l0"] - 0.01 * nnz) < 1e-12
    for key in ("fid_L", "fid_H", "mod_1", "mod_2"):
        per = 0.0
        for k in range(2):
            sk = {g: st[g][k] for g in ("f1", "f2", "rhoe", "zt")}
            zero = np.zeros_like(muL[k])
            per += alg1.objective(sk, {g: (zero, zero) for g in sk}, 0.3, 0.01, muL[k], muH[k], tab)[key]
        assert abs(t[key] - per) <= 1e-12 * max(1.0, abs(per)), key
