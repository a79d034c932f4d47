"""GPU parity of the sinogram-domain f updates (domain 1) against the FP64
oracle (oracle/modeb.py), through the C ABI, on a 64^2 slice with 90 views x
96 bins (mono 60/90 keV, Poisson noise at I0 = 1e5).

Per operator, from inputs the oracle side writes (the seeded sinograms and a
state written into the fields): the data images t_k, the Gram images
A^T A f_k, the two right-hand sides, and the f updates after the GPU's CG to a
relative residual of 1e-6 against the oracle's exact solve, all to a
relative 1e-5 of their magnitude.  Whole solve: mean |dZ| <= 0.01
and mean |d rho_e| <= 1e-3 over the body."""
import numpy as np
import pytest

from oracle import alg1, ct, model, modeb
from synthetic import phantoms as ph

pytestmark = pytest.mark.gpu
LAM = 1e-2


@pytest.fixture(scope="module")
def rc():
    from paper_2308_01290_gb300 import build_lib
    build_lib.build()
    from paper_2308_01290_gb300 import recon
    return recon


@pytest.fixture(scope="module")
def case():
    acq = ph.acquisition("small", n=64)
    P = ph.small_phantom(3, n=64)
    sL, sH = ct.simulate(P["Z"], P["rhoe"], acq, seed=11)
    geom = ct.geometry(acq)
    tab = model.Tables(acq.low, acq.high)
    return dict(acq=acq, P=P, sL=sL.astype(np.float32), sH=sH.astype(np.float32), geom=geom, tab=tab,
                g=modeb.gamma(geom))


def close(got, ref, tol, what):
    err = float(np.max(np.abs(got - ref)))
    scale = float(np.max(np.abs(ref)))
    print(what, f"max error {err:.3e} of scale {scale:.3e}")
    assert err <= tol * scale, what


def stored(x):
    return np.asarray(x, np.float32).astype(np.float64)


def test_f_update_operators_match_oracle(rc, case):
    acq, geom, tab, g = case["acq"], case["geom"], case["tab"], case["g"]
    p = rc.default_params(low=acq.low, high=acq.high, domain=1)
    s = rc.Solver(rc.geometry_from_acq(acq), p)
    s.set_data(case["sL"], case["sH"])
    t = modeb.data_images(case["sL"], case["sH"], geom, tab, g)
    close(s.read("MUL"), t[0], 1e-5, "t_1")
    close(s.read("MUH"), t[1], 1e-5, "t_2")
    shape = (acq.ny, acq.nx)
    st = dict(f1=stored(0.3 * ph.random_field(shape, 21)), f2=stored(1.0 + 0.2 * ph.random_field(shape, 22)),
              rhoe=stored(1.0 + 0.1 * ph.random_field(shape, 23)), zt=stored(1.0 + 0.1 * ph.random_field(shape, 24)))
    for name, key in (("F1", "f1"), ("F2", "f2"), ("RHO", "rhoe"), ("Z", "zt")):
        s.write(name, st[key])
    s.op("THRESH_RHS")
    close(s.read("A2"), modeb.backproject(modeb.project(st["f1"], geom), geom), 1e-5, "A^T A f1")
    close(s.read("RHS_Z"), modeb.backproject(modeb.project(st["f2"], geom), geom), 1e-5, "A^T A f2")
    beta = s.scalars()["beta"]
    hv = alg1.thresholds(st, LAM / beta, np.float32)
    b = [modeb.rhs(k, st, hv["f1" if k == 0 else "f2"], beta, t, geom, tab, g) for k in (0, 1)]
    close(s.read("RHS_F1"), b[0], 1e-5, "rhs f1")
    close(s.read("RHS_F2"), b[1], 1e-5, "rhs f2")
    s.op("SOLVE_F")
    for k, name in ((0, "F1"), (1, "F2")):
        ref = modeb.f_solve(b[k], k, beta, geom, tab, g, st["f1" if k == 0 else "f2"])
        close(s.read(name), ref, 1e-5, f"f{k + 1} after CG")
    s.close()


def test_sinogram_domain_solve_matches_oracle(rc, case):
    acq, geom, tab = case["acq"], case["geom"], case["tab"]
    iters = 12
    p = rc.default_params(low=acq.low, high=acq.high, domain=1, iters=iters)
    s = rc.Solver(rc.geometry_from_acq(acq), p)
    s.set_data(case["sL"], case["sH"])
    s.step(iters)
    Z, rho, _, _ = [x[0] for x in s.get_host()]
    s.close()
    ref = modeb.solve(case["sL"], case["sH"], geom, tab, alg1.Params(iters=iters))
    body = case["P"]["rhoe"] >= 0.1
    dZ = np.abs(Z - ref["Z"])[body]
    dr = np.abs(rho - ref["rhoe"])[body]
    print("domain 1 solve", dict(mean_dZ=float(dZ.mean()), p999_dZ=float(np.percentile(dZ, 99.9)),
                                 median_dZ=float(np.median(dZ)), n_dZ_gt_01=int((dZ > 0.1).sum()),
                                 mean_drho=float(dr.mean()), p999_drho=float(np.percentile(dr, 99.9))))
    assert dZ.mean() <= 0.01 and dr.mean() <= 1e-3


# --- domain 2: polyenergetic fidelity linearised by Gauss-Newton -------------

@pytest.fixture(scope="module")
def poly_case():
    acq = ph.acquisition("clinical", n=64)
    P = ph.clinical_phantom(5, n=64)
    sL, sH = ct.simulate(P["Z"], P["rhoe"], acq, seed=12)
    nL, nH = ct.simulate(P["Z"], P["rhoe"], acq, seed=None)
    geom = ct.geometry(acq)
    tab = model.Tables(acq.low, acq.high)
    return dict(acq=acq, P=P, sL=sL.astype(np.float32), sH=sH.astype(np.float32), nL=nL.astype(np.float32),
                nH=nH.astype(np.float32), geom=geom, tab=tab, g=modeb.gamma(geom))


def test_gauss_newton_operators_match_oracle(rc, poly_case):
    """Kramers 80 / 140 kVp arms (2 mm Al; 0.4 mm Sn on the high arm), 64^2,
    90 views x 92 bins: from a state written into the fields, the data images
    A^T v_k / gamma, the weighted Gram images A^T (W_kk o A f_k), the two
    right-hand sides and the f updates against the oracle's Gauss-Newton
    terms and exact solves.  The per-ray terms are FP32 spectrum sums whose
    v_k cancel part of their two products: 1e-4 of the magnitude."""
    c = poly_case
    acq, geom, tab, g = c["acq"], c["geom"], c["tab"], c["g"]
    p = rc.default_params(low=acq.low, high=acq.high, domain=2)
    s = rc.Solver(rc.geometry_from_acq(acq), p)
    s.set_data(c["sL"], c["sH"])
    shape = (acq.ny, acq.nx)
    st = dict(f1=stored(0.05 + 0.05 * ph.random_field(shape, 31)), f2=stored(0.9 + 0.1 * ph.random_field(shape, 32)),
              rhoe=stored(1.0 + 0.1 * ph.random_field(shape, 33)), zt=stored(1.0 + 0.1 * ph.random_field(shape, 34)))
    for name, key in (("F1", "f1"), ("F2", "f2"), ("RHO", "rhoe"), ("Z", "zt")):
        s.write(name, st[key])
    s.op("THRESH_RHS")
    l1, l2 = modeb.project(st["f1"], geom), modeb.project(st["f2"], geom)
    W11, W22, W12, v1, v2 = modeb.gn_terms(l1, l2, c["sL"], c["sH"], tab)
    close(s.read("MUL"), modeb.backproject(v1, geom) / g, 1e-4, "A^T v1 / gamma")
    close(s.read("MUH"), modeb.backproject(v2, geom) / g, 1e-4, "A^T v2 / gamma")
    close(s.read("A2"), modeb.backproject(W11 * l1, geom), 1e-5, "A^T W11 A f1")
    close(s.read("RHS_Z"), modeb.backproject(W22 * l2, geom), 1e-5, "A^T W22 A f2")
    beta = s.scalars()["beta"]
    hv = alg1.thresholds(st, LAM / beta, np.float32)
    b = [modeb.rhs_gn(k, st, hv["f1" if k == 0 else "f2"], beta, v, geom, tab, g) for k, v in ((0, v1), (1, v2))]
    close(s.read("RHS_F1"), b[0], 1e-4, "rhs f1")
    close(s.read("RHS_F2"), b[1], 1e-4, "rhs f2")
    s.op("SOLVE_F")
    for k, name, W in ((0, "F1", W11), (1, "F2", W22)):
        ref = modeb.f_solve(b[k], k, beta, geom, tab, g, st["f1" if k == 0 else "f2"], W=W)
        close(s.read(name), ref, 1e-4, f"f{k + 1} after CG")
    s.close()


def test_gauss_newton_solve_matches_oracle(rc, poly_case):
    c = poly_case
    acq, geom, tab = c["acq"], c["geom"], c["tab"]
    iters = 10
    p = rc.default_params(low=acq.low, high=acq.high, domain=2, iters=iters)
    s = rc.Solver(rc.geometry_from_acq(acq), p)
    s.set_data(c["sL"], c["sH"])
    s.step(iters)
    Z, rho, _, _ = [x[0] for x in s.get_host()]
    s.close()
    ref = modeb.solve_gn(c["sL"], c["sH"], geom, tab, alg1.Params(iters=iters))
    body = c["P"]["rhoe"] >= 0.1
    dZ = np.abs(Z - ref["Z"])[body]
    dr = np.abs(rho - ref["rhoe"])[body]
    print("domain 2 solve", dict(mean_dZ=float(dZ.mean()), p999_dZ=float(np.percentile(dZ, 99.9)),
                                 median_dZ=float(np.median(dZ)), n_dZ_gt_01=int((dZ > 0.1).sum()),
                                 mean_drho=float(dr.mean()), p999_drho=float(np.percentile(dr, 99.9))))
    assert dZ.mean() <= 0.01 and dr.mean() <= 1e-3


def test_gauss_newton_removes_beam_hardening_bias(rc, poly_case):
    """Noiseless polyenergetic sinograms of the 64^2 clinical phantom: the
    linear sinogram fidelity (domain 1) keeps the beam-hardening bias of the
    spectrum-weighted model, the Gauss-Newton fidelity (domain 2) fits the
    polyenergetic data and lands closer to the truth in rho_e and Z."""
    c = poly_case
    acq = c["acq"]
    body = c["P"]["rhoe"] >= 0.1
    err = {}
    for dom in (1, 2):
        p = rc.default_params(low=acq.low, high=acq.high, domain=dom, iters=20)
        s = rc.Solver(rc.geometry_from_acq(acq), p)
        s.set_data(c["nL"], c["nH"])
        s.step(20)
        Z, rho, _, _ = [x[0] for x in s.get_host()]
        s.close()
        err[dom] = (float(np.abs(rho - c["P"]["rhoe"])[body].mean()), float(np.abs(Z - c["P"]["Z"])[body].mean()))
    print("mean |d rho_e|, |d Z| against the truth: linear", err[1], "Gauss-Newton", err[2])
    assert err[2][0] < err[1][0] and err[2][1] < err[1][1]


@pytest.mark.parametrize("domain", [1, 2])
def test_comparator_in_sinogram_domains(rc, poly_case, domain):
    """In the sinogram domains the loaded fields hold the f updates' data
    images, so recon_direct forms the FBP pair again: its maps equal, bit for
    bit, those of an image-domain handle fed the same sinograms, before and
    after iterations, on the host and device paths."""
    import torch
    c = poly_case
    acq = c["acq"]
    g = rc.geometry_from_acq(acq)
    s0 = rc.Solver(g, rc.default_params(low=acq.low, high=acq.high, domain=0, iters=4))
    s0.set_data(c["sL"], c["sH"])
    Z0, R0 = [a[0] for a in s0.direct()]
    s0.close()
    s = rc.Solver(g, rc.default_params(low=acq.low, high=acq.high, domain=domain, iters=4))
    s.set_data(c["sL"], c["sH"])
    Z1, R1 = [a[0] for a in s.direct()]
    assert np.array_equal(Z1, Z0) and np.array_equal(R1, R0)
    s.step(4)
    dZ = torch.empty(acq.nx * acq.ny, device="cuda")
    dR = torch.empty(acq.nx * acq.ny, device="cuda")
    s.direct(Z=dZ, rhoe=dR, on_device=True)
    torch.cuda.synchronize()
    assert np.array_equal(dZ.cpu().numpy().reshape(Z0.shape), Z0)
    assert np.array_equal(dR.cpu().numpy().reshape(R0.shape), R0)
    s.close()
