"""The comparison outputs of Sec. III on the GPU, through the C ABI, against
the FP64 oracle (oracle/iqa.py): the two-step image-based comparator
(recon_direct), monoenergetic images at any energy (recon_mono) and the
image-quality metrics PSNR, NMAD and SSIM (recon_iqa).

Tolerances: the comparator is FP64 arithmetic per pixel on the stored image
pair, rounded to the map precision, so FP32 maps agree to 1e-5 of their
magnitude; the FP64 path's maps agree to the float rounding of the outputs
(the C ABI returns float maps), 1e-7.  Monoenergetic images are one product
sum per pixel from the same f: 1e-5 (FP32), 1e-7 (FP64, float outputs).  The
metrics are FP64 sums on both sides, which differ only in summation order,
1e-9."""
import numpy as np
import pytest

from oracle import alg1, iqa, model
from synthetic import phantoms as ph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2308_01290_gb300 import build_lib
    build_lib.build()
    from paper_2308_01290_gb300 import recon
    return recon, torch


def _images(n, seed, noise=4e-4):
    P = ph.small_phantom(seed, n=n)
    L = (model.mu_mm(P["rhoe"], P["Z"], 60.0) + noise * ph.normal_field((n, n), seed + 1)).astype(np.float32)
    H = (model.mu_mm(P["rhoe"], P["Z"], 90.0) + noise * ph.normal_field((n, n), seed + 2)).astype(np.float32)
    return P, L, H


def _close(got, ref, tol):
    scale = max(np.abs(ref).max(), 1e-30)
    err = np.abs(np.asarray(got, np.float64) - ref).max() / scale
    assert err <= tol, err


@pytest.mark.parametrize("precision", [1, 0])
def test_direct_is_iteration_zero_and_matches_oracle(env, precision):
    rc, _ = env
    acq = ph.acquisition("small")
    sizes = (128, 96, 63)
    imgs = [_images(n, 10 + k) for k, n in enumerate(sizes)]
    p = rc.default_params(low=acq.low, high=acq.high, iters=5, precision=precision)
    s = rc.Solver([rc.geometry(n, n) for n in sizes], [p] * len(sizes))
    s.set_data(np.concatenate([L.ravel() for _, L, _ in imgs]), np.concatenate([H.ravel() for _, _, H in imgs]))
    Zd, Rd = s.direct()
    Z0, R0, _, _ = s.get_host()
    tab = model.Tables(acq.low, acq.high)
    tol = 1e-5 if precision == 1 else 1e-7
    fdt = np.float32 if precision == 1 else np.float64
    for k, (P, L, H) in enumerate(imgs):
        assert np.array_equal(Zd[k], Z0[k]) and np.array_equal(Rd[k], R0[k]), k
        # the oracle from the image pair as the handle stores it
        uL = (L.astype(np.float64) / model.S_MM).astype(fdt).astype(np.float64)
        uH = (H.astype(np.float64) / model.S_MM).astype(fdt).astype(np.float64)
        Zr, Rr, _, _ = iqa.two_step(uL * model.S_MM, uH * model.S_MM, tab)
        _close(Rd[k], Rr, tol)
        _close(Zd[k], Zr, tol)
    # the comparator does not move with the iterations
    s.step(5)
    Zd2, Rd2 = s.direct()
    assert all(np.array_equal(a, b) for a, b in zip(Zd, Zd2))


@pytest.mark.parametrize("precision", [1, 0])
def test_mono_images_match_oracle(env, precision):
    rc, torch = env
    acq = ph.acquisition("small")
    sizes = (128, 80)
    imgs = [_images(n, 20 + k) for k, n in enumerate(sizes)]
    p = rc.default_params(low=acq.low, high=acq.high, iters=6, precision=precision)
    s = rc.Solver([rc.geometry(n, n) for n in sizes], [p] * len(sizes))
    s.set_data(np.concatenate([L.ravel() for _, L, _ in imgs]), np.concatenate([H.ravel() for _, _, H in imgs]))
    s.step(6)
    tab = model.Tables(acq.low, acq.high)
    kev = [40.0, 60.0, 73.5, 120.0]
    host = s.mono(kev)
    tot = sum(n * n for n in sizes)
    ddev = torch.empty(len(kev) * tot, device="cuda")
    s.mono(kev, ddev)
    torch.cuda.synchronize()
    dev = ddev.cpu().numpy()
    tol = 1e-5 if precision == 1 else 1e-7
    for k in range(len(sizes)):
        f1 = s.read("F1", k)
        f2 = s.read("F2", k)
        for e, E in enumerate(kev):
            ref = iqa.mono_image(f1, f2, E, tab)
            _close(host[e][k], ref, tol)
        off = sum(n * n for n in sizes[:k])
        for e in range(len(kev)):
            assert np.array_equal(dev[e * tot + off:e * tot + off + sizes[k] ** 2], host[e][k].ravel())
    big = torch.empty(17 * tot, device="cuda")
    with pytest.raises(rc.ReconError):
        s.mono([60.0] * 17, big)
    with pytest.raises(rc.ReconError):
        s.mono([60.0] * 17)
    with pytest.raises(rc.ReconError):
        s.mono([-1.0])


def test_iqa_metrics_match_oracle(env):
    rc, torch = env
    rng = np.random.default_rng(3)
    n, nx, ny = 3, 70, 45
    ref = np.stack([ph.piecewise_constant(nx, ny, 5 + k) for k in range(n)]).astype(np.float32) + 1.0
    x = (ref + 0.05 * rng.standard_normal(ref.shape)).astype(np.float32)
    mask = np.zeros(ref.shape, np.uint8)
    mask[:, 5:40, 8:60] = 1
    dx, dr = torch.from_numpy(x).cuda(), torch.from_numpy(ref).cuda()
    dm = torch.from_numpy(mask).cuda()
    got = rc.iqa(n, nx, ny, dx, dr, dm)
    got_nomask = rc.iqa(n, nx, ny, dx, dr)
    for k in range(n):
        ps, nm, ss = iqa.metrics(x[k], ref[k], mask[k].astype(bool))
        assert got[k, 0] == pytest.approx(ps, rel=1e-9) and got[k, 1] == pytest.approx(nm, rel=1e-9)
        assert got[k, 2] == pytest.approx(ss, rel=1e-9)
        ps2, nm2, ss2 = iqa.metrics(x[k], ref[k])
        assert got_nomask[k, 0] == pytest.approx(ps2, rel=1e-9) and got_nomask[k, 1] == pytest.approx(nm2, rel=1e-9)
        assert got_nomask[k, 2] == pytest.approx(ss, rel=1e-9)
    same = rc.iqa(1, nx, ny, dr[0], dr[0])
    assert same[0, 2] == pytest.approx(1.0, abs=1e-12) and same[0, 1] == 0.0
    with pytest.raises(rc.ReconError):
        rc.iqa(1, 10, 40, dx, dr)


def test_one_step_beats_two_step_on_the_small_phantom(env):
    """The paper's comparison (Sec. III) on the synthetic 128^2 workload:
    against the truth maps, Algorithm 1 has a higher PSNR and a lower NMAD
    than the two-step image-based method, for rho_e and for Z, inside the
    body."""
    rc, torch = env
    acq = ph.acquisition("small")
    P, L, H = _images(128, 0, noise=8e-4)
    p = rc.default_params(low=acq.low, high=acq.high, iters=acq.iters)
    s = rc.Solver(rc.geometry(128, 128), p)
    s.set_data(L, H)
    Zd, Rd = [a[0] for a in s.direct()]
    s.step(acq.iters)
    Z, R, _, _ = [a[0] for a in s.get_host()]
    body = (P["rhoe"] >= 0.1).astype(np.uint8)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    m = dev(body).to(torch.uint8)
    for name, one, two, truth in (("rho_e", R, Rd, P["rhoe"]), ("Z", Z, Zd, P["Z"])):
        a = rc.iqa(1, 128, 128, dev(one), dev(truth), m)[0]
        b = rc.iqa(1, 128, 128, dev(two), dev(truth), m)[0]
        print(name, "one-step", a, "two-step", b)
        assert a[0] > b[0] and a[1] < b[1], (name, a, b)
