"""GPU parity of the fan-beam input stage (projector A, transpose A^T, FBP,
scan simulation) against the FP64 oracle, through the C ABI.

FP32 tolerances: the marching index start + i * slope carries ~1e-7 relative
rounding of an O(n) index, and sums of O(n) samples add ~n * 6e-8; both stay
below 1e-5 of the sinogram's magnitude for n <= 128.  The ramp filter sums
n_bins alternating terms into a smaller result, so FBP is held to 1e-4 of
the image's magnitude."""
import numpy as np
import pytest
import torch

from oracle import ct, model
from synthetic import phantoms as ph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rc():
    from paper_2308_01290_gb300 import build_lib
    build_lib.build()
    from paper_2308_01290_gb300 import recon
    return recon


def geom_dict(nx=64, ny=56, nv=60, nb=80):
    return dict(nx=nx, ny=ny, pixel_mm=1.0, n_views=nv, n_bins=nb, sid_mm=300.0, sdd_mm=450.0,
                bin_mm=1.5 * max(nx, ny) / nb * 1.1, start_rad=0.2, arc_rad=2 * np.pi)


def to_rc(rc, g):
    return rc.geometry(g["nx"], g["ny"], g["pixel_mm"], g["n_views"], g["n_bins"], g["sid_mm"], g["sdd_mm"],
                       g["bin_mm"], g["start_rad"], g["arc_rad"])


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


@pytest.mark.parametrize("shape", [(64, 56, 60, 80), (33, 47, 17, 29), (128, 128, 180, 192)])
def test_project_matches_oracle(rc, shape):
    g = geom_dict(*shape)
    img = ph.random_field((g["ny"], g["nx"]), 1, 0, 1)
    sino = torch.zeros(g["n_views"] * g["n_bins"], device="cuda")
    x = dev(img)
    rc.project(to_rc(rc, g), 1, x, sino)
    torch.cuda.synchronize()
    ref = ct.project(img.astype(np.float32).astype(np.float64), g)
    got = sino.cpu().numpy().reshape(ref.shape)
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()


def test_backproject_adjoint_and_oracle(rc):
    g = geom_dict()
    x = ph.random_field((g["ny"], g["nx"]), 2)
    y = ph.random_field((g["n_views"], g["n_bins"]), 3)
    xs, ys = dev(x), dev(y)
    Ax = torch.zeros(g["n_views"] * g["n_bins"], device="cuda")
    Aty = torch.zeros(g["nx"] * g["ny"], device="cuda")
    G = to_rc(rc, g)
    rc.project(G, 1, xs, Ax)
    rc.backproject(G, 1, ys, Aty)
    torch.cuda.synchronize()
    Ax, Aty = Ax.cpu().double().numpy(), Aty.cpu().double().numpy()
    lhs = float(np.dot(Ax, y.astype(np.float32).astype(np.float64).ravel()))
    rhs = float(np.dot(x.astype(np.float32).astype(np.float64).ravel(), Aty))
    assert abs(lhs - rhs) <= 1e-5 * (np.abs(Ax).sum() * np.abs(y).max())
    ref = ct.backproject(y.astype(np.float32).astype(np.float64), g).ravel()
    assert np.abs(Aty - ref).max() <= 1e-5 * np.abs(ref).max()


def test_batched_projection_equals_single(rc):
    g = geom_dict(48, 40, 30, 50)
    imgs = np.stack([ph.random_field((40, 48), s) for s in range(3)]).astype(np.float32)
    out = torch.zeros(3 * 30 * 50, device="cuda")
    G = to_rc(rc, g)
    rc.project(G, 3, dev(imgs), out)
    for s in range(3):
        one = torch.zeros(30 * 50, device="cuda")
        rc.project(G, 1, dev(imgs[s]), one)
        assert torch.equal(one, out[s * 1500:(s + 1) * 1500])


def test_fbp_matches_oracle(rc):
    acq = ph.acquisition("small")
    g = ct.geometry(acq)
    P = ph.small_phantom(4)
    sL, _ = ct.simulate(P["Z"], P["rhoe"], acq, seed=4)
    img = torch.zeros(acq.nx * acq.ny, device="cuda")
    rc.fbp(rc.geometry_from_acq(acq), 1, dev(sL), img)
    torch.cuda.synchronize()
    ref = ct.fbp(sL.astype(np.float32).astype(np.float64), g)
    got = img.cpu().double().numpy().reshape(ref.shape)
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()


def test_fbp_batch_of_slices_equals_one_by_one(rc):
    """11 slices in one call (a group of 8 and a ragged group of 3 in the
    backprojection) give each slice's single-slice result bit for bit; the
    first and last also match the oracle."""
    acq = ph.acquisition("small")
    g = ct.geometry(acq)
    G = rc.geometry_from_acq(acq)
    n, nr, npx = 11, acq.n_views * acq.n_bins, acq.nx * acq.ny
    sinos = []
    for k in range(n):
        P = ph.small_phantom(40 + k)
        sinos.append(ct.simulate(P["Z"], P["rhoe"], acq, seed=40 + k)[0])
    allv = dev(np.concatenate([s_.ravel() for s_ in sinos]))
    img = torch.zeros(n * npx, device="cuda")
    rc.fbp(G, n, allv, img)
    for k in range(n):
        one = torch.zeros(npx, device="cuda")
        rc.fbp(G, 1, allv[k * nr:(k + 1) * nr], one)
        assert torch.equal(one, img[k * npx:(k + 1) * npx]), k
    torch.cuda.synchronize()
    for k in (0, n - 1):
        ref = ct.fbp(sinos[k].astype(np.float32).astype(np.float64), g)
        got = img[k * npx:(k + 1) * npx].cpu().double().numpy().reshape(ref.shape)
        assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max(), k


@pytest.mark.parametrize("nb", [83, 191, 736])
def test_fbp_interleaved_groups_equal_one_by_one(rc, nb):
    """17 slices of random sinograms: two full groups of 8, filtered
    slice-interleaved with a sliding window of 8 outputs per thread, and one
    slice filtered row by row.  Bin counts whose last window is ragged (83,
    191: not a multiple of 8) and whose tap count is not a multiple of 4 (83:
    41 taps, 191: 95) give each slice's single-slice result bit for bit."""
    g = geom_dict(nx=72, ny=64, nv=48, nb=nb)
    G = to_rc(rc, g)
    n, nr, npx = 17, g["n_views"] * nb, g["nx"] * g["ny"]
    allv = dev(np.concatenate([ph.random_field((g["n_views"], nb), 70 + k).ravel() for k in range(n)]))
    img = torch.zeros(n * npx, device="cuda")
    rc.fbp(G, n, allv, img)
    for k in range(n):
        one = torch.zeros(npx, device="cuda")
        rc.fbp(G, 1, allv[k * nr:(k + 1) * nr], one)
        assert torch.equal(one, img[k * npx:(k + 1) * npx]), k


@pytest.mark.parametrize("kind", ["small", "clinical"])
def test_simulate_noiseless_matches_oracle(rc, kind):
    acq = ph.acquisition(kind, n=64)
    P = ph.small_phantom(5, n=64)
    sL, sH = ct.simulate(P["Z"], P["rhoe"], acq, seed=None)
    p = rc.default_params(low=acq.low, high=acq.high)
    lo = torch.zeros(acq.n_views * acq.n_bins, device="cuda")
    hi = torch.zeros_like(lo)
    rc.simulate(rc.geometry_from_acq(acq), p, 1, dev(P["Z"]), dev(P["rhoe"]), None, acq.i0, lo, hi)
    torch.cuda.synchronize()
    for got, ref in ((lo, sL), (hi, sH)):
        got = got.cpu().double().numpy().reshape(ref.shape)
        assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()
