"""Pins of the oracle's monoenergetic images, two-step comparator and image
quality metrics (oracle/iqa.py; Sec. III and eq. mac_E1/E2)."""
import numpy as np
import pytest

from oracle import alg1, iqa, model
from synthetic import phantoms as ph


@pytest.mark.parametrize("kind", ["small", "clinical"])
def test_mono_images_of_uniform_materials_equal_the_model(kind):
    """f from the decomposition of a noiseless uniform material gives that
    material's attenuation at every energy: the photoelectric / Compton model
    is spanned by the two basis materials."""
    acq = ph.acquisition(kind, n=32)
    tab = model.Tables(acq.low, acq.high)
    for Z, rho in ((10.0, 1.3), (7.45, 1.0), (13.0, 1.7), (6.0, 0.3)):
        muL = np.full((3, 4), model.effective(model.mu_hat(rho, Z, tab.arms[0][0]), tab.arms[0][1]))
        muH = np.full((3, 4), model.effective(model.mu_hat(rho, Z, tab.arms[1][0]), tab.arms[1][1]))
        st = alg1.init_state(muL, muH, tab)
        for E in (30.0, 45.0, 70.0, 100.0, 140.0):
            mono = iqa.mono_image(st["f1"], st["f2"], E, tab)
            ref = model.mu_mm(rho, Z, E)
            assert np.allclose(mono, ref, rtol=1e-10, atol=0), (Z, rho, E)


def test_two_step_recovers_uniform_materials():
    acq = ph.acquisition("small", n=16)
    tab = model.Tables(acq.low, acq.high)
    for Z, rho in ((12.0, 1.5), (7.45, 1.0), (5.8, 0.9)):
        muL = np.full((4, 5), model.mu_mm(rho, Z, 60.0))
        muH = np.full((4, 5), model.mu_mm(rho, Z, 90.0))
        Zr, Rr, f1, f2 = iqa.two_step(muL, muH, tab)
        assert np.allclose(Zr, Z, rtol=1e-10) and np.allclose(Rr, rho, rtol=1e-10)


def test_psnr_nmad_closed_forms():
    rng = np.random.default_rng(4)
    ref = rng.uniform(0.5, 2.0, (20, 30))
    ref[3, 4] = 2.5                                   # the peak
    x = ref + 0.01                                    # MSE = 1e-4
    assert iqa.psnr(x, ref) == pytest.approx(10 * np.log10(2.5 ** 2 / 1e-4), rel=1e-12)
    y = ref * 1.03                                    # |y - ref| = 0.03 |ref|
    assert iqa.nmad(y, ref) == pytest.approx(0.03, rel=1e-12)
    mask = np.zeros(ref.shape, bool)
    mask[5:10, 5:12] = True
    z = ref.copy()
    z[~mask] += 100.0                                 # outside the mask: ignored
    z[mask] += 0.02
    assert iqa.psnr(z, ref, mask) == pytest.approx(10 * np.log10(ref[mask].max() ** 2 / 4e-4), rel=1e-12)
    assert iqa.nmad(z, ref, mask) == pytest.approx(0.02 * mask.sum() / ref[mask].sum(), rel=1e-12)


def test_ssim_identity_and_constant_windows():
    rng = np.random.default_rng(5)
    a = rng.uniform(0, 1, (24, 20))
    assert iqa.ssim(a, a) == pytest.approx(1.0, abs=1e-14)
    # constant windows: no variance, so a window's SSIM is (2 c1 c2 + C1) / (c1^2 + c2^2 + C1)
    ref = np.full((16, 16), 2.0)
    ref[15, 15] = 1.0                                 # L = 1; only the window centred at (10, 10) sees it
    x = np.full((16, 16), 1.5)
    x[15, 15] = 1.0
    C1 = (0.01 * 1.0) ** 2
    closed = (2 * 1.5 * 2.0 + C1) / (1.5 ** 2 + 2.0 ** 2 + C1)
    per = _brute_windows(x, ref)
    assert len(per) == 36
    assert np.allclose(per[:-1], closed, rtol=1e-10, atol=0)
    assert iqa.ssim(x, ref) == pytest.approx(np.mean(per), rel=1e-9)


def _brute_ssim(x, y, L=None):
    return float(np.mean(_brute_windows(x, y, L)))


def _brute_windows(x, y, L=None):
    """SSIM of every window (row-major over window centres), with explicit
    loops over the 2-D Gaussian weights."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    if L is None:
        L = y.max() - y.min()
    c1, c2 = (0.01 * L) ** 2, (0.03 * L) ** 2
    r, sg = 5, 1.5
    w = np.array([[np.exp(-(i * i + j * j) / (2 * sg * sg)) for i in range(-r, r + 1)] for j in range(-r, r + 1)])
    w /= w.sum()
    ny, nx = x.shape
    vals = []
    for cy in range(r, ny - r):
        for cx in range(r, nx - r):
            mx = my = sxx = syy = sxy = 0.0
            for j in range(-r, r + 1):
                for i in range(-r, r + 1):
                    wt = w[j + r, i + r]
                    a, b = x[cy + j, cx + i], y[cy + j, cx + i]
                    mx += wt * a
                    my += wt * b
                    sxx += wt * a * a
                    syy += wt * b * b
                    sxy += wt * a * b
            sxx -= mx * mx
            syy -= my * my
            sxy -= mx * my
            vals.append(((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2)))
    return np.array(vals)


def test_ssim_matches_brute_force_windows():
    rng = np.random.default_rng(6)
    ref = ph.piecewise_constant(17, 15, 3) + 0.05 * rng.standard_normal((15, 17))
    x = ref + 0.1 * rng.standard_normal(ref.shape)
    assert iqa.ssim(x, ref) == pytest.approx(_brute_ssim(x, ref), rel=1e-12)
    w = iqa.gaussian_window()
    assert len(w) == 11 and abs(w.sum() - 1) < 1e-15 and np.argmax(w) == 5
