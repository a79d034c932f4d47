"""Pins of the oracle's fan-beam projector, backprojector and FBP."""
import numpy as np
import pytest

from oracle import ct


def small_geom(nx=32, ny=28, nv=40, nb=48):
    return dict(nx=nx, ny=ny, pixel_mm=1.0, n_views=nv, n_bins=nb, sid_mm=200.0, sdd_mm=300.0,
                bin_mm=1.5 * max(nx, ny) / nb * 1.2, start_rad=0.1, arc_rad=2 * np.pi)


def test_adjoint_identity():
    g = small_geom()
    rng = np.random.default_rng(0)
    x = rng.standard_normal((g["ny"], g["nx"]))
    y = rng.standard_normal((g["n_views"], g["n_bins"]))
    lhs = np.sum(ct.project(x, g) * y)
    rhs = np.sum(x * ct.backproject(y, g))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def _ray_distance_to(geom, cx, cy):
    """Distance from (cx, cy) to each ray, from the geometry as documented:
    source sid (cos t, sin t); detector point source - sdd (cos t, sin t)
    + u (-sin t, cos t)."""
    nv, nb = geom["n_views"], geom["n_bins"]
    out = np.zeros((nv, nb))
    for k in range(nv):
        t = geom["start_rad"] + geom["arc_rad"] * k / nv
        s = np.array([geom["sid_mm"] * np.cos(t), geom["sid_mm"] * np.sin(t)])
        for b in range(nb):
            u = (b - (nb - 1) / 2) * geom["bin_mm"]
            p = s - geom["sdd_mm"] * np.array([np.cos(t), np.sin(t)]) + u * np.array([-np.sin(t), np.cos(t)])
            d = (p - s) / np.linalg.norm(p - s)
            w = np.array([cx, cy]) - s
            out[k, b] = abs(w[0] * d[1] - w[1] * d[0])
    return out


def test_joseph_gaussian_line_integrals():
    """Line integral of a Gaussian blob: sqrt(2 pi) sigma exp(-d^2 / (2 sigma^2))."""
    g = small_geom(48, 40, 24, 64)
    cx, cy, sg = 4.0, -3.0, 4.0
    x = (np.arange(g["nx"]) - (g["nx"] - 1) / 2)
    y = (np.arange(g["ny"]) - (g["ny"] - 1) / 2)
    X, Y = np.meshgrid(x, y)
    img = np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2 * sg * sg))
    d = _ray_distance_to(g, cx, cy)
    exact = np.sqrt(2 * np.pi) * sg * np.exp(-d * d / (2 * sg * sg))
    got = ct.project(img, g)
    assert np.max(np.abs(got - exact)) < 0.01 * exact.max()


def test_fbp_reconstructs_disc_from_analytic_chords():
    """FBP of exact chord lengths 2 mu sqrt(R^2 - d^2) of a uniform disc."""
    g = dict(nx=64, ny=64, pixel_mm=1.0, n_views=360, n_bins=192, sid_mm=500.0, sdd_mm=750.0,
             bin_mm=1.5 * 96 / 192, start_rad=0.0, arc_rad=2 * np.pi)
    R, mu, cx, cy = 20.0, 0.02, 3.0, -2.0
    d = _ray_distance_to(g, cx, cy)
    sino = 2 * mu * np.sqrt(np.clip(R * R - d * d, 0, None))
    img = ct.fbp(sino, g)
    x = (np.arange(64) - 31.5)
    X, Y = np.meshgrid(x, x)
    r = np.hypot(X - cx, Y - cy)
    inner = r < R - 3
    outer = r > R + 3
    assert abs(img[inner].mean() / mu - 1) < 0.01
    assert np.abs(img[inner] / mu - 1).max() < 0.05
    assert np.abs(img[outer]).max() < 0.05 * mu


def test_fbp_of_projected_disc():
    """Projector and FBP together: a pixelised disc comes back with its value."""
    g = dict(nx=64, ny=64, pixel_mm=1.0, n_views=180, n_bins=128, sid_mm=500.0, sdd_mm=750.0,
             bin_mm=1.5 * 64 / 128 * 1.2, start_rad=0.0, arc_rad=2 * np.pi)
    x = (np.arange(64) - 31.5)
    X, Y = np.meshgrid(x, x)
    disc = 0.02 * (np.hypot(X, Y) < 18)
    img = ct.fbp(ct.project(disc, g), g)
    inner = np.hypot(X, Y) < 14
    assert abs(img[inner].mean() / 0.02 - 1) < 0.01
