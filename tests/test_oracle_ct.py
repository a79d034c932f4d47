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


def _gaussian_chord_scan(spec_lo, spec_hi):
    """Noiseless scan of a Gaussian electron-density blob of one material.

    rho_e(r) = rho0 exp(-|r - c|^2 / (2 s^2)) and constant Z, so
    mu(E) = rho_e(r) (Cp Z^m / E^n + KN(E)) S and the line integral of a ray
    at distance d from c is mu_hat_1(E) S rho0 sqrt(2 pi) s exp(-d^2 / (2 s^2)),
    mu_hat_1 the model at (Z, rho_e = 1).  A photon-counting detector behind
    a spectrum of normalised weights w_b then reads
    -ln sum_b w_b exp(-(that line integral at E_b)).
    """
    from oracle import model
    from synthetic import phantoms as ph
    n, pix = 64, 4.0
    acq = ph.Acquisition(nx=n, ny=n, pixel_mm=pix, n_views=12, n_bins=96, sid_mm=1000.0, sdd_mm=1500.0,
                         bin_mm=ph.fan_bin_mm(n, pix, 96, 1000.0, 1500.0), low=spec_lo, high=spec_hi,
                         i0=1e5, iters=1)
    cx, cy, sg, rho0, Zm = 10.0, -6.0, 30.0, 1.4, 12.0
    X, Y = ph.pixel_centres(n, n, pix)
    rho = rho0 * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2 * sg * sg))
    Z = np.full((n, n), Zm)
    sL, sH = ct.simulate(Z, rho, acq, seed=None)
    geom = ct.geometry(acq)
    d = _ray_distance_to(geom, cx, cy)
    chord = rho0 * np.sqrt(2 * np.pi) * sg * np.exp(-d * d / (2 * sg * sg))   # integral of rho_e, mm
    return sL, sH, chord, Zm


def _poly_log(spec, chord, Zm):
    from oracle import model
    E, w = model.spectrum_bins(spec)
    mu1 = model.mu_mm(1.0, Zm, E)                       # 1/mm per unit rho_e, per bin
    return -np.log(np.sum(w[None, None, :] * np.exp(-mu1[None, None, :] * chord[:, :, None]), axis=2))


def test_simulate_polyenergetic_matches_analytic_chords():
    """Kramers arms (80 kVp / 2 mm Al and 140 kVp / 2 mm Al + 0.4 mm Sn):
    the oracle's noiseless -log sinograms equal -ln sum_b w_b exp(-mu(E_b) chord)
    on the analytic line integrals of a Gaussian blob, to the Joseph
    discretisation error (below 0.25 % of the largest value here).  A
    monoenergetic stand-in at the spectrum's mean attenuation (no beam
    hardening) or a missing filter each miss by more than four times that."""
    from oracle import model
    from synthetic import phantoms as ph
    lo = ph.Spectrum("kramers", kvp=80.0, filters=(ph.AL_2MM,))
    hi = ph.Spectrum("kramers", kvp=140.0, filters=(ph.AL_2MM, ph.SN_04MM))
    sL, sH, chord, Zm = _gaussian_chord_scan(lo, hi)
    tol = 2.5e-3
    for got, spec in ((sL, lo), (sH, hi)):
        exact = _poly_log(spec, chord, Zm)
        err = np.abs(got - exact).max() / exact.max()
        assert err < tol, err
        # the pin separates the polyenergetic model from plausible mistakes
        E, w = model.spectrum_bins(spec)
        mono = chord * np.sum(w * model.mu_mm(1.0, Zm, E))          # beam hardening ignored
        assert np.abs(mono - exact).max() / exact.max() > 4 * tol
        unfiltered = _poly_log(ph.Spectrum("kramers", kvp=spec.kvp), chord, Zm)
        assert np.abs(unfiltered - exact).max() / exact.max() > 4 * tol
    Elo, wlo = model.spectrum_bins(lo)
    assert abs(wlo.sum() - 1.0) < 1e-12 and np.all(wlo >= 0)


def test_simulate_mono_is_linear_in_the_chord():
    """Monoenergetic arms: -log of the noiseless counts is mu(E) times the
    line integral, exactly Beer-Lambert."""
    from oracle import model
    from synthetic import phantoms as ph
    lo, hi = ph.Spectrum("mono", kev=60.0), ph.Spectrum("mono", kev=90.0)
    sL, sH, chord, Zm = _gaussian_chord_scan(lo, hi)
    for got, E in ((sL, 60.0), (sH, 90.0)):
        exact = model.mu_mm(1.0, Zm, E) * chord
        assert np.abs(got - exact).max() / exact.max() < 3e-3


def test_kramers_weights_follow_the_unfiltered_law():
    """Without filters the detected weights are (kVp - E)/E on 1 keV bins from
    10 keV, normalised (Kramers' law as read for the acquisition model)."""
    from oracle import model
    from synthetic import phantoms as ph
    E, w = model.spectrum_bins(ph.Spectrum("kramers", kvp=80.0))
    assert E[0] == 10.0 and E[-1] == 79.0 and len(E) == 70
    ref = (80.0 - E) / E
    assert np.allclose(w, ref / ref.sum(), rtol=1e-13)
    # a filter of thickness t multiplies bin b by exp(-mu(E_b) t) before normalising
    Ef, wf = model.spectrum_bins(ph.Spectrum("kramers", kvp=80.0, filters=(ph.AL_2MM,)))
    att = np.exp(-model.mu_mm(2.34, 13.0, E) * 2.0)
    assert np.allclose(wf, ref * att / np.sum(ref * att), rtol=1e-12)
