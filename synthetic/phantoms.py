"""Seeded synthetic phantoms and acquisition settings for dual-energy CT.

This module is the only code shared by the CPU oracle side (tests) and the
CUDA side (tests, bench).  It holds shapes, material values (effective atomic
number Z and relative electron density rho_e) and scanner settings only.  It
contains none of the method's arithmetic: no attenuation model, no projection,
no reconstruction.  Everything is drawn from ``numpy.random.default_rng(seed)``
so a (kind, size, seed) triple fixes the phantom bit for bit.

The paper's scans (Gammex 467 / 1472 phantoms and a patient, Sec. III) are not
available; these phantoms stand in for them: a water body with circular or
ellipsoidal inserts whose (Z, rho_e) span soft tissue, lung and bone.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

WATER = (7.45, 1.0)
BONE = (13.0, 1.7)
LUNG = (7.5, 0.25)
AIR_Z = 1.0  # Z assigned outside the body (rho_e = 0 there, so it never attenuates)


@dataclass(frozen=True)
class Spectrum:
    """One energy arm.  kind 'mono' uses ``kev``; kind 'kramers' uses
    ``kvp`` with 1 keV bins from 10 keV, and the listed filters
    (name, Z, rho_e, thickness_mm)."""

    kind: str
    kev: float = 0.0
    kvp: float = 0.0
    filters: tuple = ()


AL_2MM = ("Al", 13.0, 2.34, 2.0)
SN_04MM = ("Sn", 50.0, 5.55, 0.4)


@dataclass(frozen=True)
class Acquisition:
    nx: int
    ny: int
    pixel_mm: float
    n_views: int
    n_bins: int
    sid_mm: float
    sdd_mm: float
    bin_mm: float
    low: Spectrum
    high: Spectrum
    i0: float
    iters: int


def fan_bin_mm(nx: int, pixel_mm: float, n_bins: int, sid_mm: float, sdd_mm: float) -> float:
    """Detector pitch that makes the detector span the image width at the
    isocentre (magnification sdd/sid)."""
    return (sdd_mm / sid_mm) * nx * pixel_mm / n_bins


def acquisition(kind: str, n: int | None = None, i0: float | None = None,
                iters: int | None = None) -> Acquisition:
    """Scanner settings of the named workload.

    kind:
      'small'   128^2, 1 mm, mono 60/90 keV, 180 views, 192 bins, I0=1e5, 50 it
      'clinical' 512^2, 1 mm, Kramers 80/140 kVp (2 mm Al, +0.4 mm Sn on 140),
                720 views, 736 bins, I0=1e5, 100 it
      'uneven'  n^2 (n in 256..512), mono 60/90, views 720 n/512, bins 736 n/512
      'volume'  512^2 slices, mono 60/90, 720 views, 736 bins, I0=5e4, 150 it
    """
    sid, sdd = 1000.0, 1500.0
    mono = (Spectrum("mono", kev=60.0), Spectrum("mono", kev=90.0))
    if kind == "small":
        n = n or 128
        views, bins = 180 * n // 128, 192 * n // 128
        lo, hi = mono
        a_i0, a_it = 1e5, 50
    elif kind == "clinical":
        n = n or 512
        views, bins = 720 * n // 512, 736 * n // 512
        lo = Spectrum("kramers", kvp=80.0, filters=(AL_2MM,))
        hi = Spectrum("kramers", kvp=140.0, filters=(AL_2MM, SN_04MM))
        a_i0, a_it = 1e5, 100
    elif kind == "uneven":
        assert n is not None
        views, bins = 720 * n // 512, 736 * n // 512
        lo, hi = mono
        a_i0, a_it = 1e5, 100
    elif kind == "volume":
        n = n or 512
        views, bins = 720 * n // 512, 736 * n // 512
        lo, hi = mono
        a_i0, a_it = 5e4, 150
    else:
        raise ValueError(kind)
    return Acquisition(nx=n, ny=n, pixel_mm=1.0, n_views=views, n_bins=bins, sid_mm=sid,
                       sdd_mm=sdd, bin_mm=fan_bin_mm(n, 1.0, bins, sid, sdd), low=lo, high=hi,
                       i0=float(i0 if i0 is not None else a_i0),
                       iters=int(iters if iters is not None else a_it))


def pixel_centres(nx: int, ny: int, pixel_mm: float):
    """x (column) and y (row) centre coordinates in mm; the grid is centred on
    the isocentre and row j has y = (j - (ny-1)/2) * pixel."""
    x = (np.arange(nx) - (nx - 1) / 2.0) * pixel_mm
    y = (np.arange(ny) - (ny - 1) / 2.0) * pixel_mm
    return np.meshgrid(x, y)


def _place_discs(rng, n_ins, semi_a, semi_b, r_lo, r_hi, margin):
    """Rejection-sample non-overlapping discs inside an ellipse (pixel units)."""
    discs = []
    tries = 0
    while len(discs) < n_ins:
        tries += 1
        if tries > 20000:
            raise RuntimeError("could not place inserts")
        r = rng.uniform(r_lo, r_hi)
        cx = rng.uniform(-semi_a, semi_a)
        cy = rng.uniform(-semi_b, semi_b)
        # whole disc (plus margin) inside the ellipse: test a ring of points
        ang = np.linspace(0, 2 * np.pi, 24, endpoint=False)
        px = cx + (r + margin) * np.cos(ang)
        py = cy + (r + margin) * np.sin(ang)
        if np.any((px / semi_a) ** 2 + (py / semi_b) ** 2 >= 1.0):
            continue
        if any(np.hypot(cx - qx, cy - qy) < r + qr + margin for qx, qy, qr in discs):
            continue
        discs.append((cx, cy, r))
    return discs


def disc_phantom(n: int, seed: int, *, n_inserts: int = 8, semi_px=(56.0, 44.0),
                 radius_px=(6.0, 12.0), z_range=(5.5, 20.0), rho_range=(0.2, 1.9),
                 fixed=(), margin=2.0) -> dict:
    """Water ellipse with circular inserts on an n x n grid.

    The default arguments are the 128^2 small workload; ``scaled_disc_phantom``
    rescales them to other sizes.  ``fixed`` lists (Z, rho_e) pairs given to
    the first inserts (e.g. bone-like and lung-like); the rest draw
    Z ~ U(z_range), rho_e ~ U(rho_range).  Returns float64 maps 'Z' and
    'rhoe' (rho_e = 0 and Z = 1 in air) and the insert list.
    """
    rng = np.random.default_rng(seed)
    a, b = semi_px
    discs = _place_discs(rng, n_inserts, a, b, radius_px[0], radius_px[1], margin=margin)
    c = (n - 1) / 2.0
    jj, ii = np.mgrid[0:n, 0:n]
    x = ii - c
    y = jj - c
    Z = np.full((n, n), AIR_Z)
    rho = np.zeros((n, n))
    body = (x / a) ** 2 + (y / b) ** 2 < 1.0
    Z[body], rho[body] = WATER
    inserts = []
    for k, (cx, cy, r) in enumerate(discs):
        if k < len(fixed):
            zk, rk = fixed[k]
        else:
            zk = rng.uniform(*z_range)
            rk = rng.uniform(*rho_range)
        m = (x - cx) ** 2 + (y - cy) ** 2 < r * r
        Z[m], rho[m] = zk, rk
        inserts.append(dict(cx=cx, cy=cy, r=r, Z=zk, rhoe=rk))
    return dict(Z=Z, rhoe=rho, inserts=inserts, body=body)


def small_phantom(seed: int, n: int = 128) -> dict:
    """128^2 workload: 56x44 px water ellipse, 8 inserts r in [6,12] px
    (scaled with n; fewer inserts below 64 px)."""
    s = n / 128.0
    return disc_phantom(n, seed, n_inserts=8 if n >= 64 else 3, semi_px=(56.0 * s, 44.0 * s),
                        radius_px=(6.0 * s, 12.0 * s), margin=2.0 * min(1.0, s))


def clinical_phantom(seed: int, n: int = 512, pixel_mm: float = 1.0) -> dict:
    """512^2 workload: 400x300 mm body ellipse, 16 inserts r in [8,20] px, the
    first bone-like (13, 1.7) and the second lung-like (7.5, 0.25)."""
    s = n / 512.0
    return disc_phantom(n, seed, n_inserts=16, semi_px=(200.0 / pixel_mm * s, 150.0 / pixel_mm * s),
                        radius_px=(8.0 * s, 20.0 * s), fixed=(BONE, LUNG))


def uneven_sizes(seed: int, n_slices: int = 64, choices=(256, 320, 384, 448, 512)) -> list:
    rng = np.random.default_rng(seed)
    return [int(v) for v in rng.choice(np.array(choices), size=n_slices)]


def volume_phantom(seed: int, n_slices: int = 160, n: int = 512, n_inserts: int = 24) -> dict:
    """Stack of n_slices n x n slices (1 mm spacing): a 400x300 mm elliptic
    water cylinder with ellipsoidal inserts (in-plane radius U[8,20] px,
    spanning 5-40 slices).  Returns float32 'Z', 'rhoe' of shape
    (n_slices, n, n)."""
    rng = np.random.default_rng(seed)
    s = n / 512.0
    a, b = 200.0 * s, 150.0 * s
    c = (n - 1) / 2.0
    jj, ii = np.mgrid[0:n, 0:n]
    x = ii - c
    y = jj - c
    body = (x / a) ** 2 + (y / b) ** 2 < 1.0
    Z = np.full((n_slices, n, n), AIR_Z, dtype=np.float32)
    rho = np.zeros((n_slices, n, n), dtype=np.float32)
    Z[:, body] = WATER[0]
    rho[:, body] = WATER[1]
    ells = []
    tries = 0
    while len(ells) < n_inserts and tries < 50000:
        tries += 1
        r = rng.uniform(8.0 * s, 20.0 * s)
        span = rng.uniform(5.0, 40.0)
        cz = rng.uniform(0, n_slices - 1)
        cx = rng.uniform(-a, a)
        cy = rng.uniform(-b, b)
        ang = np.linspace(0, 2 * np.pi, 24, endpoint=False)
        if np.any(((cx + (r + 2) * np.cos(ang)) / a) ** 2 + ((cy + (r + 2) * np.sin(ang)) / b) ** 2 >= 1):
            continue
        clash = False
        for e in ells:
            if abs(cz - e["cz"]) < (span + e["span"]) / 2 + 1 and np.hypot(cx - e["cx"], cy - e["cy"]) < r + e["r"] + 2:
                clash = True
                break
        if clash:
            continue
        k = len(ells)
        if k == 0:
            zk, rk = BONE
        elif k == 1:
            zk, rk = LUNG
        else:
            zk, rk = rng.uniform(5.5, 20.0), rng.uniform(0.2, 1.9)
        ells.append(dict(cx=cx, cy=cy, cz=cz, r=r, span=span, Z=zk, rhoe=rk))
    for e in ells:
        hz = e["span"] / 2.0
        z0 = max(0, int(np.ceil(e["cz"] - hz)))
        z1 = min(n_slices - 1, int(np.floor(e["cz"] + hz)))
        for sl in range(z0, z1 + 1):
            t = (sl - e["cz"]) / hz
            rr = e["r"] * np.sqrt(max(0.0, 1.0 - t * t))
            if rr <= 0.5:
                continue
            m = (x - e["cx"]) ** 2 + (y - e["cy"]) ** 2 < rr * rr
            Z[sl][m] = e["Z"]
            rho[sl][m] = e["rhoe"]
    return dict(Z=Z, rhoe=rho, inserts=ells, body=body)


def uniform_phantom(n: int, Z: float, rhoe: float, ny: int | None = None) -> dict:
    ny = ny or n
    return dict(Z=np.full((ny, n), float(Z)), rhoe=np.full((ny, n), float(rhoe)))


def piecewise_constant(nx: int, ny: int, seed: int, n_levels: int = 4, lo=0.0, hi=1.0) -> np.ndarray:
    """Rectangles of constant value on a constant background (float64)."""
    rng = np.random.default_rng(seed)
    g = np.full((ny, nx), rng.uniform(lo, hi))
    for _ in range(n_levels):
        x0 = rng.integers(0, max(1, nx - 2))
        y0 = rng.integers(0, max(1, ny - 2))
        w = rng.integers(2, max(3, nx // 2))
        h = rng.integers(2, max(3, ny // 2))
        g[y0:y0 + h, x0:x0 + w] = rng.uniform(lo, hi)
    return g


def random_field(shape, seed: int, lo=-1.0, hi=1.0) -> np.ndarray:
    return np.random.default_rng(seed).uniform(lo, hi, size=shape)


def normal_field(shape, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(size=shape)
