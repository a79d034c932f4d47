"""Fan-beam input stage in FP64 (oracle; test infrastructure only).

The paper works on reconstructed DECT image pairs (Sec. III) and prints no
projector.  The data-fidelity path through sinograms uses a ray-driven
fan-beam forward projector A and its matched backprojector A^T; synthetic
scans are turned into the paper's image-domain inputs by flat-detector
fan-beam FBP.  Geometry (reading R14):

* image: nx x ny pixels of ``pixel_mm``, centred on the isocentre; pixel
  (row j, column i) has centre x = (i - (nx-1)/2) p, y = (j - (ny-1)/2) p;
* view k: source S = sid (cos t, sin t), t = start + arc k / n_views, central
  ray e_c = -(cos t, sin t), flat detector at distance sdd from the source
  with axis e_u = (-sin t, cos t); bin b centre u_b = (b - (n_bins-1)/2) bin_mm;
* A: Joseph's method -- along the dominant axis the ray is sampled once per
  pixel column (or row), linear interpolation between the two neighbouring
  pixels across it (zero outside the grid), times the step length
  p |r| / max(|r_x|, |r_y|);
* A^T: the same weights scattered back (the exact transpose);
* FBP: rays rescaled to the isocentre plane (s = u sid/sdd), cosine weight
  sid / sqrt(sid^2 + s^2), Ram-Lak ramp (h(0) = 1/(4 ds^2),
  h(odd n) = -1/(pi n ds)^2), pixel-driven backprojection with weight
  1/U^2, U = (sid - x.(cos t, sin t)) / sid, linear interpolation, and a
  factor 1/2 for the full 360 degree scan.

Pins: <A x, y> = <x, A^T y>; Joseph line integrals of a Gaussian blob against
their closed form; FBP of a uniform disc returns its value; the noiseless
polyenergetic scan of a Gaussian blob of one material equals
-ln sum_b w_b exp(-mu(E_b) chord) on the analytic chords, and the Kramers
weights follow their law (tests/test_oracle_ct.py).
"""
from __future__ import annotations

import numpy as np

from . import model


def _rays(geom):
    """Source points and unit directions for every (view, bin) ray."""
    nv, nb = geom["n_views"], geom["n_bins"]
    t = geom.get("start_rad", 0.0) + geom.get("arc_rad", 2 * np.pi) * np.arange(nv) / nv
    c, s = np.cos(t), np.sin(t)
    sid, sdd = geom["sid_mm"], geom["sdd_mm"]
    u = (np.arange(nb) - (nb - 1) / 2.0) * geom["bin_mm"]
    Sx = (sid * c)[:, None] * np.ones((1, nb))
    Sy = (sid * s)[:, None] * np.ones((1, nb))
    Px = Sx - sdd * c[:, None] - u[None, :] * s[:, None]
    Py = Sy - sdd * s[:, None] + u[None, :] * c[:, None]
    rx, ry = Px - Sx, Py - Sy
    return Sx.ravel(), Sy.ravel(), rx.ravel(), ry.ravel()


def _joseph_samples(geom):
    """Yield (ray index, pixel flat index, weight) triples of Joseph's method."""
    nx, ny, p = geom["nx"], geom["ny"], geom["pixel_mm"]
    Sx, Sy, rx, ry = _rays(geom)
    xmaj = np.abs(rx) >= np.abs(ry)
    out = []
    idx = np.nonzero(xmaj)[0]
    if idx.size:
        step = p * np.hypot(rx[idx], ry[idx]) / np.abs(rx[idx])
        for i in range(nx):
            xc = (i - (nx - 1) / 2.0) * p
            t = (xc - Sx[idx]) / rx[idx]
            y = Sy[idx] + t * ry[idx]
            jf = y / p + (ny - 1) / 2.0
            j0 = np.floor(jf).astype(np.int64)
            w1 = jf - j0
            for jj, ww in ((j0, 1.0 - w1), (j0 + 1, w1)):
                ok = (jj >= 0) & (jj < ny)
                out.append((idx[ok], jj[ok] * nx + i, (ww * step)[ok]))
    idx = np.nonzero(~xmaj)[0]
    if idx.size:
        step = p * np.hypot(rx[idx], ry[idx]) / np.abs(ry[idx])
        for j in range(ny):
            yc = (j - (ny - 1) / 2.0) * p
            t = (yc - Sy[idx]) / ry[idx]
            x = Sx[idx] + t * rx[idx]
            i_f = x / p + (nx - 1) / 2.0
            i0 = np.floor(i_f).astype(np.int64)
            w1 = i_f - i0
            for ii, ww in ((i0, 1.0 - w1), (i0 + 1, w1)):
                ok = (ii >= 0) & (ii < nx)
                out.append((idx[ok], j * nx + ii[ok], (ww * step)[ok]))
    return out


def project(img, geom):
    """A img: line integrals, shape (n_views, n_bins)."""
    img = np.asarray(img, dtype=np.float64).ravel()
    nrays = geom["n_views"] * geom["n_bins"]
    sino = np.zeros(nrays)
    for ray, pix, w in _joseph_samples(geom):
        sino += np.bincount(ray, weights=w * img[pix], minlength=nrays)
    return sino.reshape(geom["n_views"], geom["n_bins"])


def backproject(sino, geom):
    """A^T sino: the exact transpose of ``project``, shape (ny, nx)."""
    sino = np.asarray(sino, dtype=np.float64).ravel()
    npx = geom["nx"] * geom["ny"]
    img = np.zeros(npx)
    for ray, pix, w in _joseph_samples(geom):
        img += np.bincount(pix, weights=w * sino[ray], minlength=npx)
    return img.reshape(geom["ny"], geom["nx"])


def ramp_kernel(n_bins, ds):
    """Ram-Lak taps h(n), n = -(n_bins-1) .. n_bins-1."""
    n = np.arange(-(n_bins - 1), n_bins)
    h = np.zeros(n.shape)
    h[n == 0] = 1.0 / (4.0 * ds * ds)
    odd = (n % 2) != 0
    h[odd] = -1.0 / (np.pi * n[odd] * ds) ** 2
    return h


def fbp(sino, geom):
    """Flat-detector fan-beam FBP of a full 360 degree scan, image (ny, nx)."""
    sino = np.asarray(sino, dtype=np.float64)
    nv, nb = sino.shape
    nx, ny, p = geom["nx"], geom["ny"], geom["pixel_mm"]
    sid, sdd = geom["sid_mm"], geom["sdd_mm"]
    ds = geom["bin_mm"] * sid / sdd
    s = (np.arange(nb) - (nb - 1) / 2.0) * ds
    weighted = sino * (sid / np.sqrt(sid * sid + s * s))[None, :]
    h = ramp_kernel(nb, ds)
    q = np.empty_like(weighted)
    for k in range(nv):
        q[k] = ds * np.convolve(weighted[k], h)[nb - 1:2 * nb - 1]
    t = geom.get("start_rad", 0.0) + geom.get("arc_rad", 2 * np.pi) * np.arange(nv) / nv
    dt = geom.get("arc_rad", 2 * np.pi) / nv
    x = (np.arange(nx) - (nx - 1) / 2.0) * p
    y = (np.arange(ny) - (ny - 1) / 2.0) * p
    X, Y = np.meshgrid(x, y)
    img = np.zeros((ny, nx))
    for k in range(nv):
        c, sn = np.cos(t[k]), np.sin(t[k])
        L = sid - (X * c + Y * sn)
        U = L / sid
        sp_ = sid * (-X * sn + Y * c) / L
        bf = sp_ / ds + (nb - 1) / 2.0
        b0 = np.floor(bf).astype(np.int64)
        w1 = bf - b0
        val = np.zeros_like(bf)
        for bb, ww in ((b0, 1.0 - w1), (b0 + 1, w1)):
            ok = (bb >= 0) & (bb < nb)
            val[ok] += ww[ok] * q[k, bb[ok]]
        img += val / (U * U)
    return 0.5 * dt * img


def geometry(acq):
    """Geometry dict from a synthetic.phantoms.Acquisition."""
    return dict(nx=acq.nx, ny=acq.ny, pixel_mm=acq.pixel_mm, n_views=acq.n_views, n_bins=acq.n_bins,
                sid_mm=acq.sid_mm, sdd_mm=acq.sdd_mm, bin_mm=acq.bin_mm, start_rad=0.0, arc_rad=2 * np.pi)


def simulate(Z, rhoe, acq, seed=None):
    """Noisy (seed) or noiseless (seed=None) -log sinograms of both arms.

    Line integrals of mu(E) follow from two projections, A(rho_e z) and
    A(rho_e), because mu(E)/S = rho_e (P(E) z + KN(E)) is linear in them.
    Expected counts I0 sum_b w_b exp(-S (P(E_b) A(rho_e z) + KN(E_b) A(rho_e)));
    Poisson counts floored at 0.5 before the log (reading R14).
    """
    geom = geometry(acq)
    zt = model.ztilde_from_z(Z)
    A1 = project(rhoe * zt, geom)
    A2 = project(rhoe, geom)
    rng = np.random.default_rng(seed) if seed is not None else None
    out = []
    for spec in (acq.low, acq.high):
        E, w = model.spectrum_bins(spec)
        lam = np.zeros_like(A1)
        for Eb, wb in zip(E, w):
            lam += wb * np.exp(-model.S_MM * (model.photo_coeff(Eb) * A1 + model.klein_nishina_barn(Eb) * A2))
        lam *= acq.i0
        if rng is None:
            counts = lam
        else:
            counts = rng.poisson(lam).astype(np.float64)
        out.append(-np.log(np.maximum(counts, 0.5) / acq.i0))
    return out[0], out[1]


def images_from_phantom(Z, rhoe, acq, seed=None):
    """(mu_L, mu_H) images in 1/mm by FBP of simulated sinograms."""
    geom = geometry(acq)
    sL, sH = simulate(Z, rhoe, acq, seed)
    return fbp(sL, geom), fbp(sH, geom), (sL, sH)
