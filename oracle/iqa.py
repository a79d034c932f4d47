"""Monoenergetic images, the two-step comparator and the image-quality
metrics of Sec. III, in FP64 (oracle; test infrastructure only).

* Monoenergetic image at any energy E (eq. mac_E1/E2 at E instead of E1, E2):
  mu(E) = S (f1 mu_hat_1(E) + f2 mu_hat_2(E)), mu_hat_k the model value of
  basis material k (reading R2 for the units).  Because the photoelectric /
  Compton model spans a two-dimensional space in E, two basis materials
  represent every material exactly at every energy.
* Two-step comparator (the image-based method of Sec. III): decomposition
  of the image pair, synthesis at E1, E2 and the closed forms eq. rho_e,
  eq. Z_m, with no regularisation -- the initialisation of Algorithm 1
  (alg1.init_state) followed by the m-th root.
* Image-quality metrics.  The paper reports PSNR, NMAD and SSIM of the Z and
  rho_e maps against the reference maps without printing their definitions;
  the readings (R18):
    PSNR = 10 log10(peak^2 / MSE), peak = max |ref|, MSE the mean squared
           difference, both over the pixels of `mask` (all pixels without);
    NMAD = sum |x - ref| / sum |ref| over the same pixels;
    SSIM = the structural similarity of Wang et al. (2004): for every pixel
           whose 11 x 11 window lies inside the image, with the window's
           normalised Gaussian weights w (sigma 1.5),
             mu_x = sum w x,  s_xx = sum w x^2 - mu_x^2,  s_xy = sum w x y - mu_x mu_y,
             ssim = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_xx + s_yy + C2)),
           C1 = (0.01 L)^2, C2 = (0.03 L)^2, L = max(ref) - min(ref) over the
           image; SSIM is the mean over those pixels.

Pins (tests/test_oracle_iqa.py): monoenergetic images of uniform materials
equal the model at every energy; the comparator recovers noiseless uniform
materials; PSNR and NMAD against closed forms; SSIM is 1 on identical
images, equals its closed form on constant images, and equals a brute-force
window-by-window evaluation on small images.
"""
from __future__ import annotations

import numpy as np

from . import alg1, model

SSIM_RADIUS = 5
SSIM_SIGMA = 1.5
SSIM_K1, SSIM_K2 = 0.01, 0.03


def mono_image(f1, f2, E_kev, tab):
    """mu(E) in 1/mm from the basis fractions (eq. mac_E1/E2 at energy E)."""
    (z1, r1), (z2, r2) = tab.basis
    return model.S_MM * (np.asarray(f1, np.float64) * model.mu_hat(r1, z1, E_kev)
                         + np.asarray(f2, np.float64) * model.mu_hat(r2, z2, E_kev))


def two_step(muL_mm, muH_mm, tab, z_clip=(0.0, 30.0), rho_air=0.1):
    """(Z, rho_e, f1, f2) of the direct image-based method: Algorithm 1's
    initialisation from images in 1/mm, then Z = m-th root of Z^m."""
    st = alg1.init_state(np.asarray(muL_mm, np.float64) / model.S_MM, np.asarray(muH_mm, np.float64) / model.S_MM,
                         tab, z_clip, rho_air)
    return model.z_from_ztilde(st["zt"]), st["rhoe"], st["f1"], st["f2"]


def psnr(x, ref, mask=None):
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    m = np.ones(ref.shape, bool) if mask is None else np.asarray(mask, bool)
    mse = np.mean((x[m] - ref[m]) ** 2)
    peak = np.max(np.abs(ref[m]))
    return float(10.0 * np.log10(peak * peak / mse)) if mse > 0 else float("inf")


def nmad(x, ref, mask=None):
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    m = np.ones(ref.shape, bool) if mask is None else np.asarray(mask, bool)
    return float(np.sum(np.abs(x[m] - ref[m])) / np.sum(np.abs(ref[m])))


def gaussian_window():
    """Normalised 1-D Gaussian weights of the SSIM window (the 2-D window is
    their outer product)."""
    t = np.arange(-SSIM_RADIUS, SSIM_RADIUS + 1, dtype=np.float64)
    g = np.exp(-t * t / (2.0 * SSIM_SIGMA * SSIM_SIGMA))
    return g / g.sum()


def _window_means(img, g):
    """sum over the window of w * img for every pixel whose window fits
    (separable: rows, then columns), shape (ny - 10, nx - 10)."""
    k = len(g)
    ny, nx = img.shape
    rows = np.zeros((ny, nx - k + 1))
    for i, wi in enumerate(g):
        rows += wi * img[:, i:i + nx - k + 1]
    out = np.zeros((ny - k + 1, nx - k + 1))
    for j, wj in enumerate(g):
        out += wj * rows[j:j + ny - k + 1, :]
    return out


def ssim(x, ref):
    x = np.asarray(x, np.float64)
    y = np.asarray(ref, np.float64)
    L = float(y.max() - y.min())
    c1, c2 = (SSIM_K1 * L) ** 2, (SSIM_K2 * L) ** 2
    g = gaussian_window()
    mx, my = _window_means(x, g), _window_means(y, g)
    sxx = _window_means(x * x, g) - mx * mx
    syy = _window_means(y * y, g) - my * my
    sxy = _window_means(x * y, g) - mx * my
    s = ((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2))
    return float(s.mean())


def metrics(x, ref, mask=None):
    """(PSNR, NMAD, SSIM) of x against ref."""
    return psnr(x, ref, mask), nmad(x, ref, mask), ssim(x, ref)
