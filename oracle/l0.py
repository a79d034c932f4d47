"""Gradient-L0 smoothing of Sec. II-C in FP64 (oracle; test infrastructure only).

min_g ||g - g~||^2 + lambda C(g) through the auxiliary split (eq. L0_aux,
L0_unconstraint): alternately (h, v) by eq. sol_hv and g by the FFT closed
form of eq. L0_sub_g, with beta raised by kappa until beta_max.

Pins (tests/test_oracle_alg1.py): piecewise-constant images with jumps above
sqrt(lambda/beta0) are fixed points; at fixed beta the relaxed objective
eq. L0_unconstraint never increases.
"""
from __future__ import annotations

import numpy as np

from .alg1 import adjoint_diff, count_nonzero_gradients, fft_solve, forward_diff, hard_threshold


def relaxed_objective(g, g_noisy, h, v, beta, lam):
    """eq. L0_unconstraint."""
    dx, dy = forward_diff(g)
    return float(np.sum((g - g_noisy) ** 2) + lam * count_nonzero_gradients(h, v)
                 + beta * (np.sum((dx - h) ** 2) + np.sum((dy - v) ** 2)))


def l0_step(g, g_noisy, beta, lam):
    """(h, v) from eq. sol_hv, then g from eq. L0_sub_g.  Returns (g, h, v)."""
    h, v, _ = hard_threshold(g, lam / beta)
    g_new = fft_solve(g_noisy + beta * adjoint_diff(h, v), 1.0, beta)
    return g_new, h, v


def l0_smooth(g_noisy, lam, beta0=None, beta_max=1e5, kappa=2.0, trace=False):
    g = np.array(g_noisy, dtype=np.float64)
    beta = 2.0 * lam if beta0 is None else beta0
    tr = []
    while beta < beta_max:
        g, h, v = l0_step(g, g_noisy, beta, lam)
        if trace:
            tr.append(relaxed_objective(g, g_noisy, h, v, beta, lam))
        beta *= kappa
    return (g, tr) if trace else g
