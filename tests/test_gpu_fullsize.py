"""Parity at the full size of the volume workload, in the launch
configuration the bench times: 160 slices of 512^2 in one batch (one launch
per kernel over all slices, multigrid-preconditioned Z^m PCG), two iterations
of the 150-iteration beta schedule, from image pairs the oracle's model makes
(mono 60/90 keV, Gaussian noise).

Properties over every slice: finite maps, and each slice's Z^m PCG stopped
at the relative residual 1e-6 (or its step cap).  Sampled slices (first,
middle, last) against the FP64 oracle run one by one on the same inputs:
mean |dZ| <= 0.01 and mean |d rho_e| <= 1e-3 over the body."""
import numpy as np
import pytest

from oracle import alg1, model
from synthetic import phantoms as ph

pytestmark = pytest.mark.gpu

N_SLICES, N, ITERS_SCHEDULE, ITERS_RUN = 160, 512, 150, 2


@pytest.fixture(scope="module")
def rc():
    from paper_2308_01290_gb300 import build_lib
    build_lib.build()
    from paper_2308_01290_gb300 import recon
    return recon


def test_volume_full_size_matches_oracle_on_sampled_slices(rc):
    acq = ph.acquisition("volume")
    tab = model.Tables(acq.low, acq.high)
    V = ph.volume_phantom(1000, n_slices=N_SLICES, n=N)
    lo = np.empty((N_SLICES, N, N), np.float32)
    hi = np.empty((N_SLICES, N, N), np.float32)
    for k in range(N_SLICES):
        Z, rho = V["Z"][k].astype(np.float64), V["rhoe"][k].astype(np.float64)
        lo[k] = model.mu_mm(rho, Z, 60.0) + 4e-4 * ph.normal_field((N, N), 3000 + k)
        hi[k] = model.mu_mm(rho, Z, 90.0) + 4e-4 * ph.normal_field((N, N), 4000 + k)
    kappa = (1e5 / 2e-2) ** (1.0 / ITERS_SCHEDULE)
    g = rc.geometry(N, N)
    p = rc.default_params(low=acq.low, high=acq.high, iters=ITERS_RUN, kappa=kappa)
    s = rc.Solver([g] * N_SLICES, [p] * N_SLICES)
    s.set_data(lo, hi)
    stats = s.step(ITERS_RUN, stats=True)
    Z, R, _, _ = s.get_host()
    s.close()
    for k, st in enumerate(stats):
        assert st.k == ITERS_RUN, k
        assert st.cg_rel_residual <= 1e-6 * 1.0001 or st.cg_iters == p.cg_max_iters, (k, st.cg_rel_residual)
        assert np.isfinite(Z[k]).all() and np.isfinite(R[k]).all(), k
    for k in (0, N_SLICES // 2, N_SLICES - 1):
        ref = alg1.solve_mm(lo[k], hi[k], tab, alg1.Params(iters=ITERS_RUN, kappa=kappa))
        body = V["rhoe"][k] >= 0.1
        dZ = np.abs(Z[k] - ref["Z"])[body]
        dr = np.abs(R[k] - ref["rhoe"])[body]
        print(f"slice {k}: mean|dZ| {dZ.mean():.3e} p99.9 {np.percentile(dZ, 99.9):.3e}, "
              f"mean|drho| {dr.mean():.3e} p99.9 {np.percentile(dr, 99.9):.3e}")
        assert dZ.mean() <= 0.01 and dr.mean() <= 1e-3, k
