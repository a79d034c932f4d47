"""recon_fbp_noalloc: the FBP entry point for callers that cannot allocate
device memory at call time (a real-time loop that forbids allocation after
start-up, or a service that reserves all its device memory up front).  It
uses a fixed scratch array inside the library instead of allocating one.

Checked through the C ABI against recon_fbp, which allocates its scratch:
the two run the same kernels on the same inputs, so two calls in a row with
different sinograms must give recon_fbp's images bit for bit, both for a
group of slices (the multi-slice backprojection) and for one slice (the
single-slice one); a request above the scratch size must be refused.  This
file runs last (its name sorts last) and also passes alone in a fresh
process."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2308_01290_gb300 import build_lib
    build_lib.build()
    from paper_2308_01290_gb300 import recon
    return recon, torch


@pytest.mark.parametrize("n", [3, 1])
def test_fbp_noalloc_matches_fbp_twice(env, n):
    rc, torch = env
    from synthetic import phantoms as ph
    acq = ph.acquisition("small")
    g = rc.geometry_from_acq(acq)
    per = acq.n_views * acq.n_bins
    assert n * per <= rc.FBP_NOALLOC_MAX
    for call in range(2):
        rng = np.random.default_rng(100 + 10 * n + call)
        sino = torch.from_numpy(rng.uniform(0.0, 4.0, size=n * per).astype(np.float32)).cuda()
        ref = torch.empty(n * acq.nx * acq.ny, device="cuda")
        out = torch.full_like(ref, float("nan"))
        rc.fbp(g, n, sino, ref)
        rc.fbp_noalloc(g, n, sino, out)
        torch.cuda.synchronize()
        ref_h, out_h = ref.cpu().numpy(), out.cpu().numpy()
        assert np.isfinite(out_h).all()
        assert np.array_equal(out_h, ref_h), (n, call, np.abs(out_h - ref_h).max())


def test_fbp_noalloc_rejects_oversize(env):
    rc, torch = env
    g = rc.geometry(64, 64, 1.0, 1000, 1000, 1000.0, 1500.0, 1.0)
    n = rc.FBP_NOALLOC_MAX // (1000 * 1000) + 1
    sino = torch.zeros(1, device="cuda")
    img = torch.zeros(1, device="cuda")
    with pytest.raises(rc.ReconError):
        rc.fbp_noalloc(g, n, sino, img)
