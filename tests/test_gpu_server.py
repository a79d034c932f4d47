"""Serving engine (continuous batching): requests of different sizes, iteration
counts and parameters arrive while others run; each result is bit-identical
to the same request solved alone, and the HBM budget gates admission."""
import numpy as np
import pytest

from oracle import model
from synthetic import phantoms as ph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rc():
    from paper_2308_01290_gb300 import build_lib
    build_lib.build()
    from paper_2308_01290_gb300 import recon
    return recon


def request(rc, k, n, iters, lam):
    acq = ph.acquisition("small")
    P = ph.small_phantom(50 + k, n=n)
    L = (model.mu_mm(P["rhoe"], P["Z"], 60.0) + 4e-4 * ph.normal_field((n, n), 60 + k)).astype(np.float32)
    H = (model.mu_mm(P["rhoe"], P["Z"], 90.0) + 4e-4 * ph.normal_field((n, n), 70 + k)).astype(np.float32)
    p = rc.default_params(low=acq.low, high=acq.high, iters=iters, lam=lam, beta0=2 * lam)
    return rc.geometry(n, n), p, L, H


def alone(rc, g, p, L, H):
    s = rc.Solver(g, p)
    s.set_data(L, H)
    s.step(p.iters)
    Z, R, _, _ = s.get_host()
    return Z[0], R[0]


def test_mixed_arrivals_equal_alone(rc):
    reqs = [request(rc, k, n, it, lm) for k, (n, it, lm) in
            enumerate([(64, 12, 1e-2), (128, 20, 5e-3), (96, 8, 2e-2), (128, 15, 1e-2), (80, 10, 1e-2)])]
    srv = rc.Server(max_slots=3, max_nx=128, max_ny=128)
    tickets = [srv.submit(*reqs[0]), srv.submit(*reqs[1])]
    out = {}
    step = 0
    while len(out) < len(reqs):
        if step == 3:
            tickets.append(srv.submit(*reqs[2]))
        if step == 5:
            tickets.append(srv.submit(*reqs[3]))
            tickets.append(srv.submit(*reqs[4]))   # waits for a free slot (3 slots)
        srv.step(2)
        for i, t in enumerate(tickets):
            if i not in out:
                r = srv.poll(t)
                if r is not None:
                    out[i] = r
        step += 1
        assert step < 200
    for i, (g, p, L, H) in enumerate(reqs):
        Z, R, res = out[i]
        assert res.status == 0 and res.iters == p.iters
        assert res.latency_ms >= res.queue_ms >= 0
        Za, Ra = alone(rc, g, p, L, H)
        assert np.array_equal(Z, Za) and np.array_equal(R, Ra), i
    st = srv.stats()
    assert st["active"] == 0 and st["queued"] == 0 and st["footprint"] == 0


def test_budget_serialises_admission(rc):
    reqs = [request(rc, 10 + k, 64, 6, 1e-2) for k in range(3)]
    one = 19 * 64 * 64 * 4 + 6 * 64 * 48 * 4   # one 64^2 solve (fields + spectra)
    srv = rc.Server(max_slots=3, max_nx=64, max_ny=64, hbm_budget_bytes=1.5 * one)
    ts = [srv.submit(*r) for r in reqs]
    srv.step(0)
    st = srv.stats()
    assert st["active"] == 1 and st["queued"] == 2
    done = {}
    for _ in range(100):
        srv.step(3)
        assert srv.stats()["active"] <= 1
        for i, t in enumerate(ts):
            if i not in done:
                r = srv.poll(t)
                if r is not None:
                    done[i] = r
        if len(done) == 3:
            break
    assert len(done) == 3
    for i, (g, p, L, H) in enumerate(reqs):
        Za, Ra = alone(rc, g, p, L, H)
        assert np.array_equal(done[i][0], Za) and np.array_equal(done[i][1], Ra)


def test_rejects_oversize_and_unknown(rc):
    srv = rc.Server(max_slots=1, max_nx=64, max_ny=64)
    g, p, L, H = request(rc, 0, 128, 5, 1e-2)
    with pytest.raises(rc.ReconError):
        srv.submit(g, p, L, H)
    assert rc.lib.recon_poll(srv.h, 12345, None, None, None) == -1   # RECON_EINVAL: unknown ticket


def test_rejects_invalid_parameters_at_submission(rc):
    """recon_submit checks a request's parameters and geometry as
    recon_init_batch does, so a bad request is refused before it can join a
    step that other requests share, and nothing is queued."""
    srv = rc.Server(max_slots=1, max_nx=64, max_ny=64)
    g, _, L, H = request(rc, 1, 64, 5, 1e-2)
    acq = ph.acquisition("small")
    base = dict(low=acq.low, high=acq.high)
    for kw in (dict(lam=-1.0), dict(beta0=0.0), dict(tau=-1.0), dict(iters=-1), dict(cg_max_iters=-1),
               dict(cg_tol=-1.0), dict(pcg_kernel=4), dict(e1_kev=50.0, e2_kev=50.0)):
        with pytest.raises(rc.ReconError):
            srv.submit(g, rc.default_params(**base, **kw), L, H)
    assert srv.stats()["queued"] == 0


def test_rejects_sinogram_beyond_fbp_limits_and_keeps_stepping(rc):
    """A sinogram request whose rows are too long for the FBP's shared-memory
    tables (4000 bins) fits the slot's sinogram capacity, so only the FBP
    limits can refuse it: recon_submit must do so, before it is queued,
    while the solves in flight keep stepping to their results."""
    acq = ph.acquisition("small", n=32)
    srv = rc.Server(max_slots=2, max_nx=64, max_ny=64, max_views=64, max_bins=4000)
    g, p, L, H = request(rc, 2, 64, 6, 1e-2)
    t = srv.submit(g, p, L, H)
    srv.step(2)
    bad = rc.geometry(acq.nx, acq.ny, acq.pixel_mm, 40, 4000, acq.sid_mm, acq.sdd_mm, 0.05)
    lo = np.zeros(40 * 4000, np.float32)
    with pytest.raises(rc.ReconError):
        srv.submit(bad, rc.default_params(low=acq.low, high=acq.high, iters=4), lo, lo)
    assert srv.stats()["queued"] == 0
    res = None
    for _ in range(20):
        srv.step(2)
        res = srv.poll(t)
        if res is not None:
            break
    assert res is not None and res[2].status == 0
    Za, Ra = alone(rc, g, p, L, H)
    assert np.array_equal(res[0], Za) and np.array_equal(res[1], Ra)
