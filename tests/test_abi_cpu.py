"""CPU-side checks of the C ABI: the library loads and exports every function
declared in include/recon.h; host-only entry points (defaults, model tables)
agree with the oracle's tables.  No GPU compute is called here."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rc():
    from paper_2308_01290_gb300 import build_lib
    build_lib.build()
    from paper_2308_01290_gb300 import recon
    return recon


def declared_functions():
    src = open(os.path.join(ROOT, "include", "recon.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(recon_[a-z_0-9]+)\s*\(", src)))


def test_exports_match_header(rc):
    decl = declared_functions()
    assert len(decl) >= 20
    for name in decl:
        assert hasattr(rc.lib, name), name
    assert set(decl) == set(rc.EXPORTS)


def test_struct_sizes_match_c_layout(rc):
    import ctypes as C
    out = (C.c_int64 * 4)()
    assert rc.lib.recon_abi_sizes(out) == 0
    assert tuple(out) == (C.sizeof(rc.Geometry), C.sizeof(rc.Spectrum), C.sizeof(rc.Params), C.sizeof(rc.Stats))
    p = rc.default_params()
    assert p.iters == 50 and p.precision == 1 and abs(p.lambda_ - 1e-2) < 1e-15


def test_model_tables_match_oracle(rc):
    from oracle import model
    from synthetic import phantoms as ph
    for kind in ("small", "clinical"):
        acq = ph.acquisition(kind, n=128)
        p = rc.default_params(low=acq.low, high=acq.high)
        t = rc.model_tables(p)
        tab = model.Tables(acq.low, acq.high)
        ref = np.concatenate([tab.a.ravel(), tab.b.ravel(), tab.P, tab.psi, [tab.r], tab.c_f, [tab.c_rho],
                              [tab.a_w], [model.S_MM]])
        assert np.allclose(t, ref, rtol=1e-12, atol=0), (kind, t - ref)


def test_strerror(rc):
    assert rc.lib.recon_strerror(-1) == b"invalid argument"
    assert rc.lib.recon_strerror(0) == b"ok"


def test_sinogram_domain_rejects_unsupported_configurations(rc):
    """Validation returns before any device work, so this runs without a GPU."""
    from synthetic import phantoms as ph
    acq = ph.acquisition("small", n=32)
    sino = rc.geometry_from_acq(acq)
    img = rc.geometry_from_acq(acq, image_input=True)
    other = rc.geometry(acq.nx, acq.ny, acq.pixel_mm, acq.n_views + 2, acq.n_bins, acq.sid_mm, acq.sdd_mm,
                        acq.bin_mm)
    p = rc.default_params(low=acq.low, high=acq.high, domain=1)
    bad = [([img], [p]),                                                   # image inputs
           ([sino, other], [p, p]),                                        # two geometries
           ([sino], [rc.default_params(domain=1, precision=0)]),           # FP64
           ([sino], [rc.default_params(domain=1, order=1)]),               # Gauss-Seidel
           ([sino], [rc.default_params(domain=2)])]
    for geoms, params in bad:
        with pytest.raises(rc.ReconError):
            rc.Solver(geoms, params)


def test_input_stage_rejects_bad_arguments_before_device_work(rc):
    """recon_project / backproject / fbp / fbp_noalloc / simulate check their
    arguments and the fan-beam geometry before any device call or
    allocation, so each bad case returns RECON_EINVAL here without a GPU (the
    buffer addresses are never touched)."""
    from synthetic import phantoms as ph
    acq = ph.acquisition("small", n=32)
    good = dict(nx=acq.nx, ny=acq.ny, pixel_mm=acq.pixel_mm, n_views=acq.n_views, n_bins=acq.n_bins,
                sid_mm=acq.sid_mm, sdd_mm=acq.sdd_mm, bin_mm=acq.bin_mm)
    bad_geoms = [dict(good, n_views=0), dict(good, n_bins=0), dict(good, nx=0),
                 dict(good, sdd_mm=acq.sid_mm),                            # detector on the source circle
                 dict(good, pixel_mm=2.0 * acq.sid_mm),                    # image reaches the source
                 dict(good, bin_mm=0.0)]
    buf = 1 << 20   # an address that validation never dereferences
    p = rc.default_params(low=acq.low, high=acq.high)
    calls = [lambda g, n: rc.project(g, n, buf, buf), lambda g, n: rc.backproject(g, n, buf, buf),
             lambda g, n: rc.fbp(g, n, buf, buf), lambda g, n: rc.fbp_noalloc(g, n, buf, buf),
             lambda g, n: rc.simulate(g, p, n, buf, buf, None, 1e5, buf, buf)]
    for call in calls:
        for kw in bad_geoms:
            with pytest.raises(rc.ReconError, match="invalid argument"):
                call(rc.geometry(**kw), 1)
        with pytest.raises(rc.ReconError, match="invalid argument"):
            call(rc.geometry(**good), 0)


def bad_params(rc):
    """Parameter sets that recon_init_batch and recon_submit must refuse."""
    from synthetic import phantoms as ph
    acq = ph.acquisition("small", n=32)
    base = dict(low=acq.low, high=acq.high)
    return [rc.default_params(**base, lam=-1.0), rc.default_params(**base, lam=0.0),
            rc.default_params(**base, beta0=0.0), rc.default_params(**base, tau=-1.0),
            rc.default_params(**base, iters=-1), rc.default_params(**base, cg_max_iters=-1),
            rc.default_params(**base, cg_tol=-1.0), rc.default_params(**base, precision=2),
            rc.default_params(**base, order=2), rc.default_params(**base, pcg_kernel=4),
            rc.default_params(**base, pcg_kernel=1),
            rc.default_params(**base, e1_kev=50.0, e2_kev=50.0)]


def test_batch_handle_rejects_bad_parameters_and_geometry(rc):
    """recon_init_batch checks every slice's parameters and geometry before
    any device work, so each bad case returns RECON_EINVAL without a GPU."""
    from synthetic import phantoms as ph
    acq = ph.acquisition("small", n=32)
    g = rc.geometry(acq.nx, acq.ny)
    for p in bad_params(rc):
        with pytest.raises(rc.ReconError, match="invalid argument"):
            rc.Solver(g, p)
    p = rc.default_params(low=acq.low, high=acq.high)
    reach = rc.geometry(acq.nx, acq.ny, 50.0, acq.n_views, acq.n_bins, acq.sid_mm, acq.sdd_mm, acq.bin_mm)
    for geom in (rc.geometry(0, 8), rc.geometry(11, 8), rc.geometry(8, 8, 1.0, -1, 8), reach,
                 rc.geometry(acq.nx, acq.ny, acq.pixel_mm, acq.n_views, acq.n_bins, acq.sid_mm, acq.sid_mm,
                             acq.bin_mm)):
        with pytest.raises(rc.ReconError, match="invalid argument"):
            rc.Solver(geom, p)


def test_fbp_limits_checked_before_device_work(rc):
    """Sinogram rows too long for the FBP's shared-memory tables (4000 bins)
    or too many views for its trigonometry table are refused by every entry
    point that reaches the FBP, before any device call: the input-stage
    calls and a batch handle on sinogram inputs."""
    from synthetic import phantoms as ph
    acq = ph.acquisition("small", n=32)
    buf = 1 << 20
    for views, bins in ((40, 4000), (7000, 64)):
        g = rc.geometry(acq.nx, acq.ny, acq.pixel_mm, views, bins, acq.sid_mm, acq.sdd_mm, 0.05)
        for call in (lambda: rc.fbp(g, 1, buf, buf), lambda: rc.fbp_noalloc(g, 1, buf, buf)):
            with pytest.raises(rc.ReconError, match="invalid argument"):
                call()
        with pytest.raises(rc.ReconError, match="invalid argument"):
            rc.Solver(g, rc.default_params(low=acq.low, high=acq.high))


def test_fbp_noalloc_limit_matches_header(rc):
    """The binding's copy of RECON_FBP_NOALLOC_MAX equals the header's."""
    src = open(os.path.join(ROOT, "include", "recon.h")).read()
    m = re.search(r"#define RECON_FBP_NOALLOC_MAX \(([0-9 *]+)\)", src)
    assert m is not None
    val = 1
    for f in m.group(1).split("*"):
        val *= int(f)
    assert rc.FBP_NOALLOC_MAX == val
