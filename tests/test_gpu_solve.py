"""GPU parity of whole solves of Algorithm 1 against the FP64 oracle, through
the C ABI, on the 128^2 workload (disc phantom, mono 60/90 keV, 180 views,
192 bins, Poisson noise at I0 = 1e5, 50 iterations).

Final-map tolerances over the body (truth rho_e >= 0.1), both precisions:
mean |dZ| <= 0.01 and mean |d rho_e| <= 1e-3, with the 99.9th percentile,
the median and the count of pixels with |dZ| > 0.1 reported.  The GPU's Z^m
step is a PCG to a relative residual of 1e-6 while the oracle solves it
exactly, and L0 thresholding (eq. sol_hv) is discontinuous: in FP32 a
gradient within rounding of the threshold can fall on the other side, and at
large beta~ the near-Poisson solves spread that change over the slice.  So
the iterates are compared on these statistics, not element by element; the
operator tests check each step element by element."""
import numpy as np
import pytest

from oracle import alg1, ct, model
from synthetic import phantoms as ph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rc():
    from paper_2308_01290_gb300 import build_lib
    build_lib.build()
    from paper_2308_01290_gb300 import recon
    return recon


@pytest.fixture(scope="module")
def small_case():
    acq = ph.acquisition("small")
    P = ph.small_phantom(0)
    muL, muH, (sL, sH) = ct.images_from_phantom(P["Z"], P["rhoe"], acq, seed=0)
    tab = model.Tables(acq.low, acq.high)
    ref = alg1.solve_mm(muL.astype(np.float32), muH.astype(np.float32), tab, alg1.Params(iters=acq.iters))
    ref_sino = alg1.solve_mm(muL, muH, tab, alg1.Params(iters=acq.iters))
    return dict(acq=acq, P=P, muL=muL, muH=muH, sL=sL, sH=sH, ref=ref, ref_sino=ref_sino, tab=tab)


def report(tag, Z, rho, ref, body):
    dZ = np.abs(Z - ref["Z"])
    dr = np.abs(rho - ref["rhoe"])
    out = dict(mean_dZ=float(dZ[body].mean()), median_dZ=float(np.median(dZ[body])),
               n_dZ_gt_01=int((dZ[body] > 0.1).sum()), mean_drho=float(dr[body].mean()),
               p999_dZ=float(np.percentile(dZ[body], 99.9)), p999_drho=float(np.percentile(dr[body], 99.9)),
               mean_dZ_all=float(dZ.mean()), mean_drho_all=float(dr.mean()))
    print(tag, out)
    return out


def parity_ok(r, precision=1):
    return r["mean_dZ"] <= 0.01 and r["mean_drho"] <= 1e-3


def map_errors(tag, maps, ref, body):
    """Error against the FP64 oracle of each final map over the body: mean,
    99.9th percentile and maximum of |GPU - oracle|, and the oracle map's
    mean magnitude for scale."""
    out = {}
    for name, got in maps.items():
        d = np.abs(np.asarray(got, np.float64) - ref[name])[body]
        out[name] = dict(mean=float(d.mean()), p999=float(np.percentile(d, 99.9)), max=float(d.max()),
                         scale=float(np.abs(ref[name][body]).mean()))
    print(tag, "per-map error", out)
    return out


@pytest.mark.parametrize("precision", [1, 0])
def test_small_solve_matches_oracle(rc, small_case, precision):
    c = small_case
    acq = c["acq"]
    p = rc.default_params(low=acq.low, high=acq.high, precision=precision, iters=acq.iters)
    s = rc.Solver(rc.geometry(acq.nx, acq.ny), p)
    s.set_data(c["muL"].astype(np.float32), c["muH"].astype(np.float32))
    s.step(acq.iters)
    Z, rho, f1, f2 = [x[0] for x in s.get_host()]
    body = c["P"]["rhoe"] >= 0.1
    r = report(f"precision={precision}", Z, rho, c["ref"], body)
    m = map_errors(f"precision={precision}", dict(Z=Z, rhoe=rho, f1=f1, f2=f2), c["ref"], body)
    assert all(np.isfinite(v["max"]) for v in m.values())
    assert parity_ok(r, precision), r
    sc = s.scalars()
    assert sc["k"] == acq.iters


def test_sinogram_input_matches_oracle_pipeline(rc, small_case):
    """GPU FBP + solve from the oracle's noisy sinograms vs oracle FBP + solve."""
    c = small_case
    acq = c["acq"]
    p = rc.default_params(low=acq.low, high=acq.high, iters=acq.iters)
    s = rc.Solver(rc.geometry_from_acq(acq), p)
    s.set_data(c["sL"].astype(np.float32), c["sH"].astype(np.float32))
    uL = s.read("MUL") * model.S_MM
    assert np.abs(uL - c["muL"]).max() <= 1e-4 * np.abs(c["muL"]).max()
    s.step(acq.iters)
    Z, rho, _, _ = [x[0] for x in s.get_host()]
    body = c["P"]["rhoe"] >= 0.1
    r = report("sinogram", Z, rho, c["ref_sino"], body)
    assert parity_ok(r), r


def test_host_sinograms_equal_device_sinograms(rc, small_case):
    """Host sinograms come in one FBP group at a time on the handle's copy
    stream, beside the FBP of the groups before, and host maps go out one
    group at a time beside the extraction of the next.  On 20 slices (groups
    of 8, 8 and 4) the maps through pinned host memory, through pageable host
    memory and through device memory are the same bit for bit, and so are
    those of a second set_data of other data on the same handle (the copies
    must wait for the work queued before them)."""
    torch = pytest.importorskip("torch")
    c = small_case
    acq = c["acq"]
    n = 20
    g = rc.geometry_from_acq(acq)
    p = rc.default_params(low=acq.low, high=acq.high, iters=3)
    sL = np.concatenate([(c["sL"] * (1.0 + 0.01 * s)).astype(np.float32).ravel() for s in range(n)])
    sH = np.concatenate([(c["sH"] * (1.0 + 0.01 * s)).astype(np.float32).ravel() for s in range(n)])
    npx = n * acq.nx * acq.ny

    def run(s, mode, lo, hi):
        if mode == "device":
            s.set_data(torch.from_numpy(lo).cuda(), torch.from_numpy(hi).cuda(), on_device=True)
        elif mode == "pinned":
            # read asynchronously: hl and hh live until this function returns
            hl, hh = torch.from_numpy(lo).pin_memory(), torch.from_numpy(hi).pin_memory()
            s.set_data(hl.data_ptr(), hh.data_ptr(), on_device=False)
        else:
            s.set_data(lo, hi)
        s.step(3)
        if mode == "pinned":
            Zp, Rp = torch.empty(npx).pin_memory(), torch.empty(npx).pin_memory()
            s.get(Z=Zp.data_ptr(), rhoe=Rp.data_ptr(), on_device=False)
            return Zp.numpy().copy(), Rp.numpy().copy()
        Z, R = np.empty(npx, np.float32), np.empty(npx, np.float32)
        s.get(Z, R)
        return Z, R

    outs = {}
    for mode in ("device", "pinned", "pageable"):
        s = rc.Solver([g] * n, [p] * n)
        outs[mode] = run(s, mode, sL, sH)
        # a second load on the same handle, of other data
        outs[mode + "2"] = run(s, mode, sH, sL)
        s.close()
    for mode in ("pinned", "pageable"):
        for k in ("", "2"):
            assert np.array_equal(outs[mode + k][0], outs["device" + k][0]), mode + k
            assert np.array_equal(outs[mode + k][1], outs["device" + k][1]), mode + k
    assert not np.array_equal(outs["device"][0], outs["device2"][0])


def test_get_async_equals_get(rc, small_case):
    """recon_get_async: two volumes (20 slices each: groups of 8, 8, 4) go
    through set_data, step and get_async back to back into two pairs of
    pinned buffers, the second volume's work running while the first one's
    maps are copied out; after sync each pair equals the synchronous
    recon_get of its volume bit for bit, and so do f1 and f2.  A third round
    into the first pair again is ordered after its earlier copies."""
    torch = pytest.importorskip("torch")
    c = small_case
    acq = c["acq"]
    n = 20
    g = rc.geometry_from_acq(acq)
    p = rc.default_params(low=acq.low, high=acq.high, iters=3)
    npx = n * acq.nx * acq.ny
    vols = []
    for v in range(2):
        sL = np.concatenate([(c["sL"] * (1.0 + 0.01 * s + 0.1 * v)).astype(np.float32).ravel() for s in range(n)])
        sH = np.concatenate([(c["sH"] * (1.0 + 0.01 * s + 0.1 * v)).astype(np.float32).ravel() for s in range(n)])
        vols.append((torch.from_numpy(sL).pin_memory(), torch.from_numpy(sH).pin_memory()))
    s = rc.Solver([g] * n, [p] * n)
    ref = []
    for lo, hi in vols:
        s.set_data(lo.data_ptr(), hi.data_ptr(), on_device=False)
        s.step(3)
        outs = [np.empty(npx, np.float32) for _ in range(4)]
        s.get(*outs)
        ref.append(outs)
    bufs = [[torch.empty(npx).pin_memory() for _ in range(4)] for _ in range(2)]
    for v, (lo, hi) in enumerate(vols):
        s.set_data(lo.data_ptr(), hi.data_ptr(), on_device=False)
        s.step(3)
        s.get_async(*[b.data_ptr() for b in bufs[v]])
    s.sync()
    for v in range(2):
        for k in range(4):
            assert np.array_equal(bufs[v][k].numpy(), ref[v][k]), (v, k)
    assert not np.array_equal(ref[0][0], ref[1][0])
    lo, hi = vols[0]
    s.set_data(lo.data_ptr(), hi.data_ptr(), on_device=False)
    s.step(3)
    s.get_async(Z=bufs[1][0].data_ptr(), rhoe=bufs[1][1].data_ptr())
    s.sync()
    assert np.array_equal(bufs[1][0].numpy(), ref[0][0]) and np.array_equal(bufs[1][1].numpy(), ref[0][1])
    s.close()


def test_one_shot_solve_equals_handle(rc, small_case):
    c = small_case
    acq = c["acq"]
    g = rc.geometry(acq.nx, acq.ny)
    Z1, R1 = rc.solve(c["muL"], c["muH"], g, 1e-2, 2e-2, 12)
    p = rc.default_params(low=acq.low, high=acq.high, iters=12)
    s = rc.Solver(g, p)
    s.set_data(c["muL"].astype(np.float32), c["muH"].astype(np.float32))
    s.step(12)
    Z2, R2, _, _ = [x[0] for x in s.get_host()]
    assert np.array_equal(Z1, Z2) and np.array_equal(R1, R2)


def test_zero_iterations_is_direct_method(rc, small_case):
    """iters = 0 returns the initialisation: the two-step image-based method."""
    c = small_case
    acq = c["acq"]
    p = rc.default_params(low=acq.low, high=acq.high, iters=0)
    s = rc.Solver(rc.geometry(acq.nx, acq.ny), p)
    mL, mH = c["muL"].astype(np.float32), c["muH"].astype(np.float32)
    s.set_data(mL, mH)
    s.step(5)
    Z, rho, _, _ = [x[0] for x in s.get_host()]
    st = alg1.init_state(mL.astype(np.float64) / model.S_MM, mH.astype(np.float64) / model.S_MM, c["tab"])
    assert np.abs(rho - st["rhoe"]).max() < 1e-5
    assert np.abs(Z - model.z_from_ztilde(st["zt"])).max() < 1e-4


def test_batch_equals_alone(rc):
    """Uneven batch: each slice's result is bit-identical to its solve alone."""
    acq = ph.acquisition("small")
    sizes = [(64, 64), (100, 70), (128, 128), (45, 63)]
    iters = [10, 20, 15, 7]
    lams = [1e-2, 5e-3, 2e-2, 1e-2]
    imgs = []
    for k, (nx, ny) in enumerate(sizes):
        n = max(nx, ny)
        P = ph.small_phantom(10 + k, n=n)
        Z, rho = P["Z"][:ny, :nx], P["rhoe"][:ny, :nx]
        L = model.mu_mm(rho, Z, 60.0) + 4e-4 * ph.normal_field((ny, nx), 20 + k)
        H = model.mu_mm(rho, Z, 90.0) + 4e-4 * ph.normal_field((ny, nx), 30 + k)
        imgs.append((L.astype(np.float32), H.astype(np.float32)))
    geoms = [rc.geometry(nx, ny) for nx, ny in sizes]
    params = [rc.default_params(low=acq.low, high=acq.high, iters=it, lam=lm, beta0=2 * lm)
              for it, lm in zip(iters, lams)]
    b = rc.Solver(geoms, params)
    b.set_data(np.concatenate([i[0].ravel() for i in imgs]), np.concatenate([i[1].ravel() for i in imgs]))
    b.step(max(iters))
    Zb, Rb, _, _ = b.get_host()
    for k in range(len(sizes)):
        s = rc.Solver(geoms[k], params[k])
        s.set_data(*imgs[k])
        s.step(iters[k])
        Zs, Rs, _, _ = s.get_host()
        assert np.array_equal(Zs[0], Zb[k]) and np.array_equal(Rs[0], Rb[k]), k
        assert b.scalars(k)["k"] == iters[k]


def test_multigrid_batch_equals_alone(rc):
    """Slices of different multigrid depths in one batch (320^2: three tile
    levels and a 5 x 5 coarsest grid; 192 x 256: two tile levels, 8 x 6; 96 x
    160 next to a 100 x 70 slice on the FFT preconditioner): each result is
    bit-identical to the slice solved alone."""
    acq = ph.acquisition("small")
    sizes = [(320, 320), (192, 256), (96, 160), (100, 70)]
    imgs = []
    for k, (nx, ny) in enumerate(sizes):
        P = ph.small_phantom(40 + k, n=max(nx, ny))
        Z, rho = P["Z"][:ny, :nx], P["rhoe"][:ny, :nx]
        L = model.mu_mm(rho, Z, 60.0) + 4e-4 * ph.normal_field((ny, nx), 50 + k)
        H = model.mu_mm(rho, Z, 90.0) + 4e-4 * ph.normal_field((ny, nx), 60 + k)
        imgs.append((L.astype(np.float32), H.astype(np.float32)))
    geoms = [rc.geometry(nx, ny) for nx, ny in sizes]
    p = rc.default_params(low=acq.low, high=acq.high, iters=8)
    b = rc.Solver(geoms, [p] * len(sizes))
    b.set_data(np.concatenate([i[0].ravel() for i in imgs]), np.concatenate([i[1].ravel() for i in imgs]))
    b.step(8)
    Zb, Rb, _, _ = b.get_host()
    for k in range(len(sizes)):
        s = rc.Solver(geoms[k], p)
        s.set_data(*imgs[k])
        s.step(8)
        Zs, Rs, _, _ = s.get_host()
        assert np.array_equal(Zs[0], Zb[k]) and np.array_equal(Rs[0], Rb[k]), sizes[k]
        s.close()


def test_stats_objective_matches_oracle(rc, small_case):
    """recon_stats of an iteration = eq. obj_unconstraint terms of the iterate
    it started from (same thresholded gradients).  The iterate is the oracle's
    state after three iterations, written into the GPU fields."""
    c = small_case
    acq = c["acq"]
    p = rc.default_params(low=acq.low, high=acq.high, iters=acq.iters)
    s = rc.Solver(rc.geometry(acq.nx, acq.ny), p)
    mL, mH = c["muL"].astype(np.float32), c["muH"].astype(np.float32)
    s.set_data(mL, mH)
    uL = mL.astype(np.float64) / model.S_MM
    uH = mH.astype(np.float64) / model.S_MM
    uL32, uH32 = uL.astype(np.float32).astype(np.float64), uH.astype(np.float32).astype(np.float64)
    ref_st = alg1.solve(uL32, uH32, c["tab"], alg1.Params(iters=3, kappa=1.0))
    st = {g: np.asarray(ref_st[g], np.float32).astype(np.float64) for g in ("f1", "f2", "rhoe", "zt")}
    s.write("MUL", uL32)
    s.write("MUH", uH32)
    for g, name in (("f1", "F1"), ("f2", "F2"), ("rhoe", "RHO"), ("zt", "Z")):
        s.write(name, st[g])
    beta = s.scalars()["beta"]
    stats = s.step(1, stats=True)[0]
    hv = alg1.thresholds(st, 1e-2 / beta, np.float32)
    ref = alg1.objective(st, hv, beta, 1e-2, uL32, uH32, c["tab"])
    assert stats.k == 1
    assert abs(stats.beta / beta - 1) < 1e-12
    for a, b in (("fid_low", "fid_L"), ("fid_high", "fid_H"), ("model_e1", "mod_1"), ("model_e2", "mod_2"),
                 ("relax", "relax")):
        assert abs(getattr(stats, a) - ref[b]) <= 1e-5 * abs(ref[b]) + 1e-12, (a, getattr(stats, a), ref[b])
    assert sum(stats.nnz) == ref["nnz"]
    assert stats.cg_rel_residual <= 1e-6 * 1.0001 or stats.cg_iters == 64


def test_invalid_sizes_rejected(rc):
    p = rc.default_params()
    with pytest.raises(rc.ReconError):
        rc.Solver(rc.geometry(11, 8), p)
    with pytest.raises(rc.ReconError):
        rc.Solver(rc.geometry(0, 8), p)
    with pytest.raises(rc.ReconError):
        rc.Solver(rc.geometry(4096, 8), p)
    s = rc.Solver(rc.geometry(8, 8), p)
    with pytest.raises(rc.ReconError):
        s.step(1)      # before set_data


@pytest.mark.parametrize("shape,precision", [((128, 128), 1), ((256, 192), 1), ((320, 320), 1), ((640, 96), 1),
                                            ((512, 512), 1), ((128, 128), 0)])
def test_multigrid_pcg_matches_fft_pcg(rc, shape, precision):
    """The Z^m PCG with the multigrid V-cycle (pcg_kernel 0 on slices that
    halve down to a small grid) and with the FFT preconditioner (pcg_kernel
    2) on the same normal equations, built by the oracle from a noisy
    phantom, with a step cap high enough for both: both reach the PCG
    tolerance and the oracle's exact solution, and the multigrid cycle takes
    fewer steps.  The FP32 widths take every layout of the fine and strip
    levels: one to four warps per row (128, 256, 320 with an idle warp) and
    ghost-column strips (640, whose level 1 is 320 wide); 512^2 runs the
    FFT preconditioner's column pass with its r.y reduction on 512-point
    columns (257 columns: 32 items of 8 and one of 1)."""
    nx, ny = shape
    acq = ph.acquisition("small")
    tab = model.Tables(acq.low, acq.high)
    n = max(nx, ny)
    P = ph.small_phantom(31, n=n)
    y0, x0 = (n - ny) // 2, (n - nx) // 2   # the middle of the phantom
    Z, rho = P["Z"][y0:y0 + ny, x0:x0 + nx], P["rhoe"][y0:y0 + ny, x0:x0 + nx]
    L = (model.mu_mm(rho, Z, 60.0) + 4e-4 * ph.normal_field((ny, nx), 32)).astype(np.float32)
    H = (model.mu_mm(rho, Z, 90.0) + 4e-4 * ph.normal_field((ny, nx), 33)).astype(np.float32)
    st = alg1.init_state(L.astype(np.float64) / model.S_MM, H.astype(np.float64) / model.S_MM, tab)
    bt = 0.3
    hv = alg1.thresholds(st, 1e-2 / bt)
    m1, m2 = alg1.synthesize(st["f1"], st["f2"], tab)
    a2, rz = alg1.z_terms(m1, m2, hv["zt"], bt, tab)
    a2, rz, z0 = [np.asarray(v, np.float32).astype(np.float64) for v in (a2, rz, st["zt"])]
    zx = alg1.z_solve(a2, rz, bt)
    steps = {}
    for path in (2, 0):
        p = rc.default_params(low=acq.low, high=acq.high, iters=50, pcg_kernel=path, beta0=bt, precision=precision,
                              cg_max_iters=400)
        s = rc.Solver(rc.geometry(nx, ny), p)
        s.set_data(L, H)
        s.write("A2", a2)
        s.write("RHS_Z", rz)
        s.write("Z", z0)
        s.op("SOLVE_Z")
        z = s.read("Z")
        res = np.linalg.norm(a2 * z + bt * alg1.laplacian(z) - rz) / np.linalg.norm(rz)
        steps[path] = s.scalars()["cg_iters"]
        print(shape, precision, "pcg_kernel", path, "steps", steps[path], "relative residual", res)
        assert res < (3e-5 if precision == 1 else 2e-6), (path, res)
        assert np.abs(z - zx).max() <= 1e-3 * np.abs(zx).max(), path
        s.close()
    assert steps[0] < steps[2], steps


def test_band_kernels_equal_strip_kernels(rc):
    """The band kernels (a row of up to 512 columns across the warps of one
    block) form every value of the ghost-column strip kernels' cycle with the
    same rounding sequence: a batch of slices 128, 256 x 192, 320 (an idle
    warp per block) and 512 wide, 10 iterations, gives bitwise the same maps
    with pcg_kernel 0 (band kernels) and 3 (strip kernels on every level)."""
    acq = ph.acquisition("small")
    shapes = [(128, 128), (256, 192), (320, 320), (512, 512)]
    lo, hi = [], []
    for k, (nx, ny) in enumerate(shapes):
        n = max(nx, ny)
        P = ph.small_phantom(40 + k, n=n)
        Z, rho = P["Z"][:ny, :nx], P["rhoe"][:ny, :nx]
        lo.append((model.mu_mm(rho, Z, 60.0) + 4e-4 * ph.normal_field((ny, nx), 50 + k)).astype(np.float32).ravel())
        hi.append((model.mu_mm(rho, Z, 90.0) + 4e-4 * ph.normal_field((ny, nx), 60 + k)).astype(np.float32).ravel())
    out = {}
    for path in (0, 3):
        p = rc.default_params(low=acq.low, high=acq.high, iters=10, pcg_kernel=path)
        s = rc.Solver([rc.geometry(nx, ny) for nx, ny in shapes], [p] * len(shapes))
        s.set_data(np.concatenate(lo), np.concatenate(hi))
        s.step(10)
        out[path] = s.get_host()
        s.close()
    for a, b in zip(out[0], out[3]):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


def test_graph_iterations_equal_separate_launches(rc, small_case):
    """Iterations run as one CUDA graph launch each (a conditional WHILE node
    for the Z^m PCG) give bitwise the maps of separate launches."""
    c = small_case
    acq = c["acq"]
    g = rc.geometry(acq.nx, acq.ny)
    p = rc.default_params(low=acq.low, high=acq.high, iters=12)
    lo = np.stack([c["muL"], 1.02 * c["muL"]]).astype(np.float32)
    hi = np.stack([c["muH"], 1.02 * c["muH"]]).astype(np.float32)
    out = []
    for graph in (False, True):
        s = rc.Solver([g, g], [p, p])
        if graph:
            s.set_graph(True)
        s.set_data(lo, hi)
        s.step(12)
        out.append(s.get_host())
        launches = s.launches()
        s.close()
        assert launches > 12 * 20, launches
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


def test_autotune_mixed_preconditioners(rc, small_case):
    """A batch with a multigrid slice (128^2) and an FFT-preconditioned one
    (100 x 70, whose sides do not halve down): autotune mode 2 regroups the
    row items of both the f solves and the FFT-preconditioned PCG, and both
    slices stay within the final-map tolerance of the untuned solve."""
    c = small_case
    acq = c["acq"]
    g0, g1 = rc.geometry(acq.nx, acq.ny), rc.geometry(100, 70)
    p = rc.default_params(low=acq.low, high=acq.high, iters=8)
    lo = np.concatenate([c["muL"].ravel(), c["muL"][:70, :100].ravel()]).astype(np.float32)
    hi = np.concatenate([c["muH"].ravel(), c["muH"][:70, :100].ravel()]).astype(np.float32)
    out = []
    for mode in (0, 2):
        s = rc.Solver([g0, g1], [p, p])
        s.set_autotune(mode)
        s.set_data(lo, hi)
        s.step(8)
        out.append(s.get_host())
        s.close()
    body = c["P"]["rhoe"] >= 0.1
    for k, b in enumerate((body, body[:70, :100])):
        assert np.isfinite(out[1][0][k]).all()
        assert np.abs(out[1][0][k] - out[0][0][k])[b].mean() <= 0.01, k
        assert np.abs(out[1][1][k] - out[0][1][k])[b].mean() <= 1e-3, k


def test_graph_mixed_preconditioners_equal_separate_launches(rc, small_case):
    """Graph mode with a multigrid slice and an FFT-preconditioned one in the
    same batch: bitwise the maps of separate launches."""
    c = small_case
    acq = c["acq"]
    g0, g1 = rc.geometry(acq.nx, acq.ny), rc.geometry(100, 70)
    p = rc.default_params(low=acq.low, high=acq.high, iters=6)
    lo = np.concatenate([c["muL"].ravel(), c["muL"][:70, :100].ravel()]).astype(np.float32)
    hi = np.concatenate([c["muH"].ravel(), c["muH"][:70, :100].ravel()]).astype(np.float32)
    out = []
    for graph in (False, True):
        s = rc.Solver([g0, g1], [p, p])
        if graph:
            s.set_graph(True)
        s.set_data(lo, hi)
        s.step(6)
        out.append(s.get_host())
        s.close()
    for a, b in zip(out[0], out[1]):
        for k in range(2):
            assert np.array_equal(a[k], b[k]), k


def test_autotune_keeps_results(rc, small_case):
    """Autotune mode 1 picks a grid of {16, 32, 64} x SMs and leaves every
    result bitwise as it was; mode 2 also picks a row-item size and stays
    within the final-map tolerance of the untuned solve."""
    c = small_case
    acq = c["acq"]
    g = rc.geometry(acq.nx, acq.ny)
    p = rc.default_params(low=acq.low, high=acq.high, iters=10)
    lo = np.stack([c["muL"], 0.98 * c["muL"]]).astype(np.float32)
    hi = np.stack([c["muH"], 0.98 * c["muH"]]).astype(np.float32)
    out, tunes = [], []
    for mode in (0, 1, 2):
        s = rc.Solver([g, g], [p, p])
        s.set_autotune(mode)
        s.set_data(lo, hi)
        s.step(10)
        out.append(s.get_host())
        tunes.append(s.tuning())
        s.close()
    assert tunes[0] == (32, 0)
    assert tunes[1][0] in (16, 32, 64) and tunes[1][1] == 0
    assert tunes[2][0] in (16, 32, 64) and tunes[2][1] in (2048, 3072, 4096)
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)
    body = c["P"]["rhoe"] >= 0.1
    for k in range(2):
        assert np.abs(out[2][0][k] - out[0][0][k])[body].mean() <= 0.01
        assert np.abs(out[2][1][k] - out[0][1][k])[body].mean() <= 1e-3
