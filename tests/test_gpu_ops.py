"""GPU parity, operator by operator, of one iteration of Algorithm 1 against
the FP64 oracle, through the C ABI (recon_debug_io / recon_debug_op).

Every operator's inputs are made on the oracle side (test images, the
oracle's initialisation and its own right-hand sides, rounded to float32),
written into the GPU's fields, and both sides compute from those same
values; no GPU output is fed to the oracle.  Sizes span several tiles with
ragged edges, degenerate 1-pixel-wide images, and full 512^2 slices in a
batch of four (the launch configuration of the benchmark).

Tolerances: FP32 storage and arithmetic give ~1e-7 relative rounding per
operation; the stencil right-hand sides sum a handful of O(1) terms and the
FFT solves accumulate ~log2(N) rounding steps, so 1e-5 of the field's
magnitude bounds every FP32 operator.  The FP64 path is held to 1e-11.
Threshold decisions are compared exactly: the oracle takes them in the
kernel's precision (float32 differences, squares and sum, no fused
multiply-add)."""
import numpy as np
import pytest

from oracle import alg1, model
from synthetic import phantoms as ph

pytestmark = pytest.mark.gpu

SIZES = [(64, 48, 1), (100, 70, 1), (63, 45, 1), (128, 128, 1), (1, 12, 1), (7, 1, 1), (512, 512, 4), (384, 320, 2)]
LAM = 1e-2


@pytest.fixture(scope="module")
def rc():
    from paper_2308_01290_gb300 import build_lib
    build_lib.build()
    from paper_2308_01290_gb300 import recon
    return recon


def noisy_images(nx, ny, seed):
    """Disc phantom in mu (1/mm) at 60/90 keV plus 1% Gaussian noise."""
    n = max(nx, ny)
    P = ph.small_phantom(seed, n=max(n, 16)) if n >= 16 else ph.uniform_phantom(n, 9.0, 1.2)
    Z = P["Z"][:ny, :nx]
    rho = np.where(P["rhoe"][:ny, :nx] > 0, P["rhoe"][:ny, :nx], 1.0)  # keep material everywhere
    Z = np.where(P["rhoe"][:ny, :nx] > 0, Z, 7.45)
    muL = model.mu_mm(rho, Z, 60.0) * (1 + 0.01 * ph.normal_field((ny, nx), seed + 1))
    muH = model.mu_mm(rho, Z, 90.0) * (1 + 0.01 * ph.normal_field((ny, nx), seed + 2))
    return muL.astype(np.float32), muH.astype(np.float32)


def close(gpu, ref, tol):
    scale = max(np.abs(ref).max(), 1e-30)
    err = np.abs(gpu - ref).max() / scale
    assert err <= tol, f"max error {err:.3e} of scale {scale:.3e} > {tol}"
    return err


def make(rc, nx, ny, nb=1, precision=1, order=0, **kw):
    acq = ph.acquisition("small")
    p = rc.default_params(low=acq.low, high=acq.high, precision=precision, order=order, **kw)
    s = rc.Solver([rc.geometry(nx, ny)] * nb, [p] * nb)
    return s, model.Tables(acq.low, acq.high)


def as_stored(x, precision):
    return np.asarray(x, np.float32 if precision == 1 else np.float64).astype(np.float64)


@pytest.mark.parametrize("nx,ny,nb", SIZES)
@pytest.mark.parametrize("precision", [1, 0])
def test_operators_one_iteration(rc, nx, ny, nb, precision):
    if nb > 1 and precision == 0:
        pytest.skip("FP64 path checked at the smaller sizes")
    s, tab = make(rc, nx, ny, nb, precision)
    imgs = [noisy_images(nx, ny, 3 + 5 * k) for k in range(nb)]
    s.set_data(np.concatenate([i[0].ravel() for i in imgs]), np.concatenate([i[1].ravel() for i in imgs]))
    tol = 1e-5 if precision == 1 else 1e-11
    fdt = np.float32 if precision == 1 else np.float64
    sc = s.scalars()
    beta, beta_t = sc["beta"], sc["beta_t"]
    for k in range(nb):
        muL, muH = imgs[k]
        uL = muL.astype(np.float64) / model.S_MM
        uH = muH.astype(np.float64) / model.S_MM
        close(s.read("MUL", k), uL, 1e-6 if precision == 1 else 1e-14)
        # --- initialisation from the stored inputs: FP64 arithmetic per pixel,
        # stored in the map precision; Cramer's rule amplifies the float32
        # rounding of mu by up to ~30, hence the FP32 operator bar of 1e-5
        ref0 = alg1.init_state(as_stored(uL, precision), as_stored(uH, precision), tab)
        for g, name in (("f1", "F1"), ("f2", "F2"), ("rhoe", "RHO"), ("zt", "Z")):
            close(s.read(name, k), ref0[g], tol)
    # every later operator starts from oracle values written into the fields
    states, stored_mu = [], []
    for k in range(nb):
        muL, muH = imgs[k]
        uL = as_stored(muL.astype(np.float64) / model.S_MM, precision)
        uH = as_stored(muH.astype(np.float64) / model.S_MM, precision)
        s.write("MUL", uL, k)
        s.write("MUH", uH, k)
        ref0 = alg1.init_state(uL, uH, tab)
        st = {g: as_stored(v, precision) for g, v in ref0.items()}
        for g, name in (("f1", "F1"), ("f2", "F2"), ("rhoe", "RHO"), ("zt", "Z")):
            s.write(name, st[g], k)
        states.append(st)
        stored_mu.append((uL, uH))
    # --- threshold + right-hand sides
    s.op("THRESH_RHS")
    for k in range(nb):
        st, (uL, uH) = states[k], stored_mu[k]
        hv = alg1.thresholds(st, LAM / beta, fdt)
        close(s.read("RHS_F1", k), alg1.rhs_f(0, st, hv["f1"], beta, uL, uH, tab), tol)
        close(s.read("RHS_F2", k), alg1.rhs_f(1, st, hv["f2"], beta, uL, uH, tab), tol)
        for g, name in (("rhoe", "DIV_RHO"), ("zt", "DIV_Z")):
            ref = beta_t * alg1.adjoint_diff(*hv[g])
            got = s.read(name, k)
            if np.abs(ref).max() > 0:
                close(got, ref, tol)
            else:
                assert np.abs(got).max() == 0
    # --- f1, f2 FFT solves of oracle right-hand sides
    rhs = []
    for k in range(nb):
        st, (uL, uH) = states[k], stored_mu[k]
        hv = alg1.thresholds(st, LAM / beta, fdt)
        r1 = as_stored(alg1.rhs_f(0, st, hv["f1"], beta, uL, uH, tab), precision)
        r2 = as_stored(alg1.rhs_f(1, st, hv["f2"], beta, uL, uH, tab), precision)
        s.write("RHS_F1", r1, k)
        s.write("RHS_F2", r2, k)
        rhs.append((r1, r2))
    s.op("SOLVE_F")
    for k in range(nb):
        close(s.read("F1", k), alg1.fft_solve(rhs[k][0], tab.c_f[0], beta), tol)
        close(s.read("F2", k), alg1.fft_solve(rhs[k][1], tab.c_f[1], beta), tol)
    # --- synthesis, rho_e rhs, Z^m normal equations, from oracle f and divergences
    news = []
    for k in range(nb):
        st = states[k]
        f1 = as_stored(alg1.fft_solve(rhs[k][0], tab.c_f[0], beta), precision)
        f2 = as_stored(alg1.fft_solve(rhs[k][1], tab.c_f[1], beta), precision)
        hv = alg1.thresholds(st, LAM / beta, fdt)
        dr = as_stored(beta_t * alg1.adjoint_diff(*hv["rhoe"]), precision)
        dz = as_stored(beta_t * alg1.adjoint_diff(*hv["zt"]), precision)
        for name, v in (("F1", f1), ("F2", f2), ("DIV_RHO", dr), ("DIV_Z", dz)):
            s.write(name, v, k)
        news.append((f1, f2, dr, dz))
    s.op("SYNTH")
    z_in = []
    for k in range(nb):
        f1, f2, dr, dz = news[k]
        m1, m2 = alg1.synthesize(f1, f2, tab)
        rr = model.rhoe_closed_form(m1, m2, tab) + dr
        a, b = model.z_coefficients(m1, m2, tab)
        close(s.read("RHS_RHO", k), rr, tol)
        close(s.read("A2", k), a * a, tol)
        close(s.read("RHS_Z", k), a * b + dz, tol)
        z_in.append((as_stored(rr, precision), as_stored(a * a, precision), as_stored(a * b + dz, precision)))
    # --- rho_e FFT solve of the oracle right-hand side
    for k in range(nb):
        s.write("RHS_RHO", z_in[k][0], k)
    s.op("SOLVE_RHO")
    for k in range(nb):
        close(s.read("RHO", k), alg1.fft_solve(z_in[k][0], 1.0, beta_t), tol)
    # --- Z^m PCG from oracle a^2, right-hand side and warm start
    for k in range(nb):
        s.write("A2", z_in[k][1], k)
        s.write("RHS_Z", z_in[k][2], k)
        s.write("Z", states[k]["zt"], k)
    s.op("SOLVE_Z")
    for k in range(nb):
        a2, rz = z_in[k][1], z_in[k][2]
        # the preconditioner's diagonal is the mean of the a^2 this solve read
        assert abs(s.scalars(k)["abar2"] / np.mean(a2) - 1) < 1e-5
        z = s.read("Z", k)
        res = a2 * z + beta_t * alg1.laplacian(z) - rz
        rel = np.linalg.norm(res) / np.linalg.norm(rz)
        assert rel < (3e-5 if precision == 1 else 1e-6), rel
        if nx * ny <= 128 * 128 or k == 0:   # exact sparse solve (slow at 512^2: once)
            zx = alg1.z_solve(a2, rz, beta_t)
            ztol = 1e-3 if precision == 1 else 1e-5
            assert np.abs(z - zx).max() <= ztol * np.abs(zx).max()
    # --- beta schedule
    s.op("NEXT_BETA")
    sc2 = s.scalars()
    kappa = (1e5 / 2e-2) ** (1 / 50)
    assert sc2["k"] == 1 and abs(sc2["beta"] / (beta * kappa) - 1) < 1e-12


def test_gauss_seidel_operator(rc):
    s, tab = make(rc, 64, 48, 1, 1, order=1)
    muL, muH = noisy_images(64, 48, 5)
    s.set_data(muL, muH)
    uL = as_stored(muL.astype(np.float64) / model.S_MM, 1)
    uH = as_stored(muH.astype(np.float64) / model.S_MM, 1)
    s.write("MUL", uL)
    s.write("MUH", uH)
    st = {g: as_stored(v, 1) for g, v in alg1.init_state(uL, uH, tab).items()}
    for g, name in (("f1", "F1"), ("f2", "F2"), ("rhoe", "RHO"), ("zt", "Z")):
        s.write(name, st[g])
    beta = s.scalars()["beta"]
    s.op("THRESH_RHS")
    s.op("SOLVE_F")
    hv = alg1.thresholds(st, LAM / beta, np.float32)
    f1n = alg1.fft_solve(alg1.rhs_f(0, st, hv["f1"], beta, uL, uH, tab), tab.c_f[0], beta)
    close(s.read("F1"), f1n, 1e-5)
    ref2 = alg1.fft_solve(alg1.rhs_f(1, dict(st, f1=f1n), hv["f2"], beta, uL, uH, tab), tab.c_f[1], beta)
    close(s.read("F2"), ref2, 1e-5)


@pytest.mark.parametrize("shape", [(512, 512), (320, 384), (448, 256), (2048, 6), (5, 2048), (3, 3),
                                   (64, 1024), (1024, 128), (256, 64), (128, 512), (64, 63), (256, 45),
                                   (384, 448), (448, 320)])
def test_fft_solve_sizes(rc, shape):
    nx, ny = shape
    s, tab = make(rc, nx, ny)
    img = np.full((ny, nx), model.mu_mm(1.0, 7.45, 60.0), np.float32)
    s.set_data(img, (img * 0.8).astype(np.float32))
    rhs32 = as_stored(ph.random_field((ny, nx), 7), 1)
    s.write("RHS_RHO", rhs32)
    s.op("SOLVE_RHO")
    bt = s.scalars()["beta_t"]
    close(s.read("RHO"), alg1.fft_solve(rhs32, 1.0, bt), 1e-5)


def test_fft_solve_large_beta(rc):
    """At beta~ = 1e5 the solve is dominated by the Laplacian symbol."""
    s, tab = make(rc, 96, 80, beta0=1e5)
    img = np.full((80, 96), model.mu_mm(1.0, 7.45, 60.0), np.float32)
    s.set_data(img, img)
    rhs32 = as_stored(ph.random_field((80, 96), 8), 1)
    s.write("RHS_RHO", rhs32)
    s.op("SOLVE_RHO")
    close(s.read("RHO"), alg1.fft_solve(rhs32, 1.0, 1e5), 1e-5)


@pytest.mark.parametrize("precision", [1, 0])
def test_z_extraction_matches_closed_form(rc, precision):
    """A6: Z = Z_w z^(1/m) from the stored z (Z = 1 where z <= 0), over z from
    the FP32 subnormal range to 1e30 (the Newton start and its closed-form
    safeguard), within one FP32 ulp of the FP64 closed form."""
    nx, ny = 70, 9
    s, _ = make(rc, nx, ny, precision=precision)
    img = np.full((ny, nx), model.mu_mm(1.0, 7.45, 60.0), np.float32)
    s.set_data(img, (img * 0.8).astype(np.float32))
    rng = np.random.default_rng(11)
    z = 10.0 ** rng.uniform(-6, 3, size=(ny, nx))
    z.flat[:12] = [0.0, -1.0, -1e-30, 1e-40, 1e-38, 1.2e-38, 1e-20, 1.0, 1e10, 1e30, 3.4e38, 2.0 ** -126]
    zs = as_stored(z, precision)
    s.write("Z", zs)
    Z = s.get_host()[0][0].astype(np.float64)
    ref = model.z_from_ztilde(zs)
    ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    bad = np.abs(Z - ref) > ulp
    assert not bad.any(), (zs[bad][:5], Z[bad][:5], ref[bad][:5])
    assert np.all(Z[zs <= 0] == 1.0)


@pytest.mark.parametrize("nx,ny,nb", [(63, 45, 1), (128, 128, 1), (512, 512, 4), (384, 320, 2), (96, 64, 1)])
@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("beta0", [0.37, 1e3])
def test_z_operator_matches_oracle(rc, nx, ny, nb, precision, beta0):
    """The Z^m normal-equation operator q = [diag(a^2) + beta~ L] p (Alg. 1,
    Z^m line, reading R5), element by element against the oracle's sparse
    z_system, as the PCG forms it: on multigrid slices (128^2, 512^2,
    384 x 320, 96 x 64) in the direction pass (k_mgs_pq in FP32, k_mg_pq in
    FP64), on the 63 x 45 slice (FFT preconditioner) in k_pcg_inv.  The FP32
    multigrid update pass (k_mgs_fwd) forms q once more for r - alpha q; the
    operator leaves -q of that pass in CG_R, which must equal the first q bit
    for bit.  FP32 to 1e-5 of the magnitude of q, FP64 to 1e-12."""
    if nb > 1 and precision == 0:
        pytest.skip("FP64 path checked at the smaller sizes")
    s, tab = make(rc, nx, ny, nb, precision, beta0=beta0)
    imgs = [noisy_images(nx, ny, 3 + 5 * k) for k in range(nb)]
    s.set_data(np.concatenate([i[0].ravel() for i in imgs]), np.concatenate([i[1].ravel() for i in imgs]))
    bt = s.scalars()["beta_t"]
    assert abs(bt / beta0 - 1) < 1e-12
    ins = []
    for k in range(nb):
        a2 = as_stored(ph.random_field((ny, nx), 20 + k, 0.05, 3.0), precision)
        p = as_stored(ph.random_field((ny, nx), 40 + k, -1.0, 1.0), precision)
        s.write("A2", a2, k)
        s.write("CG_P0", p, k)
        ins.append((a2, p))
    s.op("Z_MATVEC")
    tol = 1e-5 if precision == 1 else 1e-12
    for k in range(nb):
        a2, p = ins[k]
        ref = (alg1.z_system(a2, bt) @ p.ravel()).reshape(ny, nx)
        q = s.read("CG_Q", k)
        close(q, ref, tol)
        assert np.array_equal(s.read("CG_P1", k), p)   # p = 0 + 1 * p_old exactly
        if precision == 1 and (nx, ny) != (63, 45):
            assert np.array_equal(s.read("CG_R", k), -q)
