"""GPU parity, operator by operator, of one iteration of Algorithm 1 against
the FP64 oracle, through the C ABI (recon_debug_op / recon_debug_io).

Each operator is fed the GPU's own float32 state (read back), so the
comparison isolates that operator.  Tolerances: FP32 storage and arithmetic
give ~1e-7 relative rounding per operation; the stencil right-hand sides sum
a handful of O(1) terms and the FFT solves accumulate ~log2(N) rounding
steps, so 1e-5 of the field's magnitude bounds every FP32 operator.  The FP64
path is held to 1e-11.  Threshold decisions are compared exactly: the oracle
takes them in the kernel's precision (float32 differences, squares and sum,
no fused multiply-add)."""
import numpy as np
import pytest

from oracle import alg1, model
from synthetic import phantoms as ph

pytestmark = pytest.mark.gpu

SIZES = [(64, 48), (100, 70), (63, 45), (128, 128), (1, 12), (7, 1)]


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
    rho = P["rhoe"][:ny, :nx]
    rho = np.where(rho > 0, rho, 1.0)  # small crops: keep material everywhere
    Z = np.where(P["rhoe"][:ny, :nx] > 0, Z, 7.45)
    muL = model.mu_mm(rho, Z, 60.0) * (1 + 0.01 * ph.normal_field((ny, nx), seed + 1))
    muH = model.mu_mm(rho, Z, 90.0) * (1 + 0.01 * ph.normal_field((ny, nx), seed + 2))
    return muL.astype(np.float32), muH.astype(np.float32)


def close(gpu, ref, tol):
    scale = max(np.abs(ref).max(), 1e-30)
    err = np.abs(gpu - ref).max() / scale
    assert err <= tol, f"max error {err:.3e} of scale {scale:.3e} > {tol}"
    return err


def make(rc, nx, ny, precision=1, order=0, **kw):
    acq = ph.acquisition("small")
    p = rc.default_params(low=acq.low, high=acq.high, precision=precision, order=order, **kw)
    s = rc.Solver(rc.geometry(nx, ny), p)
    return s, model.Tables(acq.low, acq.high)


@pytest.mark.parametrize("nx,ny", SIZES)
@pytest.mark.parametrize("precision", [1, 0])
def test_operators_one_iteration(rc, nx, ny, precision):
    s, tab = make(rc, nx, ny, precision)
    muL, muH = noisy_images(nx, ny, 3)
    s.set_data(muL, muH)
    tol = 1e-5 if precision == 1 else 1e-11
    fdt = np.float32 if precision == 1 else np.float64
    uL = s.read("MUL")
    uH = s.read("MUH")
    close(uL, muL.astype(np.float64) / model.S_MM, 1e-6 if precision == 1 else 1e-14)
    # --- initialisation (FP64 arithmetic per pixel, stored in the map precision)
    ref0 = alg1.init_state(uL, uH, tab)
    for g, name in (("f1", "F1"), ("f2", "F2"), ("rhoe", "RHO"), ("zt", "Z")):
        close(s.read(name), ref0[g], 1e-6 if precision == 1 else 1e-12)
    st = {g: s.read(n) for g, n in (("f1", "F1"), ("f2", "F2"), ("rhoe", "RHO"), ("zt", "Z"))}
    sc = s.scalars()
    beta, beta_t = sc["beta"], sc["beta_t"]
    lam = 1e-2
    # --- threshold + right-hand sides
    s.op("THRESH_RHS")
    hv = alg1.thresholds(st, lam / beta, fdt)
    close(s.read("RHS_F1"), alg1.rhs_f(0, st, hv["f1"], beta, uL, uH, tab), tol)
    close(s.read("RHS_F2"), alg1.rhs_f(1, st, hv["f2"], beta, uL, uH, tab), tol)
    for g, name in (("rhoe", "DIV_RHO"), ("zt", "DIV_Z")):
        ref = beta_t * alg1.adjoint_diff(*hv[g])
        got = s.read(name)
        if np.abs(ref).max() > 0:
            close(got, ref, tol)
        else:
            assert np.abs(got).max() == 0
    # --- f1, f2 FFT solves from the GPU's right-hand sides
    r1, r2 = s.read("RHS_F1"), s.read("RHS_F2")
    s.op("SOLVE_F")
    close(s.read("F1"), alg1.fft_solve(r1, tab.c_f[0], beta), tol)
    close(s.read("F2"), alg1.fft_solve(r2, tab.c_f[1], beta), tol)
    # --- synthesis, rho_e rhs, Z^m normal equations
    f1, f2 = s.read("F1"), s.read("F2")
    dr, dz = s.read("DIV_RHO"), s.read("DIV_Z")
    s.op("SYNTH")
    m1, m2 = alg1.synthesize(f1, f2, tab)
    close(s.read("RHS_RHO"), model.rhoe_closed_form(m1, m2, tab) + dr, tol)
    a, b = model.z_coefficients(m1, m2, tab)
    close(s.read("A2"), a * a, tol)
    close(s.read("RHS_Z"), a * b + dz, tol)
    assert abs(s.scalars()["abar2"] / np.mean(s.read("A2")) - 1) < 1e-6
    # --- rho_e FFT solve
    rr = s.read("RHS_RHO")
    s.op("SOLVE_RHO")
    close(s.read("RHO"), alg1.fft_solve(rr, 1.0, beta_t), tol)
    # --- Z^m PCG: the solution satisfies the normal equations
    a2, rz = s.read("A2"), s.read("RHS_Z")
    s.op("SOLVE_Z")
    z = s.read("Z")
    res = a2 * z + beta_t * alg1.laplacian(z) - rz
    rel = np.linalg.norm(res) / np.linalg.norm(rz)
    assert rel < (3e-5 if precision == 1 else 1e-6), rel
    zx = alg1.z_solve(a2, rz, beta_t)
    ztol = 1e-3 if precision == 1 else 1e-5
    assert np.abs(z - zx).max() <= ztol * np.abs(zx).max()
    # --- beta schedule
    s.op("NEXT_BETA")
    sc2 = s.scalars()
    kappa = (1e5 / 2e-2) ** (1 / 50)
    assert sc2["k"] == 1 and abs(sc2["beta"] / (beta * kappa) - 1) < 1e-12


def test_gauss_seidel_operator(rc):
    s, tab = make(rc, 64, 48, 1, order=1)
    muL, muH = noisy_images(64, 48, 5)
    s.set_data(muL, muH)
    uL, uH = s.read("MUL"), s.read("MUH")
    st = {g: s.read(n) for g, n in (("f1", "F1"), ("f2", "F2"), ("rhoe", "RHO"), ("zt", "Z"))}
    beta = s.scalars()["beta"]
    s.op("THRESH_RHS")
    s.op("SOLVE_F")
    hv = alg1.thresholds(st, 1e-2 / beta, np.float32)
    f1n = s.read("F1")
    ref2 = alg1.fft_solve(alg1.rhs_f(1, dict(st, f1=f1n), hv["f2"], beta, uL, uH, tab), tab.c_f[1], beta)
    close(s.read("F2"), ref2, 1e-5)


@pytest.mark.parametrize("shape", [(512, 512), (320, 384), (448, 256), (2048, 6), (5, 2048), (3, 3)])
def test_fft_solve_sizes(rc, shape):
    nx, ny = shape
    s, tab = make(rc, nx, ny, 1)
    img = np.full((ny, nx), model.mu_mm(1.0, 7.45, 60.0), np.float32)
    s.set_data(img, (img * 0.8).astype(np.float32))
    rhs = ph.random_field((ny, nx), 7)
    s.write("RHS_RHO", rhs)
    rhs32 = s.read("RHS_RHO")
    s.op("SOLVE_RHO")
    bt = s.scalars()["beta_t"]
    close(s.read("RHO"), alg1.fft_solve(rhs32, 1.0, bt), 1e-5)


def test_fft_solve_large_beta(rc):
    """At beta~ = 1e5 the solve is dominated by the Laplacian symbol."""
    s, tab = make(rc, 96, 80, 1, beta0=1e5)
    img = np.full((80, 96), model.mu_mm(1.0, 7.45, 60.0), np.float32)
    s.set_data(img, img)
    rhs = ph.random_field((80, 96), 8)
    s.write("RHS_RHO", rhs)
    rhs32 = s.read("RHS_RHO")
    s.op("SOLVE_RHO")
    close(s.read("RHO"), alg1.fft_solve(rhs32, 1.0, 1e5), 1e-5)
