"""Final-map parity at the full size and schedule of the benchmarked
workloads, against the FP64 oracle's stored results (tests/golden/*.npz,
written by tests/golden/make_full_solves.py, which calls only the oracle).

* volume_slice_512: one 512^2 slice of the volume workload, image-domain
  inputs, the whole 150-iteration beta schedule (beta from 2e-2 to 1e5), in
  the FP32 path the bench times and in the plain FP64 path.
* clinical_512: the 512^2 clinical slice with bone- and lung-like inserts,
  Kramers 80 / 140 kVp arms (2 mm Al; 0.4 mm Sn on the high arm), 720 x 736
  Poisson sinograms at I0 = 1e5, FBP on the GPU, 100 iterations.

Bar over the body (truth rho_e >= 0.1): mean |dZ| <= 0.01 and mean
|d rho_e| <= 1e-3.  Reported beside it (reading R12): the 99.9th percentile
and median of |dZ|, the count of pixels with |dZ| > 0.1, and the number of
final-state L0 keep decisions of rho_e (eq. sol_hv at lambda / beta_max)
that differ between the two maps.  The inputs are regenerated from their
seeds and checked against the checksums stored with the oracle's maps."""
import importlib.util
import os

import numpy as np
import pytest

from oracle import alg1, model

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden_module():
    spec = importlib.util.spec_from_file_location("make_full_solves", os.path.join(HERE, "golden",
                                                                                   "make_full_solves.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


@pytest.fixture(scope="module")
def rc():
    from paper_2308_01290_gb300 import build_lib
    build_lib.build()
    from paper_2308_01290_gb300 import recon
    return recon


def _check_inputs(ref, lo, hi, gm):
    for key, a in (("in_low", lo), ("in_high", hi)):
        assert np.allclose(gm.checksum(a), ref[key], rtol=1e-9, atol=0), key


def _report(tag, Z, R, ref, lam=1e-2, beta_max=1e5):
    body = ref["body"]
    dZ = np.abs(Z.astype(np.float64) - ref["Z"])[body]
    dR = np.abs(R.astype(np.float64) - ref["rhoe"])[body]
    _, _, k_gpu = alg1.hard_threshold(R.astype(np.float64), lam / beta_max)
    _, _, k_ref = alg1.hard_threshold(ref["rhoe"].astype(np.float64), lam / beta_max)
    out = dict(mean_dZ=float(dZ.mean()), p999_dZ=float(np.percentile(dZ, 99.9)), median_dZ=float(np.median(dZ)),
               n_dZ_gt_01=int((dZ > 0.1).sum()), mean_drho=float(dR.mean()), p999_drho=float(np.percentile(dR, 99.9)),
               flipped_rho_decisions=int((k_gpu != k_ref).sum()))
    print(tag, out)
    return out


@pytest.mark.parametrize("precision", [1, 0])
def test_volume_slice_full_schedule_matches_oracle(rc, precision):
    gm = _golden_module()
    ref = np.load(os.path.join(HERE, "golden", "volume_slice_512.npz"))
    lo, hi, Z, rho, acq, iters = gm.volume_slice_inputs()
    assert int(ref["iters"]) == iters == 150
    _check_inputs(ref, lo, hi, gm)
    p = rc.default_params(low=acq.low, high=acq.high, iters=iters, precision=precision)
    s = rc.Solver(rc.geometry(lo.shape[1], lo.shape[0]), p)
    s.set_data(lo, hi)
    st = s.step(iters, stats=True)
    Zg, Rg, _, _ = [x[0] for x in s.get_host()]
    s.close()
    assert st[0].k == iters
    r = _report(f"volume slice, precision {precision}", Zg, Rg, ref)
    assert r["mean_dZ"] <= 0.01 and r["mean_drho"] <= 1e-3, r


def test_clinical_kramers_slice_matches_oracle(rc):
    gm = _golden_module()
    ref = np.load(os.path.join(HERE, "golden", "clinical_512.npz"))
    sL, sH, Z, rho, acq, iters = gm.clinical_inputs()
    assert int(ref["iters"]) == iters == 100
    _check_inputs(ref, sL, sH, gm)
    p = rc.default_params(low=acq.low, high=acq.high, iters=iters)
    s = rc.Solver(rc.geometry_from_acq(acq), p)
    s.set_data(sL, sH)
    st = s.step(iters, stats=True)
    Zg, Rg, _, _ = [x[0] for x in s.get_host()]
    s.close()
    assert st[0].k == iters
    r = _report("clinical Kramers slice", Zg, Rg, ref)
    assert r["mean_dZ"] <= 0.01 and r["mean_drho"] <= 1e-3, r
