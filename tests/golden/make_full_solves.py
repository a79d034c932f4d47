"""Write the oracle's final maps for the full-size parity tests.

Calls only the FP64 oracle (oracle/) and the seeded input generators
(synthetic/); nothing here touches the CUDA path.  Run from the repository
root:  python tests/golden/make_full_solves.py  (about 15 minutes on 8 cores).

Two cases, each stored as tests/golden/<name>.npz with the oracle's Z and
rho_e (float32, enough for the stated tolerances), the body mask, and
checksums of the inputs so that the test can tell when its regenerated
inputs differ from the ones the oracle saw:

* volume_slice_512: slice 80 of the 160 x 512^2 volume phantom (seed 1000),
  image pair mu(60 keV), mu(90 keV) from the oracle's model plus Gaussian
  noise of 4e-4 / mm (seeds 3080, 4080), the full 150-iteration beta schedule
  of the volume workload (Alg. 1, Sec. II-D).
* clinical_512: the 512^2 clinical phantom (seed 1000; bone-like and
  lung-like inserts), Kramers 80 / 140 kVp arms with 2 mm Al and 0.4 mm Sn on
  the high arm, 720 views x 736 bins, Poisson counts at I0 = 1e5 (seed 2000),
  the oracle's FBP of each arm, then 100 iterations (Alg. 1).
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import alg1, ct, model  # noqa: E402
from synthetic import phantoms as ph  # noqa: E402

OUT = os.path.dirname(os.path.abspath(__file__))


def volume_slice_inputs():
    """(mu_L, mu_H) in 1/mm (float32), truth (Z, rho_e), acquisition, iterations."""
    k, n = 80, 512
    V = ph.volume_phantom(1000, n_slices=160, n=n)
    Z, rho = V["Z"][k].astype(np.float64), V["rhoe"][k].astype(np.float64)
    lo = (model.mu_mm(rho, Z, 60.0) + 4e-4 * ph.normal_field((n, n), 3000 + k)).astype(np.float32)
    hi = (model.mu_mm(rho, Z, 90.0) + 4e-4 * ph.normal_field((n, n), 4000 + k)).astype(np.float32)
    return lo, hi, Z, rho, ph.acquisition("volume"), 150


def clinical_inputs():
    """(-log sinograms low, high) as float32, truth (Z, rho_e), acquisition, iterations."""
    acq = ph.acquisition("clinical")
    P = ph.clinical_phantom(1000)
    sL, sH = ct.simulate(P["Z"], P["rhoe"], acq, seed=2000)
    return sL.astype(np.float32), sH.astype(np.float32), P["Z"], P["rhoe"], acq, acq.iters


def checksum(a):
    a = np.asarray(a, np.float64)
    return np.array([a.sum(), np.abs(a).sum(), (a * a).sum()])


def main(which=("volume_slice_512", "clinical_512")):
    if "volume_slice_512" in which:
        t0 = time.time()
        lo, hi, Z, rho, acq, iters = volume_slice_inputs()
        tab = model.Tables(acq.low, acq.high)
        ref = alg1.solve_mm(lo, hi, tab, alg1.Params(iters=iters))
        np.savez_compressed(os.path.join(OUT, "volume_slice_512.npz"), Z=ref["Z"].astype(np.float32),
                            rhoe=ref["rhoe"].astype(np.float32), body=rho >= 0.1, iters=iters,
                            in_low=checksum(lo), in_high=checksum(hi))
        print(f"volume_slice_512: {time.time() - t0:.0f} s", flush=True)
    if "clinical_512" in which:
        t0 = time.time()
        sL, sH, Z, rho, acq, iters = clinical_inputs()
        geom = ct.geometry(acq)
        muL, muH = ct.fbp(sL.astype(np.float64), geom), ct.fbp(sH.astype(np.float64), geom)
        tab = model.Tables(acq.low, acq.high)
        ref = alg1.solve_mm(muL, muH, tab, alg1.Params(iters=iters))
        np.savez_compressed(os.path.join(OUT, "clinical_512.npz"), Z=ref["Z"].astype(np.float32),
                            rhoe=ref["rhoe"].astype(np.float32), body=rho >= 0.1, iters=iters,
                            in_low=checksum(sL), in_high=checksum(sH))
        print(f"clinical_512: {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main(tuple(sys.argv[1:]) or ("volume_slice_512", "clinical_512"))
