"""CPU FP64 oracle for the one-step Z / rho_e estimation of arXiv 2308.01290.

TEST INFRASTRUCTURE ONLY.  Nothing in the product (the ``paper_2308_01290_gb300``
package, its CUDA library or its bindings) may import, link or call this
package.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` use it.

It is a plain, slow, obviously correct restatement of the paper in NumPy/SciPy
FP64:

* ``model``  -- attenuation model of Sec. II-A/II-B (basis decomposition,
  photoelectric/Compton model, Klein-Nishina cross-section, closed-form
  rho_e and Z^m), spectra, basis tables.
* ``alg1``   -- Algorithm 1 (Sec. II-D): initialisation, hard threshold of the
  auxiliary gradients (eq. sol_hv), FFT-diagonalised updates of f1, f2,
  rho_e, the Z^m quadratic solve, the beta schedule and the relaxed
  objective (eq. obj_unconstraint); Z as the m-th root of Z^m.
* ``l0``     -- plain gradient-L0 smoothing (Sec. II-C), the building block.
* ``ct``     -- fan-beam Joseph projector, its exact transpose, flat-detector
  FBP and the data simulation that turns phantoms into DECT image pairs.
* ``modeb``  -- the sinogram-domain data terms of the f updates.
* ``iqa``    -- monoenergetic images at any energy, the two-step image-based
  comparator of Sec. III and the image-quality metrics PSNR, NMAD, SSIM.
* ``alg1_3d`` -- Algorithm 1 over a volume with the 3-D multi-domain
  regulariser (a third periodic difference across slices).

Parity status of every function is given in its docstring; functions with no
independent pin say "parity unpinned".
"""
