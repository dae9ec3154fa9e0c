"""CPU oracle for the PICO noise-map hot path -- TEST INFRASTRUCTURE ONLY.

This package is a plain, slow, FP64 NumPy restatement of what the paper
"Fast Voxelwise SNR Estimation for Iterative MRI Reconstructions" (PICO)
computes.  It exists to check the CUDA path; it is never a fallback for it.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA library: its
only common dependency is the seeded input generator package ``synth``.

Modules
-------
rng      counter-based SplitMix64 streams, probe and noise draws (Sec. 2.2.4)
ops      encoding operators: pre-whitening (Sec. 2.1.2), Cartesian SENSE and
         exact NUDFT spiral encodings, normal operators (Sec. 2.1.3)
solvers  conjugate gradients (Eq. 6) and the power method (Sec. 3.3)
pico     PICO estimator (Alg. 1), PMR (Sec. 1), exact covariance diagonals
         (Eqs. 8-10), closed-form SENSE g-factor, per-sample variances (Eq. A1)
cs       L1-wavelet FISTA reconstruction, its Jacobian (JVP / VJP) and the
         Jacobian PICO estimator for nonlinear reconstructions (Sec. 2.2.5)

Every function states the passage it follows.  Pins that hold the oracle to
the mathematics (closed forms, brute force, invariants) live in
``tests/test_oracle_pins.py``.
"""
from . import rng, ops, solvers, pico, cs  # noqa: F401
