"""FP64 CPU oracle for the messenger-field Wiener filter and Wiener-posterior sampler.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this package: only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.
It shares no code with the CUDA library (no kernels, headers, tables or helpers); the two meet only
through the seeded input generator ``paper_1810_02821_gb300.synth``, which holds none of the method.

It is deliberately plain and slow:

* ``dft``      — unitary 2D DFT as products with explicit DFT matrices (Eq. 6, normalised, §2.1);
* ``philox``   — Philox4x32-10 from its published definition (Salmon et al., SC'11) + Box–Muller;
* ``messenger``— Algorithm 1 (sampler) and its G -> 0 variant with lambda-cooling (§2.2), A = I or a
  diagonal pixel response A (the general t-update of the Alg. 1 definitions);
* ``dense``    — the Wiener filter of Eq. 2-3 and the posterior covariance of Eq. 4 by dense solves (with
  an optional diagonal response A);
* ``likelihood``— the Gaussian evidence of the data for a power-law P(k) and scaled noise, and its exact
  gradient with respect to (amplitude, slope, noise scale), by dense algebra;
* ``hierarchical``— Alg. 1 sweeps alternated with inverse-gamma draws of binned band powers (the power
  spectrum inference of §5);
* ``spin2``    — shear data of a convergence field (the Kaiser-Squires operator of §5's mass mapping) in
  the messenger sampler, its Wiener filter and posterior by dense algebra, and the FP64 residual of a
  shear map in the Wiener-filter system (the shear covariance applied by FFTs).

Every function is pinned by ``tests/test_oracle_*.py`` against something other than itself
(explicit DFT sums, numpy.fft, dense linear algebra, closed forms, curand's Philox, Monte-Carlo
moments). No function is "parity unpinned".
"""
from . import dft, philox, messenger, dense, likelihood, hierarchical, spin2  # noqa: F401
