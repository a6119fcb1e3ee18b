"""FP64 CPU oracle for the modal bispectrum estimator (test infrastructure).

This package is a plain, slow, direct restatement of what the estimator of
Fergusson & Shellard, "Optimal Polyspectra Estimation" (arXiv:1105.2791)
computes.  It exists to check the CUDA library; it is not part of the
product.  Only the test suite, the smoke check and the CPU-baseline leg of
the benchmark may import it.  It shares no code with the CUDA path: its own
Gauss-Legendre nodes, its own Legendre recurrence, direct Legendre sums, a
direct Fourier sum over m (no FFT), a direct sum over pixels for the cubic
term, and library linear algebra for the covariance solve.

Modules:
  sht     -- grid, normalised associated Legendre functions, synthesis/analysis
  modal   -- mode/pair orderings, cubic term, linear term, covariance, solve,
             closed forms (alpha for the local shape, covariance of beta),
             adjoint, bivector identities
  wigner  -- Wigner 3j by the Racah formula and a brute-force Gaunt sum

Parity status per function is listed in each module header.
"""
from . import sht, modal, wigner  # noqa: F401
