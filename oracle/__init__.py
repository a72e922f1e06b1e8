"""CPU FP64 oracle for the FSA convolution (arXiv 2504.19410) -- TEST INFRASTRUCTURE.

This package is a plain, slow, literal numpy statement of what the method
computes.  It exists only to check the CUDA library: only the test suite,
``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import it.  The product path (``paper_2504_19410_gb300``)
never imports it, and it never imports the product path; the two share no
code, tables or constants.  Inputs come from the neutral ``workloads``
module.

Modules
  fsa           -- the method: U^eps, W-hat, T^(1), T^(2), T, the spectrum,
                   the FFT route and the brute-force route of the discrete
                   convolution, the error norm, the App. B bound.
  closed_forms  -- exact potentials of the synthetic densities (not the method).
  dft           -- the oracle's own mixed-radix (2, 3) DFT, so that the FFT
                   route can also run with no FFT library (fsa.solve(fft="own")).

Pins (each function is checked against something other than itself in
``tests/test_oracle_*.py``): Table 2's printed 3-D double errors, Table 1's
W-hat against direct quadrature of Eq. (Fourier-Symmetric), App. B's printed
c thresholds, brute force vs the FFT route, closed-form potentials checked
against a finite-difference Laplacian, the own DFT against the DFT's
definition summed term by term, and exact invariants.  No oracle function is
"parity unpinned".
"""
from . import fsa, closed_forms, dft  # noqa: F401
