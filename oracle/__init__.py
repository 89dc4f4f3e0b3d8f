"""CPU oracle for the Fourier pseudo-spectral Navier-Stokes method with embedded Runge-Kutta
step control (Ketcheson, Mortensen, Parsani & Schilling, arXiv:1810.10197).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 restatement of what the
method computes, written from the paper for checking the CUDA implementation.  Only the
test-suite, the smoke check and the benchmark's CPU-baseline leg may import it; the product
(the ``paper_1810_10197_gb300`` package and its C-ABI library) never does, and the two share
no code.  The discrete Fourier transform is the oracle's own (``fft``), checked against the
brute-force DFT sum.

Modules
  fft       -- the oracle's own mixed-radix Cooley-Tukey DFT and the real 3D transforms
  spectral  -- grid, wavenumbers, 2/3 dealiasing, curl, Leray projection, the right-hand
               side of Eq. (ufdef) (Section 2.1) and the Boussinesq form (Section 3.2)
  rk        -- Butcher tableaus (Appendix A), one Runge-Kutta attempt, the embedded error
               norm and the step-size controller (Section 2.2.1), fixed and adaptive drivers
  diag      -- kinetic energy, enstrophy and dissipation rate (Section 3.1)
"""
