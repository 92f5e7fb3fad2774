"""Independent FP64 CPU oracle for the RT-EOM-CCSD core-hole propagation.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
the benchmark's CPU-baseline leg may import anything in this package.  It
shares no code with the CUDA library: the library never imports it and it
never imports the library.

Modules
  hamiltonian  (N-1)-electron Fock matrix and spin-orbital integrals (Section 2.1)
  fockspace    determinant-space brute force: e^{-T} H_N e^{T} projections and
               exact e^{i H_N tau} propagation (Eqs. 1-2, 5)
  spinorb      oracle A: spin-orbital CCSD residual from assembled <pq||rs>
               (Eqs. 7-8 written out as the standard non-canonical CCSD equations)
  spinexp      oracle B: spin-explicit (aa/ab/bb) Cholesky-factored residual
               (Section 3.1.1 "spin-explicit" + Cholesky vectors, Eqs. 7-8)
  propagate    first-order Adams-Moulton fixed-point propagation (Eq. 9),
               cumulant (Eqs. 5-6), Green's function (Eq. 4) and the damped
               Fourier transform to A(omega)

Parity status of every function is stated in its module header.
"""
