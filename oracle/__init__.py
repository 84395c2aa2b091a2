"""FP64 CPU oracle of the spectral point-mass filter (test infrastructure).

This package is the plain, slow reference that the CUDA path is checked
against.  It is test infrastructure only: the tests, the smoke check of the
package entry module and the CPU-baseline leg of the benchmark may import it;
the library and its Python binding never do, and nothing here imports them.

It follows the paper step by step with explicit O(N^2) complex DFT matrices
(no FFT library, no Hartley transform), numpy/scipy primitives (matrix
products, ``scipy.linalg.expm``, Cholesky) and float64 throughout.

Modules
  spectral  DFT of the point-mass density (eq. fourtrsf), the trigonometric
            interpolant (eq. interFreq), first/second spectral derivatives
            (eq. secDer, Sec. V-A coefficient c'').
  model     matrix exponential, Van Loan discretisation of the SDE (eq. dynam),
            measurement functions (eq. meas).
  filter    the filter: grid/frame, Bayes measurement update (eq. filt),
            regridding, spectral Euler time update (Sec. V-B algorithm),
            normalisation and moments.
  fdm       the finite-difference comparator (eqs. FDM, fdiff, FKEnumSol) and
            its sine-transform form (eq. FST).
  kalman    the continuous-discrete Kalman filter (closed form for linear h).

Parity status: every function is pinned by tests in tests/test_oracle_*.py;
the range and bearing measurement updates and the predictions that follow
them are pinned against quadratures and exact moment propagation
(tests/test_oracle_nonlinear.py), the 4-D terrain measurement likewise.
"""
