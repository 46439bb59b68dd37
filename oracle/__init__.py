"""FP64 CPU oracle for the semi-Lagrangian Gauss-Newton-Krylov registration solver.

TEST INFRASTRUCTURE ONLY. This package is the plain, slow, obviously correct
reference that the CUDA path is checked against. Only the test suite, the
package smoke check and the benchmark's CPU-baseline leg may import it; the
product library never does, and it shares no code with the CUDA path.

It follows Mang & Biros, "A semi-Lagrangian two-level preconditioned
Newton-Krylov solver for constrained diffeomorphic image registration"
(arXiv 1604.02153):

* ``spectral``  - pseudospectral Fourier operators (§3.2; eq. diffopregv;
                  eq. reg-precond; §3.4.2 restriction/prolongation, filters)
* ``interp``    - periodic cubic B-spline and cubic Lagrange interpolation
                  (§3.2, §3.3.2 "Interpolation", §3.5)
* ``transport`` - RK2 characteristics and the four semi-Lagrangian transport
                  solves (§3.3.2, eq. hyperbolic-pdes-slm, eq. characteristic,
                  eq. transport-along-characteristic)
* ``problem``   - objective, reduced gradient and Gauss-Newton Hessian matvec
                  (eq. varopt:objective, eq. control-elim, eq. hessian-matvec)
                  with the operation counters of Appendix C
* ``krylov``    - PCG, Chebyshev semi-iteration, Lanczos (§3.4.1, §3.4.2)
* ``solver``    - preconditioners P_REG and P_2L, Armijo line search and the
                  inexact Gauss-Newton-Krylov loop (§3.4, §3.5)

Everything is float64 numpy. ``numpy.fft`` is used as a library primitive for
the discrete Fourier transform; no blocking, fusion or reordering is applied
beyond what the paper's steps state.

Parity status of each function is given in its docstring; every function is
pinned by a CPU test unless it says "parity unpinned".
"""

from . import spectral, interp, transport, problem, krylov, solver, d3  # noqa: F401
