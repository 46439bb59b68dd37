"""GB300-native semi-Lagrangian Gauss-Newton-Krylov image registration.

Implements the data-parallel hot path of Mang & Biros (arXiv 1604.02153):
the semi-Lagrangian state, adjoint, incremental state and incremental adjoint
transport solves, the pseudospectral operators, the objective, reduced
gradient and Gauss-Newton Hessian matvec, and the two-level preconditioned
Newton-Krylov solve, as sm_103a CUDA kernels behind the C ABI of
include/reg.h (libregnk.so).

* ``build``  - in-tree nvcc build of libregnk.so
* ``regnk``  - ctypes binding (argument marshalling only)
* ``inputs`` - seeded synthetic images and velocities
"""

__all__ = ["build", "regnk", "inputs"]
