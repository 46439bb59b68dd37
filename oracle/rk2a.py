"""Stabilised RK2 (RK2A) state and adjoint solves (FP64 oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The Eulerian comparator of §3.3.1 and Appendix "RK2A derivation": the state
equation in antisymmetric form,
    d_t m + 1/2 (grad m . v + div(m v) - m div v) = 0,
and its adjoint (the first variation of that form),
    -d_t lambda - 1/2 (div(lambda v) + grad lambda . v + lambda div v) = 0,
with pseudospectral derivatives (spectral.grad / spectral.div, Nyquist
zeroed), pointwise products and Heun's method (explicit RK2) in time, the
adjoint run backward from lambda(1). Since the spectral derivative is skew
symmetric, the adjoint's right-hand side is the transpose of the state's,
and one Heun step backward is the transpose of one step forward: the
discrete adjoint is exact (the paper's δ_ADJ at machine precision).
"""

import math

import numpy as np

from . import spectral


def state_rhs(m, v, delta):
    """-1/2 (grad m . v + div(m v) - m div v)."""
    g = spectral.grad(m)
    return -0.5 * (g[0] * v[0] + g[1] * v[1] + spectral.div(m * v) - m * delta)


def adjoint_rhs(lam, v, delta):
    """1/2 (div(lam v) + grad lam . v + lam div v): d lambda / d tau in
    reversed time tau = 1 - t."""
    g = spectral.grad(lam)
    return 0.5 * (spectral.div(lam * v) + g[0] * v[0] + g[1] * v[1] + lam * delta)


def heun(u, f, ht):
    k1 = f(u)
    k2 = f(u + ht * k1)
    return u + 0.5 * ht * (k1 + k2)


def state_solve(m0, v, nt):
    """m(1) from m(0) = m0 in nt Heun steps."""
    delta = spectral.div(v)
    m = np.array(m0, dtype=np.float64)
    for _ in range(nt):
        m = heun(m, lambda x: state_rhs(x, v, delta), 1.0 / nt)
    return m


def adjoint_solve(lam1, v, nt):
    """lambda(0) from lambda(1) = lam1 in nt Heun steps backward in time."""
    delta = spectral.div(v)
    lam = np.array(lam1, dtype=np.float64)
    for _ in range(nt):
        lam = heun(lam, lambda x: adjoint_rhs(x, v, delta), 1.0 / nt)
    return lam


def cfl_steps(v, c):
    """Time steps for CFL number c: nt = ceil(max_i max|v_i| / (c h_i))
    (the time step h_t = 1/nt moves no point by more than c cells)."""
    n2, n1 = v.shape[1:]
    h1, h2 = 2.0 * np.pi / n1, 2.0 * np.pi / n2
    speed = max(float(np.max(np.abs(v[0]))) / h1, float(np.max(np.abs(v[1]))) / h2)
    return max(1, int(math.ceil(speed / c)))
