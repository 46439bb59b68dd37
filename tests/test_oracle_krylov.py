"""Pins of the oracle's Krylov methods and preconditioners (CPU only).

* PCG: finite termination on a small SPD matrix; negative-curvature exit;
* Chebyshev: the 2 rho^k error bound on diagonal SPD matrices;
* Lanczos: extremal Ritz values against a dense eigensolver;
* P_REG is the exact inverse of beta A; P_2L is symmetric at v = 0 (where the
  GN Hessian is exactly symmetric);
* KKT recovery (§4.2.2, table "KKT solve solution error"): H x = H x*,
  x* = -0.5 v*, PCG tolerance 1e-12 recovers x* for every preconditioner.
"""

import numpy as np
import pytest

from oracle import krylov, spectral, transport
from oracle.problem import Problem
from oracle.solver import Solver
from paper_1604_02153_gb300 import inputs


def spd(n, cond, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.geomspace(1.0, cond, n)
    return Q @ np.diag(ev) @ Q.T, ev


def test_pcg_finite_termination():
    A, _ = spd(12, 20.0, 0)
    b = np.random.default_rng(1).standard_normal(12)
    x, info = krylov.pcg(lambda p: A @ p, b, lambda r: r, 1e-13, 12)
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) < 1e-10
    assert info["iters"] <= 12
    # an exact preconditioner converges in one step
    Ainv = np.linalg.inv(A)
    x1, info1 = krylov.pcg(lambda p: A @ p, b, lambda r: Ainv @ r, 1e-10, 5)
    assert info1["iters"] == 1


def test_pcg_negative_curvature_exit():
    A = np.diag([1.0, 2.0, -1.0])
    b = np.array([1.0, 1.0, 1.0])
    x, info = krylov.pcg(lambda p: A @ p, b, lambda r: r, 1e-12, 10)
    assert info["negcurv"]
    assert np.all(np.isfinite(x))


@pytest.mark.parametrize("k", [3, 5, 10])
def test_chebyshev_error_bound(k):
    rng = np.random.default_rng(2)
    ev = np.geomspace(1.0, 50.0, 40)
    b = rng.standard_normal(40)
    x, mv = krylov.chebyshev(lambda p: ev * p, b, ev[0], ev[-1], k)
    assert mv == k - 1
    xs = b / ev
    err = np.sqrt(np.sum(ev * (x - xs) ** 2))
    e0 = np.sqrt(np.sum(ev * xs ** 2))
    kappa = ev[-1] / ev[0]
    rho = (np.sqrt(kappa) - 1) / (np.sqrt(kappa) + 1)
    assert err <= 2 * rho ** k * e0 * (1 + 1e-12)
    # and it is the Chebyshev polynomial: equality up to rounding at the
    # equioscillation bound is not required, but the error must be below the
    # Richardson iteration with the optimal fixed step
    xr = np.zeros(40)
    om = 2.0 / (ev[0] + ev[-1])
    for _ in range(k):
        xr = xr + om * (b - ev * xr)
    assert err < np.sqrt(np.sum(ev * (xr - xs) ** 2))


def test_lanczos_extremal_eigenvalues():
    A, ev = spd(60, 1e2, 3)
    v0 = np.random.default_rng(4).standard_normal(60)
    lo, hi, m = krylov.lanczos_extremal(lambda p: A @ p, v0, 30)
    assert abs(hi - ev[-1]) / ev[-1] < 1e-6
    assert hi <= ev[-1] * (1 + 1e-12)


def config1_problem(n, nt=4, beta=1e-2):
    m_T, vstar = inputs.sinusoid_pair(n)
    P0 = Problem(np.zeros((n, n)), m_T, nt, beta)
    m_R = P0.state_solve(vstar)
    return Problem(m_R, m_T, nt, beta), vstar


def test_reg_preconditioner_is_exact_inverse():
    n = 32
    P, _ = config1_problem(n)
    S = Solver(P, precond="REG")
    r = inputs.random_velocity(n, seed=5, vmax=1.0)
    z = S.precond_reg(r)
    back = spectral.apply_reg(z, P.beta, "H1")
    mean = np.mean(r, axis=(1, 2), keepdims=True)
    assert np.max(np.abs(back - (r - mean))) < 1e-10


def test_two_level_preconditioner_symmetric_at_zero_velocity():
    n = 32
    P, _ = config1_problem(n)
    P.state_solve(np.zeros((2, n, n)))
    S = Solver(P, precond="2L", pc_solver="cheb")
    S.estimate_eigenvalues()
    S.set_velocity_coarse(np.zeros((2, n, n)))
    a = inputs.random_velocity(n, seed=6, vmax=1.0)
    b = inputs.random_velocity(n, seed=7, vmax=1.0)
    lhs = np.sum(S.apply_precond(a) * b)
    rhs = np.sum(a * S.apply_precond(b))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)
    assert S.eig["emin"] > 1.0 and S.eig["emax"] > S.eig["emin"]


@pytest.mark.parametrize("precond,pc_solver", [("REG", None), ("2L", "cheb"), ("2L", "pcg")])
def test_kkt_recovery(precond, pc_solver):
    """§4.2.2 first experiment at 32^2: x* = -0.5 v*, b = H x*, PCG 1e-12."""
    n = 32
    P, vstar = config1_problem(n)
    P.state_solve(vstar)
    xs = -0.5 * vstar
    b = P.hessian_matvec(xs)
    S = Solver(P, precond=precond, pc_solver=pc_solver or "cheb")
    S.eta = 1e-12
    x, info = S.kkt_solve(b, 1e-12, maxit=200)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-9, info


def test_trapezoid_weights():
    w = transport.trapezoid_weights(5)
    assert w.sum() == 5.0 and w[0] == 0.5 and w[-1] == 0.5
