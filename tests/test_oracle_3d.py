"""Pins of the 3D oracle (oracle/d3.py) against what the method fixes.

* spectral gradient and divergence exact on a trigonometric polynomial; the
  regularisation operator's symbol on a single mode and its powers on a
  mode plus a constant (the k = 0 weight of eq. reg-precond);
* interpolation: integral displacements are exact shifts, zero displacement
  returns the samples (spline and Lagrange);
* reduction to 2D: fields constant along x_3 with v_3 = 0 give the 2D
  oracle's state, gradient, Gauss-Newton matvec and powers of beta A on a
  field with a nonzero mean (the 2D oracle is pinned on its own) and J times
  the x_3 extent 2 pi;
* the reduced gradient against central finite differences of J, the gap
  shrinking with the grid;
* the Gauss-Newton matvec symmetric up to the adjoint error, positive, and
  equal to the derivative of the gradient at zero residual.
"""

import numpy as np
import pytest

from oracle import d3
from oracle.problem import Problem
from paper_1604_02153_gb300 import inputs


def grid3(n1, n2, n3):
    K, J, I = np.meshgrid(*(np.arange(n) * 2 * np.pi / n for n in (n3, n2, n1)), indexing="ij")
    return I, J, K


def test_spectral_operators_on_trig_polynomials():
    n1, n2, n3 = 16, 12, 8
    x1, x2, x3 = grid3(n1, n2, n3)
    u = np.sin(x1) * np.cos(2 * x2) * np.sin(3 * x3) + np.cos(2 * x1 + x3)
    g = d3.grad(u)
    e1 = np.cos(x1) * np.cos(2 * x2) * np.sin(3 * x3) - 2 * np.sin(2 * x1 + x3)
    e2 = -2 * np.sin(x1) * np.sin(2 * x2) * np.sin(3 * x3)
    e3 = 3 * np.sin(x1) * np.cos(2 * x2) * np.cos(3 * x3) - np.sin(2 * x1 + x3)
    for a, b in zip(g, (e1, e2, e3)):
        assert np.max(np.abs(a - b)) < 1e-12
    v = np.stack([np.sin(x2), np.cos(x3) * np.sin(x1), np.sin(2 * x3 + x1)])
    assert np.max(np.abs(d3.div(v) - (np.cos(x3) * 0 + 2 * np.cos(2 * x3 + x1)))) < 1e-12
    w = np.stack([np.cos(2 * x1 - x2 + 3 * x3)] * 3)
    for p, reg in ((1, "H1"), (2, "H2")):
        Aw = d3.apply_reg(w, 0.5, reg)
        assert np.max(np.abs(Aw - 0.5 * 14 ** p * w)) < 1e-9
    # powers of beta A (eq. reg-precond): the zero entry of A's symbol becomes
    # one, so a constant c maps to beta^s c while |k|^2 = 14 maps to (14 beta)^s
    beta, c0 = 0.02, 0.7
    for s in (-1.0, -0.5, 0.5):
        P = d3.reg_power(w + c0, beta, "H1", s)
        assert np.max(np.abs(P - ((14 * beta) ** s * w + beta ** s * c0))) < 1e-9, s


@pytest.mark.parametrize("kind", ["spline", "lagrange"])
def test_interpolation_shifts_and_nodes(kind):
    n1, n2, n3 = 16, 8, 12
    u = inputs.random_field3(n1, n2, n3, seed=3, kmax=4)
    shape = u.shape
    got = d3.at_departure(u, (np.full(shape, 2.0), np.full(shape, -1.0), np.full(shape, 3.0)), kind)
    assert np.max(np.abs(got - np.roll(u, (-3, 1, -2), axis=(0, 1, 2)))) < 1e-12
    z = np.zeros(shape)
    assert np.max(np.abs(d3.at_departure(u, (z, z, z), kind) - u)) < 1e-12


@pytest.mark.parametrize("kind", ["spline", "lagrange"])
def test_reduces_to_the_2d_problem(kind):
    n, n3, nt, beta = 16, 4, 4, 1e-2
    m_T = inputs.random_field(n, seed=1, kmax=4)
    m_R = inputs.random_field(n, seed=2, kmax=4)
    v2 = inputs.random_velocity(n, seed=3, vmax=0.3)
    u2 = inputs.random_velocity(n, seed=4, vmax=1.0)
    tile = lambda a: np.repeat(a[None], n3, axis=0)
    v3 = np.stack([tile(v2[0]), tile(v2[1]), np.zeros((n3, n, n))])
    u3 = np.stack([tile(u2[0]), tile(u2[1]), np.zeros((n3, n, n))])
    P2 = Problem(m_R, m_T, nt, beta, kind=kind)
    P3 = d3.Problem3(tile(m_R), tile(m_T), nt, beta, kind=kind)
    J2, g2 = P2.objective_gradient(v2)
    J3, g3 = P3.objective_gradient(v3)
    assert abs(J3 - 2 * np.pi * J2) < 1e-12 * abs(J3)
    for c in range(2):
        assert np.max(np.abs(g3[c] - tile(g2[c]))) < 1e-12 * np.max(np.abs(g2))
    assert np.max(np.abs(g3[2])) < 1e-12 * np.max(np.abs(g2))
    H2 = P2.hessian_matvec(u2)
    H3 = P3.hessian_matvec(u3)
    for c in range(2):
        assert np.max(np.abs(H3[c] - tile(H2[c]))) < 1e-12 * np.max(np.abs(H2))
    assert np.max(np.abs(H3[2])) < 1e-12 * np.max(np.abs(H2))
    # the powers of beta A on a field with a nonzero mean (the k = 0 weight)
    from oracle import spectral
    w2 = u2 + np.array([0.3, -0.2])[:, None, None]
    w3 = np.stack([tile(w2[0]), tile(w2[1]), np.full((n3, n, n), 0.1)])
    for s in (-1.0, -0.5):
        P2s = spectral.reg_power(w2, beta, "H1", s)
        P3s = d3.reg_power(w3, beta, "H1", s)
        for c in range(2):
            assert np.max(np.abs(P3s[c] - tile(P2s[c]))) < 1e-12 * np.max(np.abs(P2s))


def test_gradient_against_finite_differences():
    gaps = []
    for n in (12, 24):
        m_T = inputs.random_field3(n, n, n, seed=1, kmax=2)
        m_R = inputs.random_field3(n, n, n, seed=2, kmax=2)
        v = inputs.random_velocity3(n, n, n, seed=3, kmax=2, vmax=0.05)
        dv = inputs.random_velocity3(n, n, n, seed=4, kmax=2, vmax=1.0)
        P = d3.Problem3(m_R, m_T, 8, 1e-2)
        _, g = P.objective_gradient(v)
        d = P.inner(g, dv)
        eps = 1e-4
        fd = (P.objective(v + eps * dv) - P.objective(v - eps * dv)) / (2 * eps)
        gaps.append(abs(fd - d) / abs(d))
    assert gaps[-1] < 1e-4 and gaps[1] < gaps[0] / 4, gaps


def test_gauss_newton_matvec_symmetric_positive_and_derivative_at_zero_residual():
    n, nt = 16, 4
    m_T = inputs.random_field3(n, n, n, seed=5, kmax=2)
    v = inputs.random_velocity3(n, n, n, seed=6, kmax=2, vmax=0.2)
    m_R = d3.Problem3(np.zeros((n, n, n)), m_T, nt, 1e-2).state_solve(v)
    P = d3.Problem3(m_R, m_T, nt, 1e-2)
    P.state_solve(v)
    a = inputs.random_velocity3(n, n, n, seed=7, kmax=2, vmax=1.0)
    b = inputs.random_velocity3(n, n, n, seed=8, kmax=2, vmax=1.0)
    Ha, Hb = P.hessian_matvec(a), P.hessian_matvec(b)
    ab, ba = P.inner(Ha, b), P.inner(a, Hb)
    assert abs(ab - ba) < 1e-3 * abs(ab)
    assert P.inner(Ha, a) > 0
    eps = 1e-4
    P.state_solve(v + eps * a)
    gp = P.gradient()
    P.state_solve(v - eps * a)
    gm = P.gradient()
    fd = (gp - gm) / (2 * eps)
    assert np.linalg.norm(fd - Ha) / np.linalg.norm(Ha) < 2e-3


def test_solve_reduces_to_the_2d_solve():
    """The Newton-Krylov solve with P_REG on a problem constant along x_3
    (v_3 = 0 throughout) takes the 2D oracle's iterations: every ratio the
    method forms (step lengths, forcing terms, the Armijo test) is the 2D one,
    the inner products carry the same factor 2 pi."""
    from oracle.solver import Solver
    n, n3, nt, beta, gtol = 16, 4, 4, 1e-2, 1e-2
    m_T, vstar = inputs.sinusoid_pair(n)
    m_R = Problem(np.zeros((n, n)), m_T, nt, beta).state_solve(vstar)
    v2, info2 = Solver(Problem(m_R, m_T, nt, beta), precond="REG").solve(np.zeros((2, n, n)), gtol)
    tile = lambda a: np.repeat(a[None], n3, axis=0)
    P3 = d3.Problem3(tile(m_R), tile(m_T), nt, beta)
    v3, info3 = P3.solve(np.zeros((3, n3, n, n)), gtol)
    assert info3["newton_iters"] == info2["newton_iters"] and info3["matvecs"] == info2["matvecs"]
    assert info3["gnorm_rel"] <= gtol
    # (the 3D and 2D FFTs round differently; PCG carries that into the
    # iterates at the 1e-10 level)
    for c in range(2):
        assert np.max(np.abs(v3[c] - tile(v2[c]))) < 1e-8 * np.max(np.abs(v2))
    assert np.max(np.abs(v3[2])) < 1e-8 * np.max(np.abs(v2))


@pytest.mark.parametrize("kind", ["spline", "lagrange"])
def test_deformation_map_shear_and_constant_velocity(kind):
    """Shear flow v = (a sin x_2, 0, 0): every characteristic keeps x_2, so
    y = x - v, u = (-a sin x_2, 0, 0) exactly and det grad y = 1 (a unit
    triangular J); a constant velocity c gives u = -c."""
    n1, n2, n3, nt, a = 16, 12, 8, 4, 0.3
    x1, x2, x3 = grid3(n1, n2, n3)
    z = np.zeros_like(x1)
    v = np.stack([a * np.sin(x2), z, z])
    u = d3.deformation_map(v, nt, kind)
    assert np.max(np.abs(u[0] + a * np.sin(x2))) < 1e-12
    assert np.max(np.abs(u[1])) < 1e-12 and np.max(np.abs(u[2])) < 1e-12
    assert np.max(np.abs(d3.det_grad_map(u) - 1.0)) < 1e-12
    c = np.array([0.37, -0.21, 0.55])
    u = d3.deformation_map(np.stack([np.full_like(x1, cc) for cc in c]), nt, kind)
    for k in range(3):
        assert np.max(np.abs(u[k] + c[k])) < 1e-12


def test_deformation_map_reduces_to_2d():
    from oracle import spectral
    from oracle import transport as transport2
    n, n3, nt = 16, 4, 4
    v2 = inputs.random_velocity(n, seed=21, vmax=0.5)
    tile = lambda a: np.repeat(a[None], n3, axis=0)
    v3 = np.stack([tile(v2[0]), tile(v2[1]), np.zeros((n3, n, n))])
    u2 = transport2.deformation_map(v2, nt, "spline")
    u3 = d3.deformation_map(v3, nt, "spline")
    for c in range(2):
        assert np.max(np.abs(u3[c] - tile(u2[c]))) < 1e-12
    assert np.max(np.abs(u3[2])) < 1e-14
    assert np.max(np.abs(d3.det_grad_map(u3) - tile(spectral.det_grad_map(u2)))) < 1e-12


def test_det_grad_map_expansion_and_composition():
    """The first-row expansion equals numpy's determinant of I + grad u at
    every node; interpolating m_T at y reproduces the state solve's m_1 up to
    the interpolation error, which falls with the grid (16^3 -> 32^3)."""
    n, nt = 12, 4
    u = 0.4 * inputs.random_velocity3(n, n, n, seed=23, kmax=2, vmax=1.0)
    d = np.stack([d3.grad(u[a]) for a in range(3)])           # d[a, b] = d_b u_a
    J = np.moveaxis(d, (0, 1), (-2, -1)) + np.eye(3)
    assert np.max(np.abs(d3.det_grad_map(u) - np.linalg.det(J))) < 1e-12
    errs = []
    for n in (16, 32):
        m_T = inputs.random_field3(n, n, n, seed=24, kmax=2)
        v = inputs.random_velocity3(n, n, n, seed=25, kmax=2, vmax=0.3)
        m1 = d3.Problem3(np.zeros_like(m_T), m_T, nt, 1e-2).state_solve(v)
        uy = d3.deformation_map(v, nt)
        h = 2.0 * np.pi / n
        X = d3.node_coordinates(n, n, n)
        my = d3.interp(m_T, X[0] + uy[0] / h, X[1] + uy[1] / h, X[2] + uy[2] / h, "spline")
        errs.append(np.linalg.norm(my - m1) / np.linalg.norm(m1))
    assert errs[0] < 1e-2 and errs[1] < errs[0] / 4, errs


def test_restriction_prolongation_and_filters():
    """R of a mode below the cut-off is that mode on the coarse grid; R P = I
    on coarse fields without Nyquist modes; P R + H = I; on fields constant
    along x_3 all three reduce to the 2D operators."""
    from oracle import spectral
    n1, n2, n3 = 32, 16, 8
    x1, x2, x3 = grid3(n1, n2, n3)
    c1, c2, c3 = grid3(n1 // 2, n2 // 2, n3 // 2)
    f = lambda a, b, c: np.cos(2 * a - 3 * b + c) + 0.5 * np.sin(a + b)
    assert np.max(np.abs(d3.restrict3(f(x1, x2, x3)) - f(c1, c2, c3))) < 1e-12
    assert np.max(np.abs(d3.prolong3(f(c1, c2, c3)) - f(x1, x2, x3))) < 1e-12
    u = np.random.default_rng(3).standard_normal((n3, n2, n1))
    uc = d3.restrict3(u)
    assert np.max(np.abs(d3.restrict3(d3.prolong3(uc)) - uc)) < 1e-12
    assert np.max(np.abs(d3.prolong3(uc) + d3.highpass3(u) - u)) < 1e-12
    u2 = np.random.default_rng(4).standard_normal((n2, n1))
    tile = lambda a, k: np.repeat(a[None], k, axis=0)
    assert np.max(np.abs(d3.restrict3(tile(u2, n3)) - tile(spectral.restrict(u2), n3 // 2))) < 1e-12
    assert np.max(np.abs(d3.highpass3(tile(u2, n3)) - tile(spectral.highpass(u2), n3))) < 1e-12
    w2 = spectral.restrict(u2)
    assert np.max(np.abs(d3.prolong3(tile(w2, n3 // 2)) - tile(spectral.prolong(w2), n3))) < 1e-12


def test_solver3_two_level_reduces_to_the_2d_solve():
    """The Newton-Krylov solve with P_2L (CHEB(10) coarse solves) on a problem
    constant along x_3, v_3 = 0 and a Lanczos start vector likewise: every
    operator of the preconditioner reduces to the 2D one, so with the same
    Chebyshev bounds (the 3D coarse grid's e_min includes the x_3 modes; the
    2D solver takes it over) the iterations and the solution are the 2D
    oracle's; with P_REG Solver3 repeats Problem3.solve."""
    from oracle.solver import Solver
    n, n3, nt, beta, gtol = 16, 8, 4, 1e-2, 1e-2
    m_T, vstar = inputs.sinusoid_pair(n)
    m_R = Problem(np.zeros((n, n)), m_T, nt, beta).state_solve(vstar)
    tile = lambda a, k: np.repeat(a[None], k, axis=0)
    lv2 = inputs.splitmix64_uniform(2 * (n // 2) ** 2, 7).reshape(2, n // 2, n // 2)
    lv3 = np.stack([tile(lv2[0], n3 // 2), tile(lv2[1], n3 // 2), np.zeros((n3 // 2, n // 2, n // 2))])
    S3 = d3.Solver3(d3.Problem3(tile(m_R, n3), tile(m_T, n3), nt, beta), precond="2L", lanczos_v0=lv3)
    eig3 = S3.estimate_eigenvalues()
    S2 = Solver(Problem(m_R, m_T, nt, beta), precond="2L", lanczos_v0=lv2)
    eig2 = S2.estimate_eigenvalues()
    assert abs(eig3["emax"] - eig2["emax"]) < 1e-10 * eig2["emax"]
    assert eig3["emin"] < eig2["emin"]
    S2.eig["emin"] = eig3["emin"]
    v2, i2 = S2.solve(np.zeros((2, n, n)), gtol)
    v3, i3 = S3.solve(np.zeros((3, n3, n, n)), gtol)
    assert i3["newton_iters"] == i2["newton_iters"] and i3["matvecs"] == i2["matvecs"]
    assert i3["gnorm_rel"] <= gtol
    for c in range(2):
        assert np.max(np.abs(v3[c] - tile(v2[c], n3))) < 1e-8 * np.max(np.abs(v2))
    assert np.max(np.abs(v3[2])) < 1e-8 * np.max(np.abs(v2))
    m_T3 = inputs.random_field3(n, n, n, seed=41, kmax=2)
    m_R3 = d3.Problem3(np.zeros_like(m_T3), m_T3, nt, beta).state_solve(
        inputs.random_velocity3(n, n, n, seed=42, kmax=2, vmax=0.3))
    va, ia = d3.Problem3(m_R3, m_T3, nt, beta).solve(np.zeros((3, n, n, n)), gtol)
    vb, ib = d3.Solver3(d3.Problem3(m_R3, m_T3, nt, beta), precond="REG").solve(np.zeros((3, n, n, n)), gtol)
    assert ia["newton_iters"] == ib["newton_iters"] and ia["pcg_iters"] == ib["pcg_iters"]
    assert np.max(np.abs(va - vb)) == 0.0


def test_solver3_nested_pcg_reduces_to_the_2d_solve():
    """P_2L with nested PCG(eps eta) coarse solves on a problem constant along
    x_3: no Chebyshev bounds enter, so the 3D solve is the 2D oracle's
    (Newton steps, matvecs, coarse matvecs of the nested solves and the
    solution)."""
    from oracle.solver import Solver
    n, n3, nt, beta, gtol = 16, 8, 4, 1e-2, 1e-2
    m_T, vstar = inputs.sinusoid_pair(n)
    m_R = Problem(np.zeros((n, n)), m_T, nt, beta).state_solve(vstar)
    tile = lambda a, k: np.repeat(a[None], k, axis=0)
    S3 = d3.Solver3(d3.Problem3(tile(m_R, n3), tile(m_T, n3), nt, beta), precond="2L",
                    pc_solver="pcg")
    S2 = Solver(Problem(m_R, m_T, nt, beta), precond="2L", pc_solver="pcg")
    v2, i2 = S2.solve(np.zeros((2, n, n)), gtol)
    v3, i3 = S3.solve(np.zeros((3, n3, n, n)), gtol)
    assert i3["newton_iters"] == i2["newton_iters"] and i3["matvecs"] == i2["matvecs"]
    # the 2D solver runs its Lanczos estimate (30 coarse matvecs) before any
    # P_2L solve; Solver3 only when CHEB needs the bounds
    assert i3["coarse_matvecs"] == i2["coarse_matvecs"] - S2.lanczos_steps
    # CG to a tolerance on the coarse split operator (not symmetric to the
    # SL scheme's adjoint error) amplifies the FP64 rounding differences of
    # the 2D and 3D transforms: the iterates agree to 1e-14 after one Newton
    # step and 2.5e-5 after four, so the solution is held to the solve's 1e-3
    for c in range(2):
        assert np.max(np.abs(v3[c] - tile(v2[c], n3))) < 1e-3 * np.max(np.abs(v2))
    assert np.max(np.abs(v3[2])) < 1e-8 * np.max(np.abs(v2))
