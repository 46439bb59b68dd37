"""Pins of the oracle's near-incompressible variant (CPU only).

The mass source w of eq. varopt carries the H1 norm of eq. varopt:regw and is
tied to the velocity by eq. icconstraint, w = div v, so J adds
beta_w/2 ||div v||^2_H1 = 1/2 <v, (M - beta A) v>,
M = beta A - beta_w grad (I - Lap) div. Eliminating w and p from the control
equations (Appendix A, eq. control-v, eq. control-w) leaves M v + b = 0,
which in the paper's form beta A v + K[b] = 0 (eq. control-elim) fixes
K = beta A M^-1 (identity on the mean). Pinned here against what the
mathematics fixes:
* trigonometric polynomials: on a gradient field grad phi the term is
  beta_w |k|^2 (1 + |k|^2) grad phi exactly, on a divergence-free field zero;
* it is the derivative of the quadratic (beta_w / 2) ||div v||^2_{H1} written
  out from its definition (w, grad w and the midpoint sum), checked by central
  differences (exact for a quadratic up to roundoff), symmetric and positive;
* the powers R^s of R = beta A - beta_w grad (I - Lap) div: R^-1 R = I,
  R^1/2 R^1/2 = R, and R^s = (beta A)^s for beta_w = 0;
* K on trigonometric polynomials: a gradient field scales by
  beta |k|^2 / (beta |k|^2 + beta_w (1 + |k|^2) |k|^2), a divergence-free
  field is kept; K tends to the Leray projection as beta_w grows;
* the L2 gradient R v + b matches central differences of J, the reduced
  gradient and Hessian are K of the L2 ones, and beta_w = 0 is the
  compressible problem;
* beta_w -> infinity: the solution approaches the incompressible (Leray)
  solution and its divergence vanishes.
"""

import numpy as np
import pytest

from oracle import spectral
from oracle.problem import Problem
from oracle.solver import Solver
from paper_1604_02153_gb300 import inputs


def _grid(n1, n2):
    x1 = 2 * np.pi * np.arange(n1) / n1
    x2 = 2 * np.pi * np.arange(n2) / n2
    X2, X1 = np.meshgrid(x2, x1, indexing="ij")
    return X1, X2


def test_reg_w_term_on_trigonometric_polynomials():
    n1, n2, bw = 32, 24, 0.7
    X1, X2 = _grid(n1, n2)
    a, b = 3, -2
    phi = np.cos(a * X1 + b * X2)
    gphi = np.stack([-a * np.sin(a * X1 + b * X2), -b * np.sin(a * X1 + b * X2)])
    k2 = a * a + b * b
    got = spectral.reg_w_term(gphi, bw)
    assert np.max(np.abs(got - bw * k2 * (1 + k2) * gphi)) < 1e-10 * bw * k2 * (1 + k2)
    # divergence free: the perpendicular gradient of psi
    psi = np.sin(2 * X1 - 5 * X2)
    rot = np.stack([-(-5) * np.cos(2 * X1 - 5 * X2), 2 * np.cos(2 * X1 - 5 * X2)])
    assert np.max(np.abs(spectral.div(rot))) < 1e-11
    # zero up to roundoff amplified by the symbol (|k|^2 = 29 here)
    scale = bw * 29 * 30 * np.max(np.abs(rot))
    assert np.max(np.abs(spectral.reg_w_term(rot, bw))) < 1e-12 * scale


def test_reg_w_term_is_derivative_of_divergence_norm():
    n1, n2, bw = 48, 32, 0.3
    h = (2 * np.pi / n1) * (2 * np.pi / n2)
    v = inputs.random_velocity(n1, n2, seed=3, kmax=10, vmax=1.0)
    u = inputs.random_velocity(n1, n2, seed=4, kmax=10, vmax=1.0)
    z = inputs.random_velocity(n1, n2, seed=5, kmax=10, vmax=1.0)

    def quad(x):
        # (beta_w / 2) int |grad w|^2 + w^2 dx with w = div x (midpoint sum)
        w = spectral.div(x)
        gw = spectral.grad(w)
        return 0.5 * bw * h * float(np.sum(gw[0] ** 2 + gw[1] ** 2 + w ** 2))

    eps = 1e-3
    fd = (quad(v + eps * u) - quad(v - eps * u)) / (2 * eps)
    an = h * float(np.sum(spectral.reg_w_term(v, bw) * u))
    assert abs(fd - an) < 1e-9 * abs(fd)
    Ru, Rz = spectral.reg_w_term(u, bw), spectral.reg_w_term(z, bw)
    assert abs(np.sum(Ru * z) - np.sum(u * Rz)) < 1e-10 * abs(np.sum(Ru * z))
    assert np.sum(Ru * u) > 0
    # a flipped sign fails the derivative check by O(1)
    assert abs(fd + an) > 0.5 * abs(fd)


@pytest.mark.parametrize("norm", ["H1", "H2"])
def test_regop_powers(norm):
    n1, n2, beta, bw = 32, 16, 0.05, 0.4
    v = inputs.random_velocity(n1, n2, seed=6, kmax=7, vmax=1.0)
    R = lambda x, s: spectral.regop_power(x, beta, norm, bw, s)
    Rv = spectral.apply_regop(v, beta, norm, bw)
    assert np.max(np.abs(R(v, 1.0) - Rv)) < 1e-10 * np.max(np.abs(Rv))
    # R^-1 R v = v up to the k = 0 mode (weight replaced by 1 in R^-1)
    v0 = v - v.mean(axis=(1, 2), keepdims=True)
    back = R(spectral.apply_regop(v0, beta, norm, bw), -1.0)
    assert np.max(np.abs(back - v0)) < 1e-10 * np.max(np.abs(v0))
    assert np.max(np.abs(R(R(v, 0.5), 0.5) - R(v, 1.0))) < 1e-9 * np.max(np.abs(Rv))
    assert np.max(np.abs(R(R(v, -0.5), -0.5) - R(v, -1.0))) < 1e-12 * np.max(np.abs(R(v, -1.0)))
    for s in (-1.0, -0.5, 0.5):
        assert np.max(np.abs(spectral.regop_power(v, beta, norm, 0.0, s) -
                             spectral.reg_power(v, beta, norm, s))) < 1e-12


def _pair(n, nt, seed=1):
    m_T = inputs.random_field(n, seed=seed, kmax=4)
    m_R = inputs.random_field(n, seed=seed + 1, kmax=4)
    return m_R, m_T


def test_gradient_against_finite_differences():
    n, nt = 64, 16
    m_R, m_T = _pair(n, nt)
    v = inputs.random_velocity(n, seed=3, vmax=0.05)
    dv = inputs.random_velocity(n, seed=4, kmax=6, vmax=1.0)
    eps = 1e-4
    slopes = {}
    for bw in (0.5, 0.0):
        P = Problem(m_R, m_T, nt, 1e-2, beta_w=bw)
        g = P.gradient_l2(v)
        d = P.inner(g, dv)
        fd = (P.objective(v + eps * dv) - P.objective(v - eps * dv)) / (2 * eps)
        slopes[bw] = (fd, d)
    fd, d = slopes[0.5]
    # the transport part carries the optimise-then-discretise gap of the SL
    # scheme (a few 1e-5 at 64^2, see the compressible pin); the beta_w term
    # adds none: its slope is exact, so both gaps coincide to roundoff
    assert abs(fd - d) < 1e-4 * abs(d)
    gap_w = fd - d
    gap_c = slopes[0.0][0] - slopes[0.0][1]
    assert abs(gap_w - gap_c) < 1e-9 * abs(d)
    # the beta_w term matters at this size: without it the slope is off
    wterm = P.inner(spectral.reg_w_term(v, 0.5), dv)
    assert abs(wterm) > 1e-2 * abs(d)
    # beta_w = 0 is the compressible problem
    Pc = Problem(m_R, m_T, nt, 1e-2)
    P0 = Problem(m_R, m_T, nt, 1e-2, beta_w=0.0)
    Jc, gc = Pc.objective_gradient(v)
    J0, g0 = P0.objective_gradient(v)
    assert Jc == J0 and np.array_equal(gc, g0)


def test_K_on_trigonometric_polynomials_and_limits():
    n1, n2, beta = 32, 24, 0.02
    X1, X2 = _grid(n1, n2)
    a, b = 3, -2
    k2 = a * a + b * b
    gphi = np.stack([-a * np.sin(a * X1 + b * X2), -b * np.sin(a * X1 + b * X2)])
    rot = np.stack([5 * np.cos(2 * X1 - 5 * X2), 2 * np.cos(2 * X1 - 5 * X2)])
    for bw in (1e-3, 0.1, 10.0):
        scale = beta * k2 / (beta * k2 + bw * (1 + k2) * k2)
        Kg = spectral.near_inc_K(gphi, beta, "H1", bw)
        assert np.max(np.abs(Kg - scale * gphi)) < 1e-11, bw
        assert np.max(np.abs(spectral.near_inc_K(rot, beta, "H1", bw) - rot)) < 1e-11, bw
    # limits on a random field (modes |k| <= 8): identity as beta_w -> 0, the
    # Leray projection as beta_w -> infinity, with the gap 1 - c of the
    # gradient part below beta |k|^2 / (beta_w (1 + |k|^2) |k|^2) <= beta / (2 beta_w)
    w = inputs.random_velocity(n1, n2, seed=8, kmax=8, vmax=1.0)
    assert np.max(np.abs(spectral.near_inc_K(w, beta, "H1", 1e-12) - w)) < 1e-8
    gaps = [np.linalg.norm(spectral.near_inc_K(w, beta, "H1", bw) - spectral.leray(w))
            / np.linalg.norm(w) for bw in (1.0, 1e3)]
    assert gaps[1] < beta / (2 * 1e3) and gaps[0] > 100 * gaps[1], gaps


def test_reduced_gradient_and_hessian_are_K_of_the_L2_ones():
    n, nt = 32, 8
    m_R, m_T = _pair(n, nt)
    v = inputs.random_velocity(n, seed=3, vmax=0.1)
    u = inputs.random_velocity(n, seed=7, kmax=6, vmax=1.0)
    bw = 2.0
    P = Problem(m_R, m_T, nt, 1e-2, beta_w=bw)
    J, g = P.objective_gradient(v)
    gl2 = P.gradient_l2(v)
    K = lambda x: spectral.near_inc_K(x, P.beta, "H1", bw)
    assert np.max(np.abs(g - K(gl2))) < 1e-10 * np.max(np.abs(g))
    # the Hessian: beta A u + K[b~] = K[R u + b~]
    Pc = Problem(m_R, m_T, nt, 1e-2)
    Pc.state_solve(v)
    P.state_solve(v)
    bt = Pc.hessian_matvec(u) - spectral.apply_reg(u, 1e-2, "H1")   # K = I: the data term b~
    Hu = P.hessian_matvec(u)
    assert np.max(np.abs(Hu - K(spectral.apply_regop(u, 1e-2, "H1", bw) + bt))) < 1e-10 * np.max(np.abs(Hu))
    assert np.max(np.abs(Hu - (spectral.apply_reg(u, 1e-2, "H1") + bt))) > 1e-3 * np.max(np.abs(Hu))


def test_large_beta_w_approaches_the_incompressible_solution():
    """The near-incompressible solve penalises div v: as beta_w grows its
    solution approaches the solution of the incompressible problem (Leray
    projection, w = 0) and its divergence vanishes."""
    n, nt, beta = 32, 4, 1e-2
    m_T, _ = inputs.sinusoid_pair(n)
    vstar = spectral.leray(inputs.random_velocity(n, seed=11, kmax=3, vmax=0.4))
    vstar = vstar + 0.3 * spectral.grad(inputs.random_field(n, seed=12, kmax=2) - 0.5)
    m_R = Problem(np.zeros((n, n)), m_T, nt, beta).state_solve(vstar)
    z = np.zeros((2, n, n))
    vi, _ = Solver(Problem(m_R, m_T, nt, beta, incompressible=True), precond="REG").solve(z, 1e-3)
    vc, _ = Solver(Problem(m_R, m_T, nt, beta), precond="REG").solve(z, 1e-3)
    dist, divn = [], []
    for bw in (1e-2, 1.0, 1e2):
        vw, info = Solver(Problem(m_R, m_T, nt, beta, beta_w=bw), precond="REG").solve(z, 1e-3)
        dist.append(np.linalg.norm(vw - vi) / np.linalg.norm(vi))
        divn.append(np.linalg.norm(spectral.div(vw)) / np.linalg.norm(vw))
    assert dist[0] > dist[1] > dist[2], dist
    assert dist[2] < 0.1 * dist[0], dist
    assert divn[0] > divn[1] > divn[2], divn
    # and the smallest beta_w stays near the compressible solution
    vw0, _ = Solver(Problem(m_R, m_T, nt, beta, beta_w=1e-6), precond="REG").solve(z, 1e-3)
    assert np.linalg.norm(vw0 - vc) < 1e-3 * np.linalg.norm(vc)
