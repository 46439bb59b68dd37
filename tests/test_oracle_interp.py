"""Pins of the oracle's periodic cubic interpolation (CPU only).

* interpolating property at the nodes (both weight families);
* cubic Lagrange is exact on cubic polynomials away from the wrap;
* the spline model equals an independent library C2 periodic cubic spline
  (scipy.interpolate.CubicSpline, bc_type="periodic") in 1D and its tensor
  product in 2D (§3.5 "Interpolation": C2-continuous cubic spline);
* fourth-order convergence on smooth periodic functions.
"""

import numpy as np
import pytest
from scipy.interpolate import CubicSpline

from oracle import interp


@pytest.mark.parametrize("kind", ["spline", "lagrange"])
def test_interpolates_at_nodes(kind):
    rng = np.random.default_rng(0)
    u = rng.standard_normal((12, 16))
    I, J = interp.node_coordinates(16, 12)
    for s1, s2 in [(0, 0), (3, -2), (-17, 25)]:
        got = interp.interp(u, I + s1, J + s2, kind)
        expect = np.roll(np.roll(u, -s1, axis=1), -s2, axis=0)
        assert np.max(np.abs(got - expect)) < 1e-12


def test_lagrange_exact_on_cubics():
    n = 32
    rng = np.random.default_rng(1)
    coef = rng.standard_normal((4, 4))
    I, J = interp.node_coordinates(n, n)
    u = sum(coef[a, b] * I ** a * J ** b for a in range(4) for b in range(4))
    p1 = rng.uniform(4, n - 5, 200)
    p2 = rng.uniform(4, n - 5, 200)
    exact = sum(coef[a, b] * p1 ** a * p2 ** b for a in range(4) for b in range(4))
    got = interp.interp(u, p1, p2, "lagrange")
    assert np.max(np.abs(got - exact)) < 1e-8 * np.max(np.abs(exact))


def test_spline_matches_library_periodic_spline_1d_and_tensor():
    n1, n2 = 24, 20
    rng = np.random.default_rng(2)
    f = rng.standard_normal(n1)
    g = rng.standard_normal(n2)
    u = g[:, None] * f[None, :]
    p1 = rng.uniform(-30, 30, 300)
    p2 = rng.uniform(-30, 30, 300)
    cs_f = CubicSpline(np.arange(n1 + 1), np.append(f, f[0]), bc_type="periodic")
    cs_g = CubicSpline(np.arange(n2 + 1), np.append(g, g[0]), bc_type="periodic")
    expect = cs_f(np.mod(p1, n1)) * cs_g(np.mod(p2, n2))
    got = interp.interp(u, p1, p2, "spline")
    assert np.max(np.abs(got - expect)) < 1e-12


@pytest.mark.parametrize("kind,order", [("spline", 4), ("lagrange", 4)])
def test_fourth_order_convergence(kind, order):
    errs = []
    rng = np.random.default_rng(3)
    q1 = rng.uniform(0, 2 * np.pi, 500)
    q2 = rng.uniform(0, 2 * np.pi, 500)
    exact = np.sin(q1 + 0.3) * np.cos(2 * q2) + 0.5 * np.cos(q1 - q2)
    for n in (32, 64, 128):
        h = 2 * np.pi / n
        I, J = interp.node_coordinates(n, n)
        X1, X2 = I * h, J * h
        u = np.sin(X1 + 0.3) * np.cos(2 * X2) + 0.5 * np.cos(X1 - X2)
        got = interp.interp(u, q1 / h, q2 / h, kind)
        errs.append(np.max(np.abs(got - exact)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > order - 0.3), (errs, rates)


def test_weights_partition_of_unity():
    t = np.linspace(0, 1, 11)
    for fn in (interp.bspline3_weights, interp.lagrange3_weights):
        assert np.max(np.abs(sum(fn(t)) - 1.0)) < 1e-14
