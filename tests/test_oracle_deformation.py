"""Pins of the oracle's deformation map and det grad y (CPU only).

* shear flow v = (a sin x2, 0): y(x) = (x1 - a sin x2, x2) exactly, det = 1;
* constant velocity c: y = x - c, det = 1;
* m_T interpolated at y equals the SL state solve's m_1 up to interpolation
  error, which falls with the grid;
* divergence-free v keeps det grad y at 1 up to discretisation error, which
  falls with the grid; a compressive v moves it by O(0.1).
"""

import numpy as np
import pytest

from oracle import interp, spectral, transport
from oracle.problem import Problem
from paper_1604_02153_gb300 import inputs


@pytest.mark.parametrize("kind", ["spline", "lagrange"])
def test_shear_flow_closed_form(kind):
    n, nt, a = 64, 8, 0.4
    X1, X2 = inputs.grid_coordinates(n, n)
    v = np.stack([a * np.sin(X2), np.zeros_like(X2)])
    u = transport.deformation_map(v, nt, kind)
    assert np.max(np.abs(u[0] + a * np.sin(X2))) < 1e-12
    assert np.max(np.abs(u[1])) < 1e-12
    assert np.max(np.abs(spectral.det_grad_map(u) - 1.0)) < 1e-12


def test_constant_velocity():
    n, nt = 32, 5
    c = (0.3, -0.8)
    v = np.stack([np.full((n, n), c[0]), np.full((n, n), c[1])])
    u = transport.deformation_map(v, nt, "spline")
    assert np.max(np.abs(u[0] + c[0])) < 1e-13 and np.max(np.abs(u[1] + c[1])) < 1e-13
    assert np.max(np.abs(spectral.det_grad_map(u) - 1.0)) < 1e-13


def test_template_at_map_matches_state_solve():
    gaps = []
    for n in (64, 128):
        nt = 8
        m_T = inputs.random_field(n, seed=1, kmax=4)
        v = inputs.random_velocity(n, seed=3, vmax=0.4)
        u = transport.deformation_map(v, nt, "spline")
        I, J = interp.node_coordinates(n, n)
        h = 2.0 * np.pi / n
        my = interp.interp(m_T, I + u[0] / h, J + u[1] / h, "spline")
        m1 = Problem(np.zeros((n, n)), m_T, nt, 1e-2).state_solve(v)
        gaps.append(np.linalg.norm(my - m1) / np.linalg.norm(m1))
    assert gaps[0] < 1e-3 and gaps[1] < gaps[0] / 4, gaps


def test_jacobian_determinant_incompressible_versus_compressible():
    errs = []
    for n in (64, 128):
        v = spectral.leray(inputs.random_velocity(n, seed=5, vmax=0.4))
        det = spectral.det_grad_map(transport.deformation_map(v, 32, "spline"))
        errs.append(np.max(np.abs(det - 1.0)))
    assert errs[0] < 1e-4 and errs[1] < errs[0] / 4, errs
    n = 64
    vc = inputs.random_velocity(n, seed=5, vmax=0.4)
    vc = vc - spectral.leray(vc)                     # a pure gradient field
    det = spectral.det_grad_map(transport.deformation_map(vc, 8, "spline"))
    assert np.max(np.abs(det - 1.0)) > 0.05
