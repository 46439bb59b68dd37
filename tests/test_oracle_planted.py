"""Planted mistakes in the oracle's incompressible, full-Newton, RK2A and
deformation-map parts, each caught by the pin that guards it (CPU only).

Every case swaps one oracle function for a plausibly wrong version (a flipped
sign, a dropped term, a transposed operand), re-runs the check its pin makes
and asserts that the check now fails.
"""

import numpy as np

from oracle import rk2a, spectral, transport
from oracle.problem import Problem
from paper_1604_02153_gb300 import inputs


def hodge_error(leray):
    n1, n2 = 32, 24
    X1, X2 = inputs.grid_coordinates(n1, n2)
    phi = np.cos(2 * X1 + X2) + 0.3 * np.sin(X1 - 3 * X2)
    psi = np.sin(X1 + 2 * X2) - 0.5 * np.cos(3 * X1 - X2)
    gphi = spectral.grad(phi)
    gpsi = spectral.grad(psi)
    sol = np.stack([-gpsi[1], gpsi[0]])
    return np.max(np.abs(leray(gphi + sol) - sol))


def test_leray_mistakes():
    assert hodge_error(spectral.leray) < 1e-12

    def flipped(b):                      # b + grad phi instead of b - grad phi
        return 2 * b - spectral.leray(b)

    def full_nyquist(b):                 # |k|^2 with the Nyquist mode kept
        n2, n1 = b.shape[1:]
        K1, K2 = spectral._k_grids(n1, n2, zero_nyquist=False)
        q = K1 * K1 + K2 * K2
        b1, b2 = np.fft.fft2(b[0]), np.fft.fft2(b[1])
        Kd1, Kd2 = spectral._k_grids(n1, n2, zero_nyquist=True)
        s = np.where(q > 0, (Kd1 * b1 + Kd2 * b2) / np.where(q > 0, q, 1), 0)
        return np.stack([np.real(np.fft.ifft2(b1 - Kd1 * s)), np.real(np.fft.ifft2(b2 - Kd2 * s))])

    def transposed(b):                   # components swapped in the projection
        return spectral.leray(b[::-1])[::-1]

    assert hodge_error(flipped) > 1e-2
    assert hodge_error(transposed) > 1e-2
    rng = np.random.default_rng(1)
    b = rng.standard_normal((2, 16, 16))
    assert np.max(np.abs(spectral.div(full_nyquist(b)))) > 1e-6   # not divergence free


def fn_fd_error(monkeypatch=None):
    n, nt = 32, 8
    m_T = inputs.random_field(n, seed=1, kmax=4)
    m_R = inputs.random_field(n, seed=2, kmax=4)
    v = inputs.random_velocity(n, seed=3, vmax=0.3)
    u = inputs.random_velocity(n, seed=9, vmax=1.0)
    P = Problem(m_R, m_T, nt, 1e-2, hessian="full")
    P.objective_gradient(v)
    H = P.hessian_matvec(u)
    G = Problem(m_R, m_T, nt, 1e-2)
    eps = 1e-4
    _, gp = G.objective_gradient(v + eps * u)
    _, gm = G.objective_gradient(v - eps * u)
    fd = (gp - gm) / (2 * eps)
    return np.linalg.norm(H - fd) / np.linalg.norm(fd)


def test_full_newton_mistakes(monkeypatch):
    assert fn_fd_error() < 2e-3
    good = transport.incadjoint_step_full

    def no_source(lt, dY, delta, dbar, sn, s, ht, kind):
        return good(lt, dY, delta, dbar, 0 * sn, 0 * s, ht, kind)

    def flipped_source(lt, dY, delta, dbar, sn, s, ht, kind):
        return good(lt, dY, delta, dbar, -sn, -s, ht, kind)

    for bad in (no_source, flipped_source):
        monkeypatch.setattr(transport, "incadjoint_step_full", bad)
        assert fn_fd_error() > 1e-2, bad.__name__
    monkeypatch.setattr(transport, "incadjoint_step_full", good)
    assert fn_fd_error() < 2e-3


def rk2a_adjoint_gap():
    n, nt = 32, 8
    v = inputs.random_velocity(n, seed=3, vmax=0.5)
    m0 = inputs.random_field(n, seed=1, kmax=6)
    fm = rk2a.state_solve(m0, v, nt)
    back = rk2a.adjoint_solve(fm, v, nt)
    return abs(np.sum(fm * fm) - np.sum(back * m0)) / np.sum(fm * fm)


def test_rk2a_mistakes(monkeypatch):
    assert rk2a_adjoint_gap() < 1e-13
    good = rk2a.adjoint_rhs

    def wrong_div_sign(lam, v, delta):       # lambda div v with the state's sign
        return good(lam, v, delta) - lam * delta

    def advective_only(lam, v, delta):       # the antisymmetric half dropped
        g = spectral.grad(lam)
        return g[0] * v[0] + g[1] * v[1]

    for bad in (wrong_div_sign, advective_only):
        monkeypatch.setattr(rk2a, "adjoint_rhs", bad)
        assert rk2a_adjoint_gap() > 1e-6, bad.__name__


def shear_error(deformation_map):
    n, nt, a = 32, 8, 0.4
    X1, X2 = inputs.grid_coordinates(n, n)
    v = np.stack([a * np.sin(X2), np.zeros_like(X2)])
    u = deformation_map(v, nt, "spline")
    return max(np.max(np.abs(u[0] + a * np.sin(X2))), np.max(np.abs(u[1])))


def test_deformation_map_mistakes(monkeypatch):
    assert shear_error(transport.deformation_map) < 1e-12

    def last_step_only(v, nt, kind):       # the departure displacement not carried along
        n2, n1 = v.shape[1:]
        h = (2 * np.pi / n1, 2 * np.pi / n2)
        dX = transport.characteristic(v, nt, kind, backward=False)
        return np.stack([h[0] * dX[0], h[1] * dX[1]])

    def forward_map(v, nt, kind):          # the forward characteristic instead of the backward one
        return -transport.deformation_map(v, nt, kind)

    for bad in (last_step_only, forward_map):
        assert shear_error(bad) > 1e-2, bad.__name__
