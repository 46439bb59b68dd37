"""Pins of the oracle's spectral operators against closed forms (CPU only).

Each operator is checked on trigonometric polynomials, where the continuous
operator has a closed form and the pseudospectral one is exact (§3.2), and on
identities that a plausible mistake (wrong sign, transposed axis, missing
scale, wrong Nyquist handling) would break.
"""

import numpy as np
import pytest

from oracle import spectral
from paper_1604_02153_gb300.inputs import grid_coordinates


def trig_poly(n1, n2, modes, seed):
    """Random trig polynomial and its analytic d/dx1, d/dx2 and Laplacian."""
    rng = np.random.default_rng(seed)
    X1, X2 = grid_coordinates(n1, n2)
    u = np.zeros((n2, n1))
    d1 = np.zeros_like(u)
    d2 = np.zeros_like(u)
    lap = np.zeros_like(u)
    for (k1, k2) in modes:
        a, b = rng.standard_normal(2)
        ph = k1 * X1 + k2 * X2
        u += a * np.cos(ph) + b * np.sin(ph)
        d1 += k1 * (-a * np.sin(ph) + b * np.cos(ph))
        d2 += k2 * (-a * np.sin(ph) + b * np.cos(ph))
        lap += -(k1 * k1 + k2 * k2) * (a * np.cos(ph) + b * np.sin(ph))
    return u, d1, d2, lap


MODES = [(0, 0), (1, 0), (0, 1), (3, -2), (-5, 7), (7, 3), (2, 9)]


@pytest.mark.parametrize("n1,n2", [(32, 32), (32, 24), (20, 32)])
def test_gradient_exact_on_trig_polynomials(n1, n2):
    u, d1, d2, _ = trig_poly(n1, n2, [m for m in MODES if abs(m[0]) < n1 / 2 and abs(m[1]) < n2 / 2], 1)
    g = spectral.grad(u)
    assert np.max(np.abs(g[0] - d1)) < 1e-11
    assert np.max(np.abs(g[1] - d2)) < 1e-11


def test_divergence_exact():
    n = 32
    u, d1, _, _ = trig_poly(n, n, MODES, 2)
    w, _, e2, _ = trig_poly(n, n, MODES, 3)
    dv = spectral.div(np.stack([u, w]))
    assert np.max(np.abs(dv - (d1 + e2))) < 1e-11


def test_nyquist_zeroed_in_first_derivative():
    n = 16
    X1, X2 = grid_coordinates(n, n)
    u = np.cos(8 * X1)   # the Nyquist mode of a 16-point grid
    g = spectral.grad(u)
    assert np.max(np.abs(g)) < 1e-12


@pytest.mark.parametrize("norm,p", [("H1", 1), ("H2", 2), ("H3", 3)])
def test_regularisation_operator(norm, p):
    """A = -Lap, Lap^2, -Lap^3 (eq. diffopregv): symbol |k|^(2p), checked by
    applying the analytic Laplacian p times."""
    n = 32
    u, _, _, lap = trig_poly(n, n, MODES, 4)
    beta = 0.37
    Au = spectral.apply_reg(np.stack([u, u]), beta, norm)[0]
    # build (-Lap)^p u from the closed-form Laplacian of each mode
    rng_modes = MODES
    expect = np.zeros_like(u)
    rng = np.random.default_rng(4)
    X1, X2 = grid_coordinates(n, n)
    for (k1, k2) in rng_modes:
        a, b = rng.standard_normal(2)
        ph = k1 * X1 + k2 * X2
        expect += (k1 * k1 + k2 * k2) ** p * (a * np.cos(ph) + b * np.sin(ph))
    assert np.max(np.abs(Au - beta * expect)) < 1e-9 * max(1.0, np.max(np.abs(expect)))
    if p == 1:
        assert np.max(np.abs(Au + beta * lap)) < 1e-10


def test_reg_powers_and_null_space():
    """(beta A)^s with the k=0 weight replaced by one (eq. reg-precond)."""
    n = 32
    beta = 1e-2
    u, _, _, lap = trig_poly(n, n, MODES, 5)
    v = np.stack([u, 2 * u])
    inv = spectral.reg_power(v, beta, "H1", -1.0)
    back = spectral.apply_reg(inv, beta, "H1")
    mean = np.mean(v, axis=(1, 2), keepdims=True)
    # A kills the mean, the inverse maps the mean to mean / beta
    assert np.max(np.abs(back - (v - mean))) < 1e-10
    assert np.allclose(np.mean(inv, axis=(1, 2)), mean[:, 0, 0] / beta, atol=1e-10)
    half = spectral.reg_power(v, beta, "H2", -0.5)
    twice = spectral.reg_power(half, beta, "H2", -0.5)
    assert np.max(np.abs(twice - spectral.reg_power(v, beta, "H2", -1.0))) < 1e-10
    up = spectral.reg_power(half, beta, "H2", 0.5)
    assert np.max(np.abs(up - v)) < 1e-10


def test_restriction_prolongation():
    """R P = I on coarse fields without Nyquist; P R = low-pass; R of a trig
    polynomial with |k_i| < n_i/4 is its coarse samples (§3.4.2)."""
    n = 32
    low = [(0, 0), (1, 2), (-3, 5), (7, -7), (4, 0)]
    uf, *_ = trig_poly(n, n, low, 6)
    uc, *_ = trig_poly(n // 2, n // 2, low, 6)
    assert np.max(np.abs(spectral.restrict(uf) - uc)) < 1e-12
    assert np.max(np.abs(spectral.prolong(uc) - uf)) < 1e-12
    rng = np.random.default_rng(7)
    w = rng.standard_normal((n, n))
    assert np.max(np.abs(spectral.prolong(spectral.restrict(w)) - spectral.lowpass(w))) < 1e-12
    c = spectral.restrict(w)
    assert np.max(np.abs(spectral.restrict(spectral.prolong(c)) - c)) < 1e-12
    assert np.max(np.abs(spectral.lowpass(w) + spectral.highpass(w) - w)) < 1e-12
    # adjoint relation P = (N_f / N_c) R^T in the Euclidean inner product
    z = rng.standard_normal((n // 2, n // 2))
    lhs = np.sum(spectral.prolong(z) * w)
    rhs = 4.0 * np.sum(z * spectral.restrict(w))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_fft_against_brute_force_dft():
    """numpy's FFT (the library primitive) equals the O(n^4) DFT sum at 16^2."""
    n = 16
    rng = np.random.default_rng(8)
    u = rng.standard_normal((n, n))
    j = np.arange(n)
    E = np.exp(-2j * np.pi * np.outer(j, j) / n)
    dft = E @ u @ E.T
    assert np.max(np.abs(dft - spectral.fft2(u))) < 1e-11


def test_spline_symbol_matches_bspline_samples():
    """Sampling a B-spline series multiplies by (2 + cos w)/3 per axis."""
    n = 16
    rng = np.random.default_rng(9)
    c = rng.standard_normal((n, n))
    # direct sampling: u[j,i] = sum c[j+b, i+a] * beta3(a) beta3(b), beta3(0)=2/3, beta3(+-1)=1/6
    w = {-1: 1 / 6, 0: 2 / 3, 1: 1 / 6}
    u = np.zeros_like(c)
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            u += w[a] * w[b] * np.roll(np.roll(c, -a, axis=1), -b, axis=0)
    assert np.max(np.abs(spectral.spline_prefilter(u) - c)) < 1e-12


def test_leray_keeps_solenoidal_part_of_hodge_decomposition():
    """b = grad phi + curl psi + const (curl psi = (-d2 psi, d1 psi)): the
    Leray projection (§3.1, K[b] = -grad Lap^-1 div b + b) removes exactly
    the gradient part."""
    n1, n2 = 32, 24
    modes = [(1, 0), (0, 1), (3, -2), (-5, 7), (7, 3), (2, 9)]
    phi, p1, p2, _ = trig_poly(n1, n2, modes, seed=41)
    psi, s1, s2, _ = trig_poly(n1, n2, modes, seed=42)
    const = np.array([0.3, -0.7])[:, None, None]
    sol = np.stack([-s2, s1]) + const
    b = np.stack([p1, p2]) + sol
    assert np.max(np.abs(spectral.leray(b) - sol)) < 1e-12 * np.max(np.abs(b))
    assert np.max(np.abs(spectral.leray(np.stack([p1, p2])))) < 1e-12 * np.max(np.abs(p1))
    assert np.max(np.abs(spectral.leray(sol) - sol)) < 1e-12


@pytest.mark.parametrize("n1,n2", [(16, 16), (16, 12), (12, 20)])
def test_leray_is_an_orthogonal_projector_onto_discretely_solenoidal_fields(n1, n2):
    rng = np.random.default_rng(n1 * 100 + n2)
    a = rng.standard_normal((2, n2, n1))     # all modes, Nyquist lines included
    b = rng.standard_normal((2, n2, n1))
    Ka, Kb = spectral.leray(a), spectral.leray(b)
    scale = np.max(np.abs(b))
    assert np.max(np.abs(spectral.div(Kb))) < 1e-12 * n1 * scale
    assert np.max(np.abs(spectral.leray(Kb) - Kb)) < 1e-12 * scale
    assert abs(np.sum(Ka * b) - np.sum(a * Kb)) < 1e-11 * np.sum(np.abs(a * b))
    assert abs(np.sum(Kb * (b - Kb))) < 1e-11 * np.sum(b * b)
    # a field that is a gradient is removed entirely
    g = spectral.grad(rng.standard_normal((n2, n1)))
    assert np.max(np.abs(spectral.leray(g))) < 1e-11 * np.max(np.abs(g))


def test_leray_matches_dense_projection_built_from_grad_and_div():
    """Brute force on a 6 x 8 grid: the matrix of K equals
    I - G (D G)^+ D with G, D the dense matrices of the (pinned) spectral
    gradient and divergence; (D G)^+ is the pseudo-inverse, which leaves the
    modes where div(grad .) vanishes untouched."""
    n1, n2 = 8, 6
    N = n1 * n2
    G = np.zeros((2 * N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        G[:, j] = spectral.grad(e.reshape(n2, n1)).ravel()
    D = np.zeros((N, 2 * N))
    Kmat = np.zeros((2 * N, 2 * N))
    for j in range(2 * N):
        e = np.zeros(2 * N)
        e[j] = 1.0
        D[:, j] = spectral.div(e.reshape(2, n2, n1)).ravel()
        Kmat[:, j] = spectral.leray(e.reshape(2, n2, n1)).ravel()
    K_bf = np.eye(2 * N) - G @ np.linalg.pinv(D @ G, rcond=1e-10) @ D
    assert np.max(np.abs(Kmat - K_bf)) < 1e-12
