"""Pins of the oracle's RK2A comparator (Appendix "RK2A derivation"; CPU only).

* the discrete adjoint is the exact transpose of the state solve: the
  paper's δ_ADJ (§4.1.3) at machine precision, against 1e-6..1e-3 for SL;
* the spatial operator of the state equation is skew for a divergence-free
  velocity (<m, A m> = 0), the property the antisymmetric form is built for;
* constant velocity: the exact solution is a shift; Heun's error falls by
  4x per halving of h_t (second order) for a band-limited field;
* SL converges to the RK2A reference as the grid is refined (the trend of
  the paper's table "Convergence of SL to RK2A").
"""

import numpy as np

from oracle import rk2a, spectral
from oracle.problem import Problem
from paper_1604_02153_gb300 import inputs


def delta_adj(forward, adjoint, m0):
    fm = forward(m0)
    a = float(np.sum(fm * fm))
    b = float(np.sum(adjoint(fm) * m0))
    return abs(a - b) / abs(a)


def test_rk2a_adjoint_is_the_exact_transpose():
    n, nt = 64, 16
    v = inputs.random_velocity(n, seed=3, vmax=0.5)
    m0 = inputs.random_field(n, seed=1, kmax=8)
    d = delta_adj(lambda m: rk2a.state_solve(m, v, nt), lambda l: rk2a.adjoint_solve(l, v, nt), m0)
    assert d < 1e-13, d
    # SL's forward and adjoint solves are not transposes of each other
    P = Problem(np.zeros((n, n)), m0, nt, 1e-2)
    P.state_solve(v)

    def sl_adjoint(lam1):
        P.m_R = lam1 + P.m[-1]            # lambda(1) = m_R - m_1 = lam1
        return P.adjoint_solve()[0]

    d_sl = delta_adj(lambda m: Problem(np.zeros((n, n)), m, nt, 1e-2).state_solve(v), sl_adjoint, m0)
    assert d_sl > 100 * d, (d_sl, d)


def test_state_operator_is_skew_for_divergence_free_velocity():
    n = 48
    v = spectral.leray(inputs.random_velocity(n, seed=5, vmax=1.0))
    delta = spectral.div(v)
    m = inputs.random_field(n, seed=2, kmax=12)
    Am = rk2a.state_rhs(m, v, delta)
    assert abs(np.sum(m * Am)) < 1e-12 * np.sum(np.abs(m * Am))
    # and the adjoint operator is its negative there
    x = inputs.random_field(n, seed=4, kmax=12)
    assert abs(np.sum(x * Am) - np.sum(rk2a.adjoint_rhs(x, v, delta) * m)) < 1e-12 * np.sum(np.abs(x * Am))


def test_constant_velocity_shift_second_order_in_time():
    n = 64
    X1, X2 = inputs.grid_coordinates(n, n)
    c = np.array([0.7, -0.4])
    v = np.stack([np.full((n, n), c[0]), np.full((n, n), c[1])])
    m0 = np.sin(3 * X1 + X2) + 0.5 * np.cos(X1 - 2 * X2)
    exact = np.sin(3 * (X1 - c[0]) + (X2 - c[1])) + 0.5 * np.cos((X1 - c[0]) - 2 * (X2 - c[1]))
    errs = [np.max(np.abs(rk2a.state_solve(m0, v, nt) - exact)) for nt in (16, 32, 64)]
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs
    assert errs[-1] < 1e-3


def test_sl_converges_to_rk2a_reference():
    """Reference: RK2A at CFL 0.2 on 256^2 (SMOOTH A-like data: band-limited
    field, smooth velocity). SL at the same CFL on n = 64, 128 (compared
    after spectral prolongation): the error falls with n."""
    nref = 256
    m0f = inputs.random_field(nref, seed=1, kmax=6)
    vf = inputs.random_velocity(nref, seed=3, kmax=3, vmax=0.5)
    nt_ref = rk2a.cfl_steps(vf, 0.2)
    ref = rk2a.state_solve(m0f, vf, nt_ref)
    errs = []
    for levels in (2, 1):                 # n = 64, 128
        m0, v = m0f, vf
        for _ in range(levels):
            m0, v = spectral.restrict(m0), spectral.restrict_vec(v)
        n = m0.shape[0]
        nt = rk2a.cfl_steps(v, 0.2)
        up = Problem(np.zeros((n, n)), m0, nt, 1e-2).state_solve(v)
        for _ in range(levels):
            up = spectral.prolong(up)
        errs.append(np.linalg.norm(up - ref) / np.linalg.norm(ref))
    assert errs[1] < errs[0] / 2, errs
    assert errs[1] < 1e-2, errs


def test_sl_error_grows_with_cfl_number():
    """Table t:convergence-SL-to-RK2A-transporteqs (§4.1.2): SL at CFL 0.2
    matches the RK2A(0.2) reference closely and loses one to two digits at
    CFL 5 (here at 64^2 against RK2A(0.2) on 128^2)."""
    nref = 128
    m0f = inputs.random_field(nref, seed=1, kmax=6)
    vf = inputs.random_velocity(nref, seed=3, kmax=3, vmax=0.5)
    ref = rk2a.state_solve(m0f, vf, rk2a.cfl_steps(vf, 0.2))
    m0, v = spectral.restrict(m0f), spectral.restrict_vec(vf)
    n = m0.shape[0]
    errs = {}
    for c in (0.2, 1.0, 5.0):
        m1 = Problem(np.zeros((n, n)), m0, rk2a.cfl_steps(v, c), 1e-2).state_solve(v)
        errs[c] = np.linalg.norm(spectral.prolong(m1) - ref) / np.linalg.norm(ref)
    assert errs[0.2] < errs[1.0] < errs[5.0], errs
    assert errs[5.0] > 5 * errs[0.2], errs
