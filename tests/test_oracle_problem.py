"""Pins of the oracle's objective, gradient and Gauss-Newton Hessian (CPU only).

* v = 0 closed forms: m = m_T, lambda = m_R - m_T for all t, so
  g(0) = (m_R - m_T) grad m_T, and H u = beta A u + (u . grad m_T) grad m_T
  exactly (the trapezoid in time is exact on the linear-in-t m~);
* the gradient against central finite differences of the discrete objective:
  below 1e-6 relative at 128^2 for smooth data and a small velocity, and the
  optimise-then-discretise gap falls at least 8x per grid doubling (§3.1
  remark on consistency);
* the incremental state m~_1 against finite differences of the state map;
* GN Hessian: positivity, near-symmetry bounded by the adjoint error, and the
  quadratic-form identity <H u, u> = beta <A u, u> + ||m~_1[u]||^2 up to it;
* 16^2 brute force: the assembled dense Hessian is close to the
  discretise-then-optimise J_F^T J_F + beta A from a finite-difference
  Jacobian of the state map, and PCG reproduces the dense solve;
* operation counts equal Appendix C (SL columns, GN rows).
"""

import numpy as np
import pytest

from oracle import krylov, spectral
from oracle.problem import Problem
from paper_1604_02153_gb300 import inputs


def smooth_problem(n, nt, vmax=0.05, kmax=4, beta=1e-2, kind="spline"):
    m_T = inputs.random_field(n, seed=1, kmax=kmax)
    m_R = inputs.random_field(n, seed=2, kmax=kmax)
    v = inputs.random_velocity(n, seed=3, vmax=vmax)
    return Problem(m_R, m_T, nt, beta, kind=kind), v


@pytest.mark.parametrize("kind", ["spline", "lagrange"])
def test_closed_forms_at_zero_velocity(kind):
    n, nt = 32, 5
    P, _ = smooth_problem(n, nt, kind=kind)
    z = np.zeros((2, n, n))
    J, g = P.objective_gradient(z)
    gm = spectral.grad(P.m_T)
    assert np.max(np.abs(g - (P.m_R - P.m_T) * gm)) < 1e-12
    assert abs(J - 0.5 * P.inner(P.m_R - P.m_T, P.m_R - P.m_T)) < 1e-14
    u = inputs.random_velocity(n, seed=9, vmax=1.0)
    Hu = P.hessian_matvec(u)
    expect = spectral.apply_reg(u, P.beta, "H1") + (u[0] * gm[0] + u[1] * gm[1]) * gm
    assert np.max(np.abs(Hu - expect)) < 1e-12 * np.max(np.abs(expect))
    # m~(t_j) = -t_j u . grad m_T; at t = 1:
    assert np.max(np.abs(P.mt_final + (u[0] * gm[0] + u[1] * gm[1]))) < 1e-12


def test_gradient_against_finite_differences():
    gaps = []
    for n in (32, 64, 128):
        P, v = smooth_problem(n, 16)
        dv = inputs.random_velocity(n, seed=4, vmax=1.0)
        _, g = P.objective_gradient(v)
        d = P.inner(g, dv)
        eps = 1e-4
        fd = (P.objective(v + eps * dv) - P.objective(v - eps * dv)) / (2 * eps)
        gaps.append(abs(fd - d) / abs(d))
    assert gaps[-1] < 1e-6, gaps
    assert gaps[1] < gaps[0] / 8 and gaps[2] < gaps[1] / 8, gaps


def test_gradient_sign_and_scale_not_consistent_with_mistakes():
    """A flipped sign of lambda or a dropped regularisation term would break
    the FD agreement by O(1); check the finite-difference slope directly on a
    problem where both terms matter."""
    n = 64
    P, v = smooth_problem(n, 16, vmax=0.05, beta=0.3)
    dv = inputs.random_velocity(n, seed=5, vmax=1.0)
    _, g = P.objective_gradient(v)
    b_only = g - spectral.apply_reg(v, P.beta, "H1")
    eps = 1e-4
    fd = (P.objective(v + eps * dv) - P.objective(v - eps * dv)) / (2 * eps)
    full = P.inner(g, dv)
    assert abs(fd - full) < 1e-4 * abs(fd)
    assert abs(fd - P.inner(b_only, dv)) > 1e-2 * abs(fd)


def test_incremental_state_linearises_state_map():
    n, nt = 64, 16
    P, v = smooth_problem(n, nt)
    u = inputs.random_velocity(n, seed=6, vmax=1.0)
    P.state_solve(v)
    P.hessian_matvec(u)
    mt = P.mt_final
    eps = 1e-4
    Q = Problem(P.m_R, P.m_T, nt, P.beta)
    fd = (Q.state_solve(v + eps * u) - Q.state_solve(v - eps * u)) / (2 * eps)
    assert np.linalg.norm(mt - fd) / np.linalg.norm(fd) < 1e-4


def test_hessian_symmetry_positivity_and_quadratic_form():
    n, nt = 64, 8
    P, v = smooth_problem(n, nt, vmax=0.2)
    P.state_solve(v)
    u = inputs.random_velocity(n, seed=7, vmax=1.0)
    w = inputs.random_velocity(n, seed=8, vmax=1.0)
    Hu = P.hessian_matvec(u)
    mt_u = P.mt_final
    Hw = P.hessian_matvec(w)
    a, b = P.inner(Hu, w), P.inner(u, Hw)
    assert abs(a - b) / abs(a) < 1e-3
    quad = P.inner(Hu, u)
    assert quad > 0
    reg = P.inner(u, spectral.apply_reg(u, P.beta, "H1"))
    data = P.inner(mt_u, mt_u)
    assert abs(quad - (reg + data)) / quad < 1e-3


def _dense_hessian(P, n):
    cols = []
    for k in range(2 * n * n):
        e = np.zeros(2 * n * n)
        e[k] = 1.0
        cols.append(P.hessian_matvec(e.reshape(2, n, n)).ravel())
    return np.array(cols).T


def test_brute_force_16():
    n, nt = 16, 4
    X1, X2 = inputs.grid_coordinates(n, n)
    m_T = 0.5 + 0.3 * np.sin(X1) * np.cos(X2) + 0.1 * np.cos(2 * X1 - X2)
    m_R = 0.5 + 0.3 * np.cos(X1 + 0.4) * np.sin(X2) + 0.1 * np.sin(X1 + 2 * X2)
    v = 0.05 * np.stack([np.sin(X2), np.cos(X1)])
    P = Problem(m_R, m_T, nt, 1e-1)
    P.state_solve(v)
    H = _dense_hessian(P, n)
    asym = np.linalg.norm(H - H.T) / np.linalg.norm(H)
    assert asym < 1e-2
    ev = np.linalg.eigvalsh(0.5 * (H + H.T))
    assert ev[0] > 0
    # discretise-then-optimise Gauss-Newton Hessian from an FD Jacobian of the
    # discrete state map v -> m_1: J_F^T J_F + beta A
    Q = Problem(m_R, m_T, nt, 1e-1)
    eps = 1e-6
    JF = np.zeros((n * n, 2 * n * n))
    for k in range(2 * n * n):
        e = np.zeros(2 * n * n)
        e[k] = eps
        JF[:, k] = ((Q.state_solve(v + e.reshape(2, n, n)) -
                     Q.state_solve(v - e.reshape(2, n, n))) / (2 * eps)).ravel()
    A = np.zeros((2 * n * n, 2 * n * n))
    for k in range(2 * n * n):
        e = np.zeros(2 * n * n)
        e[k] = 1.0
        A[:, k] = spectral.apply_reg(e.reshape(2, n, n), P.beta, "H1").ravel()
    H_dto = JF.T @ JF + A
    assert np.linalg.norm(H - H_dto) / np.linalg.norm(H_dto) < 5e-2
    # PCG on the matrix-free operator equals the dense solve
    rhs = inputs.random_velocity(n, seed=3, vmax=1.0)
    x_dense = np.linalg.solve(H, rhs.ravel()).reshape(2, n, n)
    x, info = krylov.pcg(P.hessian_matvec, rhs,
                         lambda r: spectral.reg_power(r, P.beta, "H1", -1.0), 1e-12, 300)
    assert np.linalg.norm(x - x_dense) / np.linalg.norm(x_dense) < 1e-6, info


def _golden_counts(path, nt, d=2):
    out = {}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        row, ffts, ips = [s.strip() for s in line.split(";")]
        env = {"d": d, "nt": nt, "__builtins__": {}}
        out[row] = [eval(ffts, env), eval(ips, env)]
    return out


@pytest.mark.parametrize("nt", [1, 4, 7])
def test_operation_counts_match_appendix_c(repo_root, nt):
    table = _golden_counts(f"{repo_root}/tests/golden/complexity_sl.txt", nt)
    assert table == Problem.table_counts(nt)
    n = 16
    P, v = smooth_problem(n, nt)
    P.reset_counts()
    P.state_solve(v)
    assert P.counts["SE"] == table["SE"]
    P.reset_counts()
    P.adjoint_solve()
    assert P.counts["AE"] == table["AE"]
    P.reset_counts()
    P.objective(v)
    assert P.counts["J"] == table["J"]
    P.reset_counts()
    P.gradient()
    assert P.counts["g"] == table["g"]
    P.reset_counts()
    P.hessian_matvec(v)
    assert P.counts["matvec"] == table["matvec"]


def test_gauss_newton_equals_gradient_derivative_at_zero_residual():
    """Where m_1(v) = m_R the adjoint vanishes, every dropped lambda term is
    zero and the GN Hessian is the full Hessian: H u equals the directional
    derivative of the gradient (up to the optimise-then-discretise gap)."""
    n, nt = 64, 8
    m_T = inputs.random_field(n, seed=1, kmax=4)
    v = inputs.random_velocity(n, seed=3, vmax=0.2)
    m_R = Problem(np.zeros((n, n)), m_T, nt, 1e-2).state_solve(v)
    P = Problem(m_R, m_T, nt, 1e-2)
    u = inputs.random_velocity(n, seed=4, vmax=1.0)
    P.state_solve(v)
    Hu = P.hessian_matvec(u)
    eps = 1e-4
    fd = (P.gradient(v + eps * u) - P.gradient(v - eps * u)) / (2 * eps)
    assert np.linalg.norm(fd - Hu) / np.linalg.norm(Hu) < 2e-4


def test_incompressible_gradient_and_hessian_are_leray_projections():
    """Incompressible problem (w = 0, K the Leray projection of §3.1): for a
    divergence-free v and u, g_inc = K g and H_inc u = K H u (K commutes
    with A and fixes v and u); g_inc is divergence free and orthogonal to
    gradient fields, and its slope along a divergence-free direction
    matches central finite differences of J."""
    n, nt = 64, 8
    m_T = inputs.random_field(n, seed=1, kmax=4)
    m_R = inputs.random_field(n, seed=2, kmax=4)
    v = spectral.leray(inputs.random_velocity(n, seed=3, vmax=0.05))
    u = spectral.leray(inputs.random_velocity(n, seed=9, vmax=1.0))
    Pc = Problem(m_R, m_T, nt, 1e-2)
    Pi = Problem(m_R, m_T, nt, 1e-2, incompressible=True)
    Jc, gc = Pc.objective_gradient(v)
    Ji, gi = Pi.objective_gradient(v)
    assert Ji == Jc
    assert np.max(np.abs(gi - spectral.leray(gc))) < 1e-12 * np.max(np.abs(gc))
    assert np.max(np.abs(spectral.div(gi))) < 1e-12 * n * np.max(np.abs(gi))
    w = spectral.grad(inputs.random_field(n, seed=5, kmax=4))
    assert abs(Pi.inner(gi, w)) < 1e-10 * abs(Pc.inner(gc, w))
    Hc = Pc.hessian_matvec(u)
    Hi = Pi.hessian_matvec(u)
    assert np.max(np.abs(Hi - spectral.leray(Hc))) < 1e-12 * np.max(np.abs(Hc))
    assert np.max(np.abs(Hi - Hc)) > 1e-3 * np.max(np.abs(Hc))   # K is not the identity here
    dv = spectral.leray(inputs.random_velocity(n, seed=4, vmax=1.0))
    d = Pi.inner(gi, dv)
    eps = 1e-4
    fd = (Pi.objective(v + eps * dv) - Pi.objective(v - eps * dv)) / (2 * eps)
    assert abs(fd - d) < 1e-4 * abs(d)


def _fn_problem(n, nt, zero_residual=False):
    m_T = inputs.random_field(n, seed=1, kmax=4)
    m_R = inputs.random_field(n, seed=2, kmax=4)
    v = inputs.random_velocity(n, seed=3, vmax=0.3)
    if zero_residual:
        m_R = Problem(np.zeros((n, n)), m_T, nt, 1e-2).state_solve(v)
    return m_R, m_T, v


def test_full_newton_hessian_is_the_derivative_of_the_gradient():
    """eq. hessian-matvec with its lambda terms (full Newton): H u equals the
    central difference of the reduced gradient along u up to the
    optimise-then-discretise gap, which shrinks with the grid; on this
    problem (large residual) the Gauss-Newton matvec misses it by O(1), so
    a dropped or flipped lambda term would fail."""
    errs = []
    for n in (32, 128):
        nt = 8
        m_R, m_T, v = _fn_problem(n, nt)
        u = inputs.random_velocity(n, seed=9, vmax=1.0)
        P = Problem(m_R, m_T, nt, 1e-2, hessian="full")
        P.objective_gradient(v)
        Hfn = P.hessian_matvec(u)
        G = Problem(m_R, m_T, nt, 1e-2)
        G.objective_gradient(v)
        Hgn = G.hessian_matvec(u)
        eps = 1e-4
        _, gp = G.objective_gradient(v + eps * u)
        _, gm = G.objective_gradient(v - eps * u)
        fd = (gp - gm) / (2 * eps)
        e_fn = np.linalg.norm(Hfn - fd) / np.linalg.norm(fd)
        e_gn = np.linalg.norm(Hgn - fd) / np.linalg.norm(fd)
        assert e_fn < 2e-3 and e_gn > 0.5, (n, e_fn, e_gn)
        errs.append(e_fn)
    assert errs[1] < errs[0] / 3, errs


def test_full_newton_equals_gauss_newton_at_zero_residual():
    """m_R = m_1(v): the adjoint lambda vanishes, so do the terms that the
    Gauss-Newton approximation drops (§3.4.1 footnote)."""
    n, nt = 32, 4
    m_R, m_T, v = _fn_problem(n, nt, zero_residual=True)
    u = inputs.random_velocity(n, seed=9, vmax=1.0)
    out = []
    for h in ("gn", "full"):
        P = Problem(m_R, m_T, nt, 1e-2, hessian=h)
        P.objective_gradient(v)
        assert max(np.max(np.abs(l)) for l in P.lam) < 1e-13
        out.append(P.hessian_matvec(u))
    assert np.max(np.abs(out[0] - out[1])) < 1e-12 * np.max(np.abs(out[0]))


def test_full_newton_matvec_is_symmetric_within_the_adjoint_error():
    n, nt = 64, 8
    m_R, m_T, v = _fn_problem(n, nt)
    P = Problem(m_R, m_T, nt, 1e-2, hessian="full")
    P.objective_gradient(v)
    a = inputs.random_velocity(n, seed=11, vmax=1.0)
    b = inputs.random_velocity(n, seed=12, vmax=1.0)
    ab, ba = P.inner(P.hessian_matvec(a), b), P.inner(a, P.hessian_matvec(b))
    assert abs(ab - ba) < 1e-2 * abs(ab)


@pytest.mark.parametrize("nt", [1, 4, 7])
def test_full_newton_counts_against_appendix_c(repo_root, nt):
    """Interpolations per full-Newton matvec equal Appendix C's FN row
    (d + (d+3) nt + 1: the source div(lambda v~) is interpolated at Y_D once
    per step). FFTs: the table's FN row counts 2(d+1) fewer than this
    schedule, which recomputes div v (as the GN row does) and takes the
    source at all nt + 1 time levels that Heun's rule touches."""
    fn = _golden_counts(f"{repo_root}/tests/golden/complexity_sl_fn.txt", nt)
    n, d = 16, 2
    m_R, m_T, v = _fn_problem(n, nt)
    P = Problem(m_R, m_T, nt, 1e-2, hessian="full")
    P.objective_gradient(v)
    P.reset_counts()
    P.hessian_matvec(inputs.random_velocity(n, seed=9, vmax=1.0))
    assert P.counts["matvec"][1] == fn["matvec"][1]
    assert P.counts["matvec"][0] == fn["matvec"][0] + 2 * (d + 1)
