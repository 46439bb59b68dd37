"""RK2 characteristics and semi-Lagrangian transport solves (FP64 oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

§3.3.2 rewrites the state, adjoint, incremental state and incremental adjoint
equations (eq. hyperbolic-pdes-slm) in the common form D_t u = f(u, v), with
D_t the Lagrangian derivative along the characteristics of eq. characteristic.
Each time step has two parts: trace the characteristic back over one step to
its departure point, then integrate f along it with explicit RK2 (Heun),
interpolating the transported quantity at the departure point
(eq. transport-along-characteristic).

Departure points (§3.3.2 "Tracing the Characteristic", Heun's method, velocity
stationary so they are computed once per velocity and reused by every step):
* forward-in-time equations (state, incremental state), d X / dt = v:
      X* = x - h_t v(x),    X_D = x - (h_t/2) (v(x) + v(X*));
* backward-in-time equations (adjoint, incremental adjoint) run in reversed
  time tau = 1 - t, where the characteristic speed is -v:
      Y* = x + h_t v(x),    Y_D = x + (h_t/2) (v(x) + v(Y*)).
v(X*) and v(Y*) are interpolated (d interpolations per characteristic,
Appendix C). Departure points are returned as displacements in index units,
(X_D - x) / h, so that the node index and the offset stay separate.

Source terms along the characteristic (Heun; the paper's "explicit RK2" of
§3.3.2 "Transport"): with u_bar = u_prev(departure point),
      u_new = u_bar + (h_t/2) (f(u_bar at departure) + f(u* at x)),
      u*    = u_bar + h_t f(u_bar at departure).
"""

import numpy as np

from . import interp


def characteristic(v, nt, kind, backward):
    """Departure-point displacement (index units) of one time step.

    v: (2, n2, n1) stationary velocity. backward=False gives X_D (state and
    incremental state); backward=True gives Y_D (adjoint and incremental
    adjoint). Returns (d1, d2), each (n2, n1).
    """
    n2, n1 = v.shape[1:]
    h1 = 2.0 * np.pi / n1
    h2 = 2.0 * np.pi / n2
    ht = 1.0 / nt
    s = 1.0 if backward else -1.0
    I, J = interp.node_coordinates(n1, n2)
    p1 = I + s * ht * v[0] / h1
    p2 = J + s * ht * v[1] / h2
    vs1 = interp.interp(v[0], p1, p2, kind)
    vs2 = interp.interp(v[1], p1, p2, kind)
    d1 = s * 0.5 * ht * (v[0] + vs1) / h1
    d2 = s * 0.5 * ht * (v[1] + vs2) / h2
    return d1, d2


def at_departure(u, disp, kind):
    """u interpolated at the departure points x + disp (index units)."""
    n2, n1 = u.shape
    I, J = interp.node_coordinates(n1, n2)
    return interp.interp(u, I + disp[0], J + disp[1], kind)


def state_step(m_prev, dX, kind):
    """State equation eq. state-slm: D_t m = 0, so m_j = m_{j-1}(X_D)."""
    return at_departure(m_prev, dX, kind)


def adjoint_step(lam_next, dY, delta, delta_bar, ht, kind):
    """Adjoint equation eq. adj-slm in reversed time: D_tau lam = lam div v.

    lam_next = lambda_{j+1}; delta = div v at the nodes; delta_bar = div v
    at the departure points Y_D (interpolated once per velocity).
    Returns lambda_j (Heun along the characteristic).
    """
    lb = at_departure(lam_next, dY, kind)
    lstar = lb + ht * lb * delta_bar
    return lb + 0.5 * ht * (lb * delta_bar + lstar * delta)


def incadjoint_step_full(lt_next, dY, delta, delta_bar, src_next, src, ht, kind):
    """Full-Newton incremental adjoint eq. inc-adj-slm in reversed time:
    D_tau lam~ = lam~ div v + div(lambda v~).

    src_next = div(lambda_{j+1} v~), src = div(lambda_j v~) at the nodes;
    src_next is interpolated at Y_D like lam~_{j+1}. Heun with the source at
    the departure point (level j+1) and at the node (level j); dropping both
    sources gives adjoint_step (the Gauss-Newton incremental adjoint).
    """
    lb = at_departure(lt_next, dY, kind)
    sb = at_departure(src_next, dY, kind)
    f_dep = lb * delta_bar + sb
    lstar = lb + ht * f_dep
    return lb + 0.5 * ht * (f_dep + lstar * delta + src)


def incstate_step(mt_prev, dX, vt_dep, gm_prev_dep, vt, gm_cur, ht, kind):
    """Incremental state eq. inc-state-slm: D_t m~ = -v~ . grad m.

    vt_dep = v~(X_D) (2 fields, interpolated once per matvec);
    gm_prev_dep = grad m_{j-1}(X_D) (2 fields); gm_cur = grad m_j at the
    nodes. The source does not depend on m~, so Heun's predictor drops out
    and the step is the trapezoidal rule along the characteristic.
    """
    mb = at_departure(mt_prev, dX, kind)
    f_dep = -(vt_dep[0] * gm_prev_dep[0] + vt_dep[1] * gm_prev_dep[1])
    f_arr = -(vt[0] * gm_cur[0] + vt[1] * gm_cur[1])
    return mb + 0.5 * ht * (f_dep + f_arr)


def trapezoid_weights(nt):
    """Weights w_j of the trapezoidal rule in time on t_j = j/nt, j = 0..nt
    (the time integral in eq. control-elim and eq. hessian-matvec)."""
    w = np.ones(nt + 1)
    w[0] = 0.5
    w[-1] = 0.5
    return w


def deformation_map(v, nt, kind):
    """Displacement u = y - x (physical units, (2, n2, n1)) of the
    deformation map y with m_1 = m_T o y (§2): y(x) is where the
    characteristic through x at t = 1 was at t = 0, the composition of the
    nt departure maps X_D. With u_0 = 0, each step interpolates the previous
    displacement at the departure points and adds the step's own:
        u_j = u_{j-1}(X_D) + (X_D - x),
    so that interpolating m_T at x + u is the SL state solve's m_1 up to the
    interpolation error of composing instead of chaining."""
    n2, n1 = v.shape[1:]
    h = (2.0 * np.pi / n1, 2.0 * np.pi / n2)
    dX = characteristic(v, nt, kind, backward=False)
    u = np.zeros((2, n2, n1))
    for _ in range(nt):
        u = np.stack([at_departure(u[c], dX, kind) + h[c] * dX[c] for c in range(2)])
    return u
