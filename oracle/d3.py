"""The registration problem on 3D periodic grids (FP64 oracle, d = 3).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper's formulation is written for d = 2 or 3 (§2, §3); its experiments
are 2D and it names 3D as the next step. This module restates, for d = 3,
what spectral.py, interp.py, transport.py and problem.py compute for d = 2:

* grid (§3.2): the 3-torus of side 2 pi, n_i nodes per axis, h_i = 2 pi / n_i;
  arrays u[k, j, i] (axis 0 is x_3, axis 2 the fastest, x_1), vector fields
  v[c, k, j, i] with c = 0, 1, 2 for x_1, x_2, x_3;
* pseudospectral gradient and divergence (Nyquist modes zeroed), the
  regularisation operator A with symbol |k|^(2p) (eq. diffopregv) and its
  powers with the zero entry of that symbol replaced by one (eq. reg-precond);
* periodic tricubic interpolation (§3.5): the tensor product of the 1D cubic
  weights over the 4 x 4 x 4 stencil, B-spline weights on the coefficients
  of the spline interpolant (the samples divided by the B-spline sampling
  symbol per axis) or Lagrange weights on the samples;
* RK2 characteristics and the semi-Lagrangian state, adjoint, incremental
  state and (Gauss-Newton) incremental adjoint steps of §3.3.2, the same
  Heun and trapezoidal updates as in 2D with three velocity components;
* J (eq. varopt:objective), the reduced gradient g = beta A v + int lambda
  grad m dt (eq. control-elim) and the Gauss-Newton Hessian matvec
  H v~ = beta A v~ + int lambda~ grad m dt (eq. hessian-matvec, lambda terms
  dropped), compressible (K = I), trapezoidal rule in time;
* the inexact Newton-Krylov solve of §3.4.1 with PCG and the spectral
  preconditioner P_REG = (beta A)^-1 (eq. reg-precond), the steps of
  solver.Solver.solve;
* the deformation map y (u = y - x, the composition of the departure maps)
  and det grad y (§2, §4), as transport.deformation_map and
  spectral.det_grad_map do in 2D;
* the two-level preconditioner P_2L of §3.4.2 (spectral restriction,
  prolongation and high-pass on the 3-torus, the coarse split operator with
  CHEB(k), Lanczos and e_min bounds) in Solver3, the steps of solver.Solver.

Pinned in tests/test_oracle_3d.py: spectral operators exact on trigonometric
polynomials, integral shifts exact, nodal interpolation, reduction to the 2D
oracle on fields constant along x_3 with v_3 = 0 (J, g, H v~ and the whole
solve), the gradient against central finite differences of J, and the
Hessian's symmetry and agreement with finite differences of the gradient at
zero residual; the deformation map by the shear flow (exact u and det = 1),
a constant velocity (u = -c), reduction to the 2D map and determinant, and
m_T o y approaching the state solve's m_1 under grid refinement; the
determinant's expansion against numpy.linalg.det; spectral restriction,
prolongation and high-pass on trigonometric polynomials, R P = I, P R + H =
I and reduction to the 2D operators; the P_2L solve by reduction to the 2D
P_2L solve (same Chebyshev bounds), and Solver3 with P_REG = Problem3.solve.
"""

import numpy as np

from . import interp as interp2
from . import krylov
from .spectral import wavenumbers


# -- spectral ------------------------------------------------------------------
def _k_grids(n1, n2, n3, zero_nyquist):
    k = []
    for n in (n1, n2, n3):
        kk = wavenumbers(n).copy()
        if zero_nyquist:
            kk[n // 2] = 0.0
        k.append(kk)
    K3, K2, K1 = np.meshgrid(k[2], k[1], k[0], indexing="ij")   # shapes (n3, n2, n1)
    return K1, K2, K3


def _shape(u):
    n3, n2, n1 = u.shape[-3:]
    return n1, n2, n3


def fftn(u):
    return np.fft.fftn(u)


def ifftn_real(uh):
    return np.real(np.fft.ifftn(uh))


def grad(u):
    """Spectral gradient (i k_1, i k_2, i k_3) u^, shape (3, n3, n2, n1)."""
    K = _k_grids(*_shape(u), zero_nyquist=True)
    uh = fftn(u)
    return np.stack([ifftn_real(1j * Kc * uh) for Kc in K])


def div(v):
    """Spectral divergence of a 3-component field (Nyquist zeroed)."""
    K = _k_grids(*_shape(v), zero_nyquist=True)
    return ifftn_real(sum(1j * K[c] * fftn(v[c]) for c in range(3)))


def reg_symbol(n1, n2, n3, reg_norm):
    """|k|^(2p) of A = -Lap, Lap^2, -Lap^3 (H1, H2, H3; eq. diffopregv)."""
    p = {"H1": 1, "H2": 2, "H3": 3}[reg_norm]
    K1, K2, K3 = _k_grids(n1, n2, n3, zero_nyquist=False)
    return (K1 * K1 + K2 * K2 + K3 * K3) ** p


def reg_power(v, beta, reg_norm, s):
    """(beta A)^s per component. For s != 1 the zero entry of A's symbol (at
    k = 0) is replaced by one before the power (eq. reg-precond), so the mean
    of each component is scaled by beta^s."""
    gam = reg_symbol(*_shape(v), reg_norm)
    if s != 1:
        gam = np.where(gam == 0, 1, gam)
    g = (beta * gam.astype(np.float64)) ** s
    return np.stack([ifftn_real(g * fftn(v[c])) for c in range(v.shape[0])])


def lowpass_mask3(n1, n2, n3):
    """Modes with |k_i| < n_i / 4 on every axis (§3.4.2 "Filters"): exactly
    those the grid of n_i / 2 points holds without its own Nyquist modes."""
    K1, K2, K3 = _k_grids(n1, n2, n3, zero_nyquist=False)
    return (np.abs(K1) < n1 / 4) & (np.abs(K2) < n2 / 4) & (np.abs(K3) < n3 / 4)


def highpass3(u):
    n1, n2, n3 = _shape(u)
    return ifftn_real(~lowpass_mask3(n1, n2, n3) * fftn(u))


def _kept(n):
    """Fine-grid and coarse-grid FFT indices of the wavenumbers |k| < n / 4."""
    k = np.arange(-(n // 4) + 1, n // 4)
    return k % n, k % (n // 2)


def restrict3(u):
    """Spectral restriction to the grid of n_i / 2 points (§3.4.2): the
    trigonometric interpolant of the modes the cut-off keeps, sampled on
    the coarse grid (numpy's inverse transform is normalised, so the kept
    coefficients scale by N_c / N_f)."""
    n1, n2, n3 = _shape(u)
    (f1, c1), (f2, c2), (f3, c3) = _kept(n1), _kept(n2), _kept(n3)
    U = fftn(u)
    C = np.zeros((n3 // 2, n2 // 2, n1 // 2), dtype=complex)
    C[np.ix_(c3, c2, c1)] = U[np.ix_(f3, f2, f1)] / 8.0
    return ifftn_real(C)


def prolong3(u):
    """Spectral prolongation to the grid of 2 n_i points by zero padding; the
    coarse Nyquist modes are dropped, so restrict3(prolong3(u)) = u on fields
    without them and prolong3(restrict3(u)) is the low-pass part of u."""
    c1n, c2n, c3n = _shape(u)
    (f1, c1), (f2, c2), (f3, c3) = _kept(2 * c1n), _kept(2 * c2n), _kept(2 * c3n)
    C = fftn(u)
    U = np.zeros((2 * c3n, 2 * c2n, 2 * c1n), dtype=complex)
    U[np.ix_(f3, f2, f1)] = C[np.ix_(c3, c2, c1)] * 8.0
    return ifftn_real(U)


def restrict_vec3(v):
    return np.stack([restrict3(v[c]) for c in range(v.shape[0])])


def prolong_vec3(v):
    return np.stack([prolong3(v[c]) for c in range(v.shape[0])])


def highpass_vec3(v):
    return np.stack([highpass3(v[c]) for c in range(v.shape[0])])


def apply_reg(v, beta, reg_norm):
    return reg_power(v, beta, reg_norm, 1)


def spline_prefilter(u):
    """Coefficients of the periodic tricubic B-spline interpolant of u: the
    DFT divided by the sampling symbol (2 + cos(2 pi k / n)) / 3 per axis."""
    n1, n2, n3 = _shape(u)
    s = [(2.0 + np.cos(2.0 * np.pi * wavenumbers(n) / n)) / 3.0 for n in (n1, n2, n3)]
    sym = s[2][:, None, None] * s[1][None, :, None] * s[0][None, None, :]
    return ifftn_real(fftn(u) / sym)


# -- interpolation ---------------------------------------------------------------
def coefficients(u, kind):
    if kind == "spline":
        return spline_prefilter(u)
    if kind == "lagrange":
        return np.array(u, dtype=np.float64, copy=True)
    raise ValueError(kind)


def evaluate(c, p1, p2, p3, kind):
    """The tricubic interpolant with coefficients c at index-space points."""
    n1, n2, n3 = _shape(c)
    wfun = interp2.bspline3_weights if kind == "spline" else interp2.lagrange3_weights
    f = [np.floor(p) for p in (p1, p2, p3)]
    w = [wfun(p - fp) for p, fp in zip((p1, p2, p3), f)]
    i0 = [fp.astype(np.int64) for fp in f]
    out = np.zeros(np.shape(p1), dtype=np.float64)
    for cz in range(4):
        kk = np.mod(i0[2] + (cz - 1), n3)
        for b in range(4):
            jj = np.mod(i0[1] + (b - 1), n2)
            for a in range(4):
                ii = np.mod(i0[0] + (a - 1), n1)
                out += c[kk, jj, ii] * w[0][a] * w[1][b] * w[2][cz]
    return out


def node_coordinates(n1, n2, n3):
    K, J, I = np.meshgrid(np.arange(n3, dtype=np.float64), np.arange(n2, dtype=np.float64),
                          np.arange(n1, dtype=np.float64), indexing="ij")
    return I, J, K


def interp(u, p1, p2, p3, kind):
    return evaluate(coefficients(u, kind), p1, p2, p3, kind)


# -- transport -------------------------------------------------------------------
def characteristic(v, nt, kind, backward):
    """Departure displacement in index units (Heun, §3.3.2), 3 arrays."""
    n1, n2, n3 = _shape(v)
    h = [2.0 * np.pi / n for n in (n1, n2, n3)]
    ht = 1.0 / nt
    s = 1.0 if backward else -1.0
    X = node_coordinates(n1, n2, n3)
    p = [X[c] + s * ht * v[c] / h[c] for c in range(3)]
    vs = [interp(v[c], *p, kind) for c in range(3)]
    return tuple(s * 0.5 * ht * (v[c] + vs[c]) / h[c] for c in range(3))


def at_departure(u, disp, kind):
    X = node_coordinates(*_shape(u))
    return interp(u, X[0] + disp[0], X[1] + disp[1], X[2] + disp[2], kind)


def state_step(m_prev, dX, kind):
    return at_departure(m_prev, dX, kind)


def adjoint_step(lam_next, dY, delta, delta_bar, ht, kind):
    lb = at_departure(lam_next, dY, kind)
    lstar = lb + ht * lb * delta_bar
    return lb + 0.5 * ht * (lb * delta_bar + lstar * delta)


def incstate_step(mt_prev, dX, vt_dep, gm_prev_dep, vt, gm_cur, ht, kind):
    mb = at_departure(mt_prev, dX, kind)
    f_dep = -sum(vt_dep[c] * gm_prev_dep[c] for c in range(3))
    f_arr = -sum(vt[c] * gm_cur[c] for c in range(3))
    return mb + 0.5 * ht * (f_dep + f_arr)


def trapezoid_weights(nt):
    w = np.ones(nt + 1)
    w[0] = 0.5
    w[-1] = 0.5
    return w


# -- deformation map -------------------------------------------------------------
def deformation_map(v, nt, kind="spline"):
    """Displacement u = y - x (physical units, (3, n3, n2, n1)) of the
    deformation map y with m_1 = m_T o y (§2, computed from v after the
    solve): y(x) is where the characteristic through x at t = 1 was at t = 0,
    the composition of the nt departure maps X_D. From u_0 = 0, each step
    interpolates the previous displacement at the departure points and adds
    the step's own: u_j = u_{j-1}(X_D) + (X_D - x)."""
    n1, n2, n3 = _shape(v)
    h = [2.0 * np.pi / n for n in (n1, n2, n3)]
    dX = characteristic(v, nt, kind, backward=False)
    u = np.zeros((3,) + v.shape[1:])
    for _ in range(nt):
        u = np.stack([at_departure(u[c], dX, kind) + h[c] * dX[c] for c in range(3)])
    return u


def det_grad_map(u):
    """det grad y for y = x + u (u periodic, (3, n3, n2, n1)): the determinant
    of J = I + grad u, J[a][b] = delta_ab + d_b u_a, with spectral derivatives,
    expanded along the first row (the quantity bounded in the beta selection
    of §4)."""
    d = [grad(u[a]) for a in range(3)]    # d[a][b] = d_b u_a
    J = [[(1.0 if a == b else 0.0) + d[a][b] for b in range(3)] for a in range(3)]
    return (J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1])
            - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0])
            + J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]))


# -- the problem -----------------------------------------------------------------
class Problem3:
    """One compressible registration problem on an (n3, n2, n1) grid."""

    def __init__(self, m_R, m_T, nt, beta, reg_norm="H1", kind="spline"):
        self.m_R = np.asarray(m_R, dtype=np.float64)
        self.m_T = np.asarray(m_T, dtype=np.float64)
        self.n1, self.n2, self.n3 = _shape(self.m_R)
        self.nt = int(nt)
        self.ht = 1.0 / self.nt
        self.beta = float(beta)
        self.reg_norm = reg_norm
        self.kind = kind
        self.hh = np.prod([2.0 * np.pi / n for n in (self.n1, self.n2, self.n3)])
        self.w = trapezoid_weights(self.nt)

    def inner(self, a, b):
        """<a, b>_h = h_1 h_2 h_3 sum(a b) (midpoint rule)."""
        return self.hh * float(np.sum(a * b))

    def state_solve(self, v):
        self.v = np.array(v, dtype=np.float64, copy=True)
        self.dX = characteristic(self.v, self.nt, self.kind, backward=False)
        m = [self.m_T]
        for _ in range(self.nt):
            m.append(state_step(m[-1], self.dX, self.kind))
        self.m = m
        self.gm = [grad(mj) for mj in m]
        self.dY = characteristic(self.v, self.nt, self.kind, backward=True)
        self.delta = div(self.v)
        self.delta_bar = at_departure(self.delta, self.dY, self.kind)
        return m[-1]

    def objective(self, v):
        self.state_solve(v)
        r = self.m[-1] - self.m_R
        return 0.5 * self.inner(r, r) + 0.5 * self.inner(self.v, apply_reg(self.v, self.beta,
                                                                          self.reg_norm))

    def gradient(self):
        """g = beta A v + int_0^1 lambda grad m dt at the last state solve."""
        nt, ht = self.nt, self.ht
        lam = [None] * (nt + 1)
        lam[nt] = self.m_R - self.m[nt]
        for j in range(nt - 1, -1, -1):
            lam[j] = adjoint_step(lam[j + 1], self.dY, self.delta, self.delta_bar, ht, self.kind)
        b = np.zeros((3,) + self.m_R.shape)
        for j in range(nt + 1):
            b += ht * self.w[j] * lam[j] * self.gm[j]
        self.lam = lam
        return apply_reg(self.v, self.beta, self.reg_norm) + b

    def objective_gradient(self, v):
        J = self.objective(v)
        return J, self.gradient()

    def data_matvec(self, vt):
        """The Gauss-Newton data term Q v~ = H v~ - beta A v~."""
        vt = np.asarray(vt, dtype=np.float64)
        return self.hessian_matvec(vt) - apply_reg(vt, self.beta, self.reg_norm)

    def hessian_matvec(self, vt):
        """Gauss-Newton H v~ at the velocity of the last state solve."""
        nt, ht = self.nt, self.ht
        vt = np.asarray(vt, dtype=np.float64)
        vt_dep = [at_departure(vt[c], self.dX, self.kind) for c in range(3)]
        mt = np.zeros(self.m_R.shape)
        for j in range(1, nt + 1):
            G = [at_departure(self.gm[j - 1][c], self.dX, self.kind) for c in range(3)]
            mt = incstate_step(mt, self.dX, vt_dep, G, vt, self.gm[j], ht, self.kind)
        lt = -mt
        b = ht * self.w[nt] * lt * self.gm[nt]
        for j in range(nt - 1, -1, -1):
            lt = adjoint_step(lt, self.dY, self.delta, self.delta_bar, ht, self.kind)
            b = b + ht * self.w[j] * lt * self.gm[j]
        return apply_reg(vt, self.beta, self.reg_norm) + b

    def solve(self, v0, gtol, max_newton=50, max_pcg=100, max_backtracks=10, c1=1e-4, gabs=1e-5):
        """Inexact Gauss-Newton-Krylov with Armijo backtracking (§3.4.1):
        stop when ||g||_inf <= gtol ||g(0)||_inf; forcing term
        min(0.5, ||g||_2 / ||g(0)||_2); PCG with P_REG. Returns (v, info)."""
        z = np.zeros((3,) + self.m_R.shape)
        _, g_ref = self.objective_gradient(z)
        gref_inf = float(np.max(np.abs(g_ref)))
        gref_2 = float(np.sqrt(np.sum(g_ref * g_ref)))
        v = np.array(v0, dtype=np.float64, copy=True)
        J, g = self.objective_gradient(v)
        info = {"J0": J, "newton_iters": 0, "pcg_iters": 0, "matvecs": 0,
                "line_search_fail": False}
        rel = 1.0
        for k in range(max_newton + 1):
            ginf = float(np.max(np.abs(g)))
            rel = ginf / gref_inf
            if rel <= gtol or ginf <= gabs or k == max_newton:
                break
            eta = min(0.5, float(np.sqrt(np.sum(g * g))) / gref_2)
            vt, kinfo = krylov.pcg(self.hessian_matvec, -g,
                                   lambda r: reg_power(r, self.beta, self.reg_norm, -1), eta, max_pcg)
            info["pcg_iters"] += kinfo["iters"]
            info["matvecs"] += kinfo["matvecs"]
            slope = self.inner(g, vt)
            alpha, accepted = 1.0, False
            for _ in range(max_backtracks + 1):
                Jt = self.objective(v + alpha * vt)
                if Jt <= J + c1 * alpha * slope:
                    accepted = True
                    break
                alpha *= 0.5
            if not accepted:
                info["line_search_fail"] = True
                self.state_solve(v)
                break
            v = v + alpha * vt
            J = Jt
            g = self.gradient()
            info["newton_iters"] += 1
        info["J"] = J
        info["gnorm_rel"] = rel
        return v, info


# -- the two-level preconditioner -------------------------------------------------
class Solver3:
    """The inexact Newton-Krylov solve of Problem3.solve with P_REG or the
    two-level preconditioner P_2L of §3.4.2, read as solver.Solver reads it
    in 2D:
        r'  = (beta A)^-1/2 r,  r_c = R r',
        s_c = (I + (beta A_c)^-1/2 Q_c (beta A_c)^-1/2)^-1 r_c  by CHEB(k)
              or PCG(eps * eta_k) (pc_solver "cheb" or "pcg"),
        z   = (beta A)^-1/2 (P s_c + H r')
    with R, P the spectral restriction and prolongation, H the high-pass
    filter and Q_c the Gauss-Newton data term of the coarse problem (m_R,
    m_T and v restricted, the same nt). CHEB bounds: e_max from Lanczos on the
    coarse split operator at v = 0 (lanczos_steps steps from lanczos_v0,
    times emax_safety), e_min = min over the coarse modes of 1 + 1/(beta
    gamma_k)."""

    def __init__(self, problem, precond="2L", cheb_iters=10, gabs=1e-5, max_newton=50,
                 max_pcg=100, lanczos_steps=30, emax_safety=1.05, lanczos_v0=None, c1=1e-4,
                 max_backtracks=10, pc_solver="cheb", pc_eps=0.1):
        self.p = problem
        self.precond = precond
        self.pc_solver = pc_solver
        self.pc_eps = pc_eps
        self.eta = 0.5
        self.cheb_iters = cheb_iters
        self.gabs = gabs
        self.max_newton = max_newton
        self.max_pcg = max_pcg
        self.lanczos_steps = lanczos_steps
        self.emax_safety = emax_safety
        self.lanczos_v0 = lanczos_v0
        self.c1 = c1
        self.max_backtracks = max_backtracks
        self.eig = None
        self.coarse_matvecs = 0
        self.coarse = None
        if precond == "2L":
            p = problem
            self.coarse = Problem3(restrict3(p.m_R), restrict3(p.m_T), p.nt, p.beta, p.reg_norm,
                                   p.kind)

    def coarse_split_op(self, s):
        c = self.coarse
        u = reg_power(s, c.beta, c.reg_norm, -0.5)
        q = c.data_matvec(u)
        self.coarse_matvecs += 1
        return s + reg_power(q, c.beta, c.reg_norm, -0.5)

    def estimate_eigenvalues(self):
        c = self.coarse
        shape = (3,) + c.m_R.shape
        c.state_solve(np.zeros(shape))
        if self.lanczos_v0 is None:
            v0 = np.random.default_rng(1234).uniform(-1.0, 1.0, shape)
        else:
            v0 = np.asarray(self.lanczos_v0, dtype=np.float64).reshape(shape)
        _, rmax, _ = krylov.lanczos_extremal(self.coarse_split_op, v0, self.lanczos_steps)
        gam = reg_symbol(c.n1, c.n2, c.n3, c.reg_norm).astype(np.float64)
        gam = np.where(gam == 0, 1.0, gam)
        emin = float(np.min(1.0 + 1.0 / (c.beta * gam)))
        self.eig = {"emin": emin, "emax": rmax * self.emax_safety}
        return self.eig

    def apply_precond(self, r):
        p = self.p
        if self.precond == "REG":
            return reg_power(r, p.beta, p.reg_norm, -1)
        r1 = reg_power(r, p.beta, p.reg_norm, -0.5)
        if self.pc_solver == "cheb":
            sc, _ = krylov.chebyshev(self.coarse_split_op, restrict_vec3(r1), self.eig["emin"],
                                     self.eig["emax"], self.cheb_iters)
        else:
            sc, _ = krylov.pcg(self.coarse_split_op, restrict_vec3(r1), lambda x: x,
                               self.pc_eps * self.eta, self.max_pcg)
        return reg_power(prolong_vec3(sc) + highpass_vec3(r1), p.beta, p.reg_norm, -0.5)

    def solve(self, v0, gtol):
        """Problem3.solve's loop with this preconditioner; returns (v, info)."""
        p = self.p
        z = np.zeros((3,) + p.m_R.shape)
        _, g_ref = p.objective_gradient(z)
        gref_inf = float(np.max(np.abs(g_ref)))
        gref_2 = float(np.sqrt(np.sum(g_ref * g_ref)))
        if self.precond == "2L" and self.pc_solver == "cheb" and self.eig is None:
            self.estimate_eigenvalues()
        v = np.array(v0, dtype=np.float64, copy=True)
        J, g = p.objective_gradient(v)
        info = {"J0": J, "newton_iters": 0, "pcg_iters": 0, "matvecs": 0,
                "line_search_fail": False}
        rel = 1.0
        for k in range(self.max_newton + 1):
            ginf = float(np.max(np.abs(g)))
            rel = ginf / gref_inf
            if rel <= gtol or ginf <= self.gabs or k == self.max_newton:
                break
            eta = min(0.5, float(np.sqrt(np.sum(g * g))) / gref_2)
            self.eta = eta
            if self.coarse is not None:
                self.coarse.state_solve(restrict_vec3(v))
            vt, kinfo = krylov.pcg(p.hessian_matvec, -g, self.apply_precond, eta, self.max_pcg)
            info["pcg_iters"] += kinfo["iters"]
            info["matvecs"] += kinfo["matvecs"]
            slope = p.inner(g, vt)
            alpha, accepted = 1.0, False
            for _ in range(self.max_backtracks + 1):
                Jt = p.objective(v + alpha * vt)
                if Jt <= J + self.c1 * alpha * slope:
                    accepted = True
                    break
                alpha *= 0.5
            if not accepted:
                info["line_search_fail"] = True
                p.state_solve(v)
                break
            v = v + alpha * vt
            J = Jt
            g = p.gradient()
            info["newton_iters"] += 1
        info["J"] = J
        info["gnorm_rel"] = rel
        info["coarse_matvecs"] = self.coarse_matvecs
        return v, info
