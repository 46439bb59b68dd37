"""Objective, reduced gradient and Gauss-Newton Hessian matvec (FP64 oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Problem (§2, eq. varopt):
    minimise J[v] = 1/2 ||m_1 - m_R||^2 + beta/2 <v, A v>
                    [+ beta_w/2 ||div v||^2_H1]
    subject to d_t m + grad m . v = 0, m(0) = m_T, periodic;
compressible (w and its constraint omitted: K = I, the default),
incompressible (div v = 0, w = 0: K = the Leray projection of §3.1,
spectral.leray) or near-incompressible (beta_w > 0: the mass source
w = div v of eq. icconstraint carries the H1 norm of eq. varopt:regw, so J
adds beta_w/2 ||div v||^2_H1; with w and p eliminated from the control
equations eq. control-v and eq. control-w, K = beta A M^-1 with
M = beta A - beta_w grad (I - Lap) div, spectral.near_inc_K).

Discrete inner product (§3.2, midpoint rule): <a, b>_h = h_1 h_2 sum a b.

Optimise-then-discretise (§3.1):
* reduced gradient, eq. control-elim:
      g = beta A v + K[int_0^1 lambda grad m dt],
  lambda from the adjoint eq. adj-pde-elim with final value
  lambda_1 = -(m_1 - m_R) (eq. adj-pde-fc-elim);
* Gauss-Newton Hessian matvec, eq. hessian-matvec with every term in lambda
  dropped (§3.4.1 footnote, §3.5 "Hessian"):
      H v~ = beta A v~ + K[int_0^1 lambda~ grad m dt],
  m~ from eq. inc-state-pde-elim (m~(0) = 0), lambda~ from
  eq. inc-adj-pde-elim without the div(lambda v~) term, lambda~_1 = -m~_1;
* full-Newton Hessian matvec (hessian="full"), eq. hessian-matvec as
  written: H v~ = beta A v~ + K[int_0^1 lambda~ grad m + lambda grad m~ dt],
  lambda~ from eq. inc-adj-slm with the div(lambda v~) source, lambda the
  adjoint of the last gradient evaluation (its history is kept).
Time integrals use the trapezoidal rule on the nt + 1 time levels (the paper
only states a midpoint rule for integral operators, which fixes the spatial
sum; no half-step values exist in time).

Operation counts follow Appendix C (table "computational complexity", SL
columns): ``counts[row] = [FFTs, IPs]`` for rows "SE", "AE", "incSE",
"incAE", "J", "g", "matvec". The schedule is the paper's: no gradient field
is stored across solves, so grad m_j is recomputed by FFT (1 forward + d
inverse FFTs) wherever it is used; grad m_0 = grad m_T is computed once per
image pair. An FFT is one 2D transform of one scalar field; an IP is one
scalar interpolation including its spline prefilter. With K the Leray
projection, each application of K adds 2d FFTs (d forward, d inverse: one
Fourier multiplier on a d-vector field), beyond the table.
"""

import numpy as np

from . import spectral, transport

D = 2  # spatial dimension


class Problem:
    """One registration problem on an (n2, n1) grid with nt time steps."""

    def __init__(self, m_R, m_T, nt, beta, reg_norm="H1", kind="spline", incompressible=False,
                 hessian="gn", beta_w=0.0):
        self.m_R = np.asarray(m_R, dtype=np.float64)
        self.m_T = np.asarray(m_T, dtype=np.float64)
        self.n2, self.n1 = self.m_R.shape
        self.nt = int(nt)
        self.ht = 1.0 / self.nt
        self.beta = float(beta)
        self.reg_norm = reg_norm
        self.kind = kind
        self.incompressible = bool(incompressible)
        self.beta_w = float(beta_w)
        assert self.beta_w >= 0.0 and not (self.incompressible and self.beta_w > 0.0)
        assert hessian in ("gn", "full")
        self.full_newton = hessian == "full"
        self.lam = None
        self.h1 = 2.0 * np.pi / self.n1
        self.h2 = 2.0 * np.pi / self.n2
        self.w = transport.trapezoid_weights(self.nt)
        self.grad_mT = spectral.grad(self.m_T)   # grad m_0, once per image pair
        self.counts = {}
        self.v = None

    # -- bookkeeping --------------------------------------------------------
    def K(self, b, row):
        """The operator K of eq. control-elim: identity (compressible), the
        Leray projection (incompressible, w = 0) or beta A M^-1
        (near-incompressible)."""
        if self.beta_w > 0.0:
            self._count(row, ffts=2 * D)
            return spectral.near_inc_K(b, self.beta, self.reg_norm, self.beta_w)
        if not self.incompressible:
            return b
        self._count(row, ffts=2 * D)
        return spectral.leray(b)

    def regop(self, v):
        """R v for the regularisation term 1/2 <v, R v> of J: beta A v, with
        -beta_w grad (I - Lap) div v added for the near-incompressible
        problem (spectral.reg_w_term)."""
        return spectral.apply_regop(v, self.beta, self.reg_norm, self.beta_w)

    def reg(self, v):
        """beta A v, the first term of the reduced gradient and the Hessian."""
        return spectral.apply_reg(v, self.beta, self.reg_norm)

    def _count(self, row, ffts=0, ips=0):
        c = self.counts.setdefault(row, [0, 0])
        c[0] += ffts
        c[1] += ips

    def reset_counts(self):
        self.counts = {}

    def inner(self, a, b):
        """<a, b>_h = h_1 h_2 sum(a b) (midpoint rule, §3.2)."""
        return self.h1 * self.h2 * float(np.sum(a * b))

    def _grad_m(self, j, row):
        """grad m_j; recomputed by FFT for j >= 1 (1 + d FFTs, Appendix C)."""
        if j == 0:
            return self.grad_mT
        self._count(row, ffts=1 + D)
        return spectral.grad(self.m[j])

    # -- state (SE) and objective (J) -----------------------------------------
    def state_solve(self, v, row="SE"):
        """Forward characteristic (d IPs) and nt state steps (nt IPs)."""
        self.v = np.array(v, dtype=np.float64, copy=True)
        self.dX = transport.characteristic(self.v, self.nt, self.kind, backward=False)
        self._count(row, ips=D)
        m = [self.m_T]
        for _ in range(self.nt):
            m.append(transport.state_step(m[-1], self.dX, self.kind))
            self._count(row, ips=1)
        self.m = m
        self.dY = None
        self.lam = None          # the adjoint belongs to the previous velocity
        return m[-1]

    def objective(self, v):
        """J[v] (eq. varopt:objective); counted as row "J" = SE + 2d FFTs."""
        self.state_solve(v, row="J")
        Av = self.regop(self.v)
        self._count("J", ffts=2 * D)
        r = self.m[-1] - self.m_R
        return 0.5 * self.inner(r, r) + 0.5 * self.inner(self.v, Av)

    # -- adjoint (AE) and gradient (g) ---------------------------------------
    def _div_v(self, row):
        self._count(row, ffts=D + 1)
        return spectral.div(self.v)

    def adjoint_solve(self, row="AE"):
        """Backward characteristic (d IPs), div v (d+1 FFTs), div v at Y_D
        (1 IP), nt adjoint steps (nt IPs). Needs the state at self.v."""
        nt, ht = self.nt, self.ht
        self.dY = transport.characteristic(self.v, nt, self.kind, backward=True)
        self._count(row, ips=D)
        delta = self._div_v(row)
        delta_bar = transport.at_departure(delta, self.dY, self.kind)
        self._count(row, ips=1)
        lam = [None] * (nt + 1)
        lam[nt] = self.m_R - self.m[nt]          # eq. adj-pde-fc-elim
        for j in range(nt - 1, -1, -1):
            lam[j] = transport.adjoint_step(lam[j + 1], self.dY, delta, delta_bar,
                                            ht, self.kind)
            self._count(row, ips=1)
        self.lam = lam
        return lam

    def gradient(self, v=None):
        """Reduced gradient g (eq. control-elim), row "g".

        Runs the state solve first if v is given (counted under "J", as the
        paper charges the forward solve to the objective).
        """
        if v is not None:
            self.state_solve(v, row="J")
        lam = self.adjoint_solve(row="g")
        b = np.zeros((2, self.n2, self.n1))
        for j in range(self.nt + 1):
            gm = self._grad_m(j, "g")
            b += self.ht * self.w[j] * lam[j] * gm
        self._count("g", ffts=2 * D)
        self.b = b
        return self.reg(self.v) + self.K(b, "g")

    def gradient_l2(self, v=None):
        """The L2 gradient of J, R v + int_0^1 lambda grad m dt (R of regop):
        the derivative that finite differences of J check. For the
        compressible and near-incompressible problems the reduced gradient
        of eq. control-elim is K of it: K M = beta A and K b = K[b]."""
        self.gradient(v)
        return self.regop(self.v) + self.b

    def objective_gradient(self, v):
        J = self.objective(v)
        return J, self.gradient()

    # -- Gauss-Newton Hessian matvec -----------------------------------------
    def ensure_adjoint_characteristic(self):
        if self.dY is None:
            self.dY = transport.characteristic(self.v, self.nt, self.kind, backward=True)

    def hessian_matvec(self, vt, row="matvec"):
        """GN Hessian matvec H(v) v~ at the velocity of the last state solve.

        incSE: v~(X_D) once (d IPs); per step grad m_j (d+1 FFTs) and
        interpolation of m~_{j-1} and grad m_{j-1} (1 + d IPs).
        incAE (GN): div v (d+1 FFTs), div v at Y_D (1 IP), nt steps (nt IPs);
        the time integral of lambda~ grad m recomputes grad m_j (d+1 FFTs
        per level j >= 1); beta A v~ (2d FFTs).
        """
        nt, ht, kind = self.nt, self.ht, self.kind
        vt = np.asarray(vt, dtype=np.float64)
        if self.full_newton:
            return self._hessian_matvec_full(vt, row)
        self.ensure_adjoint_characteristic()
        vt_dep = np.stack([transport.at_departure(vt[c], self.dX, kind) for c in range(2)])
        self._count(row, ips=D)
        mt = np.zeros((self.n2, self.n1))
        gm_prev = self.grad_mT
        for j in range(1, nt + 1):
            gm_cur = self._grad_m(j, row)
            gm_prev_dep = np.stack([transport.at_departure(gm_prev[c], self.dX, kind)
                                    for c in range(2)])
            mt = transport.incstate_step(mt, self.dX, vt_dep, gm_prev_dep, vt, gm_cur,
                                         ht, kind)
            self._count(row, ips=1 + D)
            gm_prev = gm_cur
        self.mt_final = mt
        delta = self._div_v(row)
        delta_bar = transport.at_departure(delta, self.dY, kind)
        self._count(row, ips=1)
        lt = -mt                                   # eq. inc-adj-fc-elim
        bt = self.ht * self.w[nt] * lt * self._grad_m(nt, row)
        for j in range(nt - 1, -1, -1):
            lt = transport.adjoint_step(lt, self.dY, delta, delta_bar, ht, kind)
            self._count(row, ips=1)
            bt = bt + self.ht * self.w[j] * lt * self._grad_m(j, row)
        self._count(row, ffts=2 * D)
        return self.reg(vt) + self.K(bt, row)

    def _hessian_matvec_full(self, vt, row):
        """Full-Newton matvec (eq. hessian-matvec with its lambda terms).

        Needs the adjoint history lambda_0..lambda_nt of a gradient evaluation
        at the current velocity. incSE as in the GN matvec, keeping m~_j;
        div(lambda_j v~) at the nt + 1 time levels (d + 1 FFTs each); incAE
        with that source (2 IPs per step: lambda~_{j+1} and the source at
        Y_D, plus div v at Y_D once); the time integral of
        lambda~ grad m + lambda grad m~ recomputes grad m_j and grad m~_j
        (d + 1 FFTs per level j >= 1; m~_0 = 0).
        """
        assert self.lam is not None, "full-Newton matvec needs the gradient at this velocity"
        nt, ht, kind = self.nt, self.ht, self.kind
        lam = self.lam
        self.ensure_adjoint_characteristic()
        vt_dep = np.stack([transport.at_departure(vt[c], self.dX, kind) for c in range(2)])
        self._count(row, ips=D)
        mt = [np.zeros((self.n2, self.n1))]
        gm_prev = self.grad_mT
        for j in range(1, nt + 1):
            gm_cur = self._grad_m(j, row)
            gm_prev_dep = np.stack([transport.at_departure(gm_prev[c], self.dX, kind)
                                    for c in range(2)])
            mt.append(transport.incstate_step(mt[-1], self.dX, vt_dep, gm_prev_dep, vt, gm_cur,
                                              ht, kind))
            self._count(row, ips=1 + D)
            gm_prev = gm_cur
        self.mt_final = mt[-1]
        src = []
        for j in range(nt + 1):
            src.append(spectral.div(lam[j] * vt))
            self._count(row, ffts=D + 1)
        delta = self._div_v(row)
        delta_bar = transport.at_departure(delta, self.dY, kind)
        self._count(row, ips=1)

        def grad_mt(j):
            if j == 0:
                return np.zeros((2, self.n2, self.n1))
            self._count(row, ffts=1 + D)
            return spectral.grad(mt[j])

        lt = -mt[nt]                                   # eq. inc-adj-fc-elim
        bt = ht * self.w[nt] * (lt * self._grad_m(nt, row) + lam[nt] * grad_mt(nt))
        for j in range(nt - 1, -1, -1):
            lt = transport.incadjoint_step_full(lt, self.dY, delta, delta_bar, src[j + 1], src[j],
                                                ht, kind)
            self._count(row, ips=2)
            bt = bt + ht * self.w[j] * (lt * self._grad_m(j, row) + lam[j] * grad_mt(j))
        self._count(row, ffts=2 * D)
        return self.reg(vt) + self.K(bt, row)

    def data_matvec(self, vt):
        """Data term Q v~ = H v~ - beta A v~ (eq. reduced-space-kkt-system)."""
        return self.hessian_matvec(vt) - self.reg(np.asarray(vt, dtype=np.float64))

    # -- Appendix C reference counts -----------------------------------------
    @staticmethod
    def table_counts(nt, d=D):
        """FFT / IP counts of the SL columns of Appendix C for one call."""
        return {
            "SE": [0, d + nt],
            "AE": [d + 1, d + nt + 1],
            "incSE": [(d + 1) * nt, d + (d + 1) * nt],
            "incAE": [d + 1, nt + 1],
            "J": [2 * d, d + nt],
            "g": [2 * d + (d + 1) * (nt + 1), d + nt + 1],
            "matvec": [2 * d + (d + 1) * (2 * nt + 1), d + (d + 2) * nt + 1],
        }
