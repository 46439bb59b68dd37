"""Preconditioners and the inexact Gauss-Newton-Krylov loop (FP64 oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

* P_REG (eq. reg-precond): P_REG^-1 r = (beta A)^-1 r, zero weight -> 1.
* P_2L (§3.4.2 "Nested Preconditioner"), read as follows (the paper gives
  prose only):
      r'  = (beta A)^-1/2 r                          split preconditioning
      r_c = R r'                                     cut-off + restriction
      s_c = (I + (beta A_c)^-1/2 Q_c (beta A_c)^-1/2)^-1 r_c   coarse solve,
            CHEB(k) or PCG(eps * eta)
      z   = (beta A)^-1/2 (P s_c + H r')             prolong, high band kept
  with R, P the spectral restriction/prolongation, H the ideal high-pass
  filter and Q_c the Gauss-Newton data term on a coarse problem built by
  spectrally restricting m_R, m_T and v (same nt).
* CHEB bounds (§3.4.2 "Eigenvalue Estimates"): e_max from Lanczos on the
  coarse split operator at v = 0 (30 steps from a given start vector), times
  a safety factor of 1.05 (the paper gives none); e_min from
  min(1 + 1/(beta gamma_k)) over the coarse grid; a change of beta rescales
  (e - 1) by beta_old / beta_new.
* Incompressible problems (K the Leray projection): the initial guess and
  the Lanczos start vector are projected onto divergence-free fields, so
  that every iterate stays in the space the constraint div v = 0 defines
  (K commutes with A and with the filters, restriction and prolongation).
* Outer loop (§3.4.1, §3.5): stop when ||g_k||_inf / ||g_ref||_inf <= gtol or
  ||g_k||_inf <= gabs; g_ref = g(v = 0) (the paper's g_0 for a zero initial
  guess; fixed at v = 0 so that warm starts and beta stages share one
  target). Forcing term eta_k = min(0.5, ||g_k||_2 / ||g_ref||_2) (the
  quadratic choice of Nocedal & Wright, made relative). Armijo backtracking
  with c1 = 1e-4, halving, at most 10 halvings (the paper names the rule but
  not its constants).
"""

import numpy as np

from . import krylov, spectral
from .problem import Problem


class Solver:
    def __init__(self, problem, precond="2L", pc_solver="cheb", cheb_iters=10,
                 pc_eps=0.1, gabs=1e-5, max_newton=50, max_pcg=100,
                 lanczos_steps=30, emax_safety=1.05, lanczos_v0=None,
                 c1=1e-4, max_backtracks=10, coarse_nt=None, coarse_kind=None):
        self.p = problem
        self.precond = precond
        self.pc_solver = pc_solver
        self.cheb_iters = cheb_iters
        self.pc_eps = pc_eps
        self.gabs = gabs
        self.max_newton = max_newton
        self.max_pcg = max_pcg
        self.lanczos_steps = lanczos_steps
        self.emax_safety = emax_safety
        self.lanczos_v0 = lanczos_v0
        self.c1 = c1
        self.max_backtracks = max_backtracks
        self.coarse = None
        self.eig = None
        self.coarse_matvecs = 0
        self.eta = 0.5
        if precond == "2L":
            p = problem
            # coarse_nt: time steps of the coarse problem (default: the same
            # nt; §3.4.2 expects the preconditioner's PDE solves to need
            # little accuracy)
            # coarse_kind: its interpolation model (default: the problem's)
            self.coarse = Problem(spectral.restrict(p.m_R), spectral.restrict(p.m_T),
                                  coarse_nt or p.nt, p.beta, p.reg_norm, coarse_kind or p.kind,
                                  p.incompressible, beta_w=p.beta_w)

    # -- preconditioners -----------------------------------------------------
    @staticmethod
    def reg_pow(p, x, s):
        """(beta A)^s (eq. reg-precond)."""
        return spectral.reg_power(x, p.beta, p.reg_norm, s)

    def precond_reg(self, r):
        return self.reg_pow(self.p, r, -1.0)

    def coarse_split_op(self, s):
        """(I + (beta A_c)^-1/2 Q_c (beta A_c)^-1/2) s on the coarse grid."""
        c = self.coarse
        u = self.reg_pow(c, s, -0.5)
        q = c.data_matvec(u)
        self.coarse_matvecs += 1
        return s + self.reg_pow(c, q, -0.5)

    def estimate_eigenvalues(self):
        """e_min, e_max of the coarse split operator at v = 0."""
        c = self.coarse
        c.state_solve(np.zeros((2, c.n2, c.n1)))
        if self.lanczos_v0 is None:
            v0 = np.random.default_rng(1234).uniform(-1.0, 1.0, (2, c.n2, c.n1))
        else:
            v0 = np.asarray(self.lanczos_v0, dtype=np.float64).reshape(2, c.n2, c.n1)
        if c.incompressible:
            v0 = spectral.leray(v0)
        _, rmax, _ = krylov.lanczos_extremal(self.coarse_split_op, v0, self.lanczos_steps)
        gam = spectral.reg_symbol(c.n1, c.n2, c.reg_norm).astype(np.float64)
        gam[0, 0] = 1.0
        emin = float(np.min(1.0 + 1.0 / (c.beta * gam)))
        self.eig = {"emin": emin, "emax": rmax * self.emax_safety, "beta": c.beta}
        return self.eig

    def set_beta(self, beta):
        """Continuation in beta: eigenvalue estimates rescaled, not recomputed."""
        old = self.p.beta
        self.p.beta = float(beta)
        if self.coarse is not None:
            self.coarse.beta = float(beta)
        if self.eig is not None:
            s = old / float(beta)
            self.eig = {"emin": 1.0 + (self.eig["emin"] - 1.0) * s,
                        "emax": 1.0 + (self.eig["emax"] - 1.0) * s,
                        "beta": float(beta)}

    def precond_2l(self, r):
        p = self.p
        r1 = self.reg_pow(p, r, -0.5)
        rc = spectral.restrict_vec(r1)
        rh = np.stack([spectral.highpass(r1[c]) for c in range(2)])
        if self.pc_solver == "cheb":
            sc, _ = krylov.chebyshev(self.coarse_split_op, rc, self.eig["emin"],
                                     self.eig["emax"], self.cheb_iters)
        else:
            sc, _ = krylov.pcg(self.coarse_split_op, rc, lambda x: x,
                               self.pc_eps * self.eta, self.max_pcg)
        z1 = spectral.prolong_vec(sc) + rh
        return self.reg_pow(p, z1, -0.5)

    def apply_precond(self, r):
        if self.precond == "REG":
            return self.precond_reg(r)
        return self.precond_2l(r)

    def set_velocity_coarse(self, v):
        if self.coarse is not None:
            self.coarse.state_solve(spectral.restrict_vec(v))

    # -- Newton-Krylov -------------------------------------------------------
    def kkt_solve(self, rhs, rtol, maxit=None):
        """PCG on H(v) x = rhs at the current velocity (state already solved)."""
        if self.precond == "2L":
            if self.eig is None:
                self.estimate_eigenvalues()
            self.set_velocity_coarse(self.p.v)
        return krylov.pcg(self.p.hessian_matvec, rhs, self.apply_precond, rtol,
                          maxit or self.max_pcg)

    def solve(self, v0, gtol, g_ref=None):
        """Inexact GN-Krylov with Armijo line search; returns (v, info)."""
        p = self.p
        n = (2, p.n2, p.n1)
        if g_ref is None:
            g_ref = p.gradient(np.zeros(n))
        gref_inf = float(np.max(np.abs(g_ref)))
        gref_2 = float(np.sqrt(np.sum(g_ref * g_ref)))
        if self.precond == "2L" and self.eig is None:
            self.estimate_eigenvalues()
        v = np.array(v0, dtype=np.float64, copy=True)
        if p.incompressible:
            v = spectral.leray(v)
        J, g = p.objective_gradient(v)
        info = {"J0": J, "newton_iters": 0, "pcg_iters": 0, "matvecs": 0,
                "line_search_fail": False, "log": []}
        for k in range(self.max_newton + 1):
            ginf = float(np.max(np.abs(g)))
            rel = ginf / gref_inf
            info["log"].append({"J": J, "gnorm_rel": rel})
            if rel <= gtol or ginf <= self.gabs or k == self.max_newton:
                break
            self.eta = min(0.5, float(np.sqrt(np.sum(g * g))) / gref_2)
            vt, kinfo = self.kkt_solve(-g, self.eta)
            info["pcg_iters"] += kinfo["iters"]
            info["matvecs"] += kinfo["matvecs"]
            slope = p.inner(g, vt)
            alpha = 1.0
            accepted = False
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
