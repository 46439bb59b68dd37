"""Krylov building blocks: PCG, Chebyshev semi-iteration, Lanczos (FP64 oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Vectors are numpy arrays of any shape; inner products are plain Euclidean
sums (the grid weight h_1 h_2 is a constant factor that no Krylov method
below depends on).
"""

import numpy as np


def dot(a, b):
    return float(np.sum(a * b))


def pcg(apply_A, b, apply_Minv, rtol, maxit):
    """Preconditioned conjugate gradients (Hestenes-Stiefel), zero initial guess.

    §3.4.1: the Newton system is solved by PCG; the solve stops when negative
    curvature occurs (p^T A p <= 0) and keeps the current iterate (at the
    first iteration that iterate is the preconditioned right-hand side, the
    usual steepest-descent fallback). Stops when ||r||_2 <= rtol ||b||_2.

    Returns (x, info) with info = {"iters", "matvecs", "relres", "negcurv"}.
    """
    x = np.zeros_like(b)
    r = np.array(b, copy=True)
    bnorm = np.sqrt(dot(b, b))
    info = {"iters": 0, "matvecs": 0, "relres": 1.0, "negcurv": False}
    if bnorm == 0.0:
        info["relres"] = 0.0
        return x, info
    z = apply_Minv(r)
    p = np.array(z, copy=True)
    rz = dot(r, z)
    for it in range(maxit):
        q = apply_A(p)
        info["matvecs"] += 1
        pq = dot(p, q)
        if pq <= 0.0:
            info["negcurv"] = True
            if it == 0:
                x = np.array(z, copy=True)
            break
        alpha = rz / pq
        x = x + alpha * p
        r = r - alpha * q
        info["iters"] = it + 1
        rel = np.sqrt(dot(r, r)) / bnorm
        info["relres"] = rel
        if rel <= rtol:
            break
        z = apply_Minv(r)
        rz_new = dot(r, z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, info


def chebyshev(apply_A, b, emin, emax, k):
    """Chebyshev semi-iteration with k steps, zero initial guess (§3.4.2 CHEB(k)).

    Three-term Chebyshev acceleration for an SPD operator with spectrum in
    [emin, emax] (Axelsson, Iterative Solution Methods, Ch. 5; Saad,
    Iterative Methods for Sparse Linear Systems, Sec. 12.3). The k-th iterate
    x_k = (I - P_k(A)) A^-1 b with P_k the scaled Chebyshev polynomial of
    degree k, so ||x_k - A^-1 b||_A <= 2 rho^k ||A^-1 b||_A with
    rho = (sqrt(kappa) - 1) / (sqrt(kappa) + 1), kappa = emax / emin.
    k updates need k - 1 operator applications (the residual after the last
    update is never read). Returns (x, matvecs).
    """
    theta = 0.5 * (emax + emin)
    delta = 0.5 * (emax - emin)
    sigma = theta / delta
    rho = 1.0 / sigma
    x = np.zeros_like(b)
    r = np.array(b, copy=True)
    d = r / theta
    matvecs = 0
    for it in range(k):
        x = x + d
        if it == k - 1:
            break
        r = r - apply_A(d)
        matvecs += 1
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = (rho_new * rho) * d + (2.0 * rho_new / delta) * r
        rho = rho_new
    return x, matvecs


def lanczos_extremal(apply_A, v0, steps):
    """Extremal Ritz values of a symmetric operator after ``steps`` Lanczos steps.

    §3.4.2 ("Eigenvalue Estimates for the CHEB Method") estimates e_max with
    Lanczos (about 30 matvecs, §4.2.1). This is the plain Lanczos process
    with full reorthogonalisation, started from v0; it stops early on an
    invariant subspace. Returns (ritz_min, ritz_max, matvecs).
    """
    q = v0 / np.sqrt(dot(v0, v0))
    Q = [q]
    alphas, betas = [], []
    beta = 0.0
    q_prev = np.zeros_like(q)
    for _ in range(steps):
        w = apply_A(q)
        alpha = dot(q, w)
        w = w - alpha * q - beta * q_prev
        for qq in Q:                        # full reorthogonalisation
            w = w - dot(qq, w) * qq
        alphas.append(alpha)
        beta = np.sqrt(dot(w, w))
        if beta <= 1e-14 * abs(alpha):
            break
        betas.append(beta)
        q_prev = q
        q = w / beta
        Q.append(q)
    m = len(alphas)
    T = np.diag(alphas) + np.diag(betas[: m - 1], 1) + np.diag(betas[: m - 1], -1)
    ev = np.linalg.eigvalsh(T)
    return float(ev[0]), float(ev[-1]), m
