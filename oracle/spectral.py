"""Pseudospectral Fourier operators on the periodic grid (FP64 oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Grid (§3.2): the periodic domain is the 2-torus of side 2*pi, discretised by a
regular grid with n_i nodes per axis, h_i = 2*pi/n_i, node (i, j) at
(i*h_1, j*h_2). The paper writes the domain as (-pi, pi)^d; on the torus this
is the same set shifted by pi, which changes no operator below.

Arrays are indexed ``u[j, i]``: axis 0 is x_2, axis 1 (fastest) is x_1.
Vector fields are ``v[c, j, i]`` with c = 0 for x_1 and c = 1 for x_2.

Wavenumbers are the integers k in FFT order {0, .., n/2-1, -n/2, .., -1}.
Readings where the paper is silent:
* odd derivatives (grad, div) zero the Nyquist mode k = -n/2;
* even operators (the Laplacian powers of eq. diffopregv) keep |k|^2 there;
* the regularisation operator has a null space at k = 0; following
  eq. reg-precond the zero spectral weight is replaced by one wherever the
  operator is inverted or raised to a negative/fractional power.
"""

import numpy as np


def wavenumbers(n):
    """Integer wavenumbers of an n-point periodic grid, in FFT order."""
    return np.fft.fftfreq(n, d=1.0 / n)


def _k_grids(n1, n2, zero_nyquist):
    k1 = wavenumbers(n1).copy()
    k2 = wavenumbers(n2).copy()
    if zero_nyquist:
        k1[n1 // 2] = 0.0
        k2[n2 // 2] = 0.0
    K2, K1 = np.meshgrid(k2, k1, indexing="ij")  # shapes (n2, n1)
    return K1, K2


def fft2(u):
    return np.fft.fft2(u)


def ifft2_real(uh):
    return np.real(np.fft.ifft2(uh))


def grad(u):
    """Spectral gradient: d/dx_i <-> i*k_i (§3.2 pseudospectral basis).

    Returns an array of shape (2, n2, n1). Nyquist modes are zeroed.
    Pinned: exact on trigonometric polynomials (tests/test_oracle_spectral.py).
    """
    n2, n1 = u.shape
    K1, K2 = _k_grids(n1, n2, zero_nyquist=True)
    uh = fft2(u)
    return np.stack([ifft2_real(1j * K1 * uh), ifft2_real(1j * K2 * uh)])


def div(v):
    """Spectral divergence d v_1/dx_1 + d v_2/dx_2 (Nyquist zeroed)."""
    n2, n1 = v.shape[1:]
    K1, K2 = _k_grids(n1, n2, zero_nyquist=True)
    return ifft2_real(1j * K1 * fft2(v[0]) + 1j * K2 * fft2(v[1]))


def leray(b):
    """Leray projection K[b] = -grad Lap^-1 div b + b (§3.1, the K of
    eq. control-elim when the divergence w is set to zero): the part of a
    periodic vector field that the spectral divergence maps to zero.

    Written out as its definition: phi solves Lap phi = div b with the
    Laplacian taken as div(grad .) of the two operators above (so that div K b
    is exactly zero for the discrete div; the modes where div(grad .) vanishes,
    k = 0 and the Nyquist lines, keep phi = 0), then K b = b - grad phi.
    """
    n2, n1 = b.shape[1:]
    K1, K2 = _k_grids(n1, n2, zero_nyquist=True)
    lap = -(K1 * K1 + K2 * K2)                      # symbol of div(grad .)
    dh = fft2(div(b))
    phih = np.where(lap != 0.0, dh / np.where(lap != 0.0, lap, 1.0), 0.0)
    return b - grad(ifft2_real(phih))


def det_grad_map(u):
    """det grad y for y = x + u (u periodic, (2, n2, n1)): (1 + d1 u1)(1 + d2 u2)
    - d2 u1 d1 u2 with spectral derivatives (the determinant of the deformation
    gradient of §2 and the bound of §4's beta selection)."""
    g1, g2 = grad(u[0]), grad(u[1])
    return (1.0 + g1[0]) * (1.0 + g2[1]) - g1[1] * g2[0]


def reg_symbol(n1, n2, reg_norm):
    """Spectral weights gamma(k) = |k|^(2p) of the regularisation operator A.

    eq. diffopregv: A = -Laplacian (H1, p = 1), Laplacian^2 (H2, p = 2),
    -Laplacian^3 (H3, p = 3). With the Fourier symbol of the Laplacian being
    -|k|^2, each of these has the nonnegative symbol |k|^(2p).
    """
    p = {"H1": 1, "H2": 2, "H3": 3}[reg_norm]
    K1, K2 = _k_grids(n1, n2, zero_nyquist=False)
    return (K1 * K1 + K2 * K2) ** p


def apply_reg(v, beta, reg_norm):
    """beta * A[v] componentwise (the beta_v A term of eq. control-elim)."""
    n2, n1 = v.shape[1:]
    g = beta * reg_symbol(n1, n2, reg_norm)
    return np.stack([ifft2_real(g * fft2(v[c])) for c in range(v.shape[0])])


def reg_w_term(v, beta_w):
    """-beta_w grad (I - Lap) div v: the near-incompressible regularisation of
    §2 with the mass source eliminated.

    eq. varopt:regw puts the H1 norm ||w||^2 = int grad w . grad w + w^2 on
    the mass source w, and eq. icconstraint ties it to the velocity,
    w = div v. The control equations of the optimality system (Appendix A,
    eq. control-v and eq. control-w) read
        beta_v A v + grad p + b = 0,    beta_w B w + p = 0,
    with B = I - Lap the first variation of that norm. Eliminating
    p = -beta_w B w and w = div v leaves
        beta_v A v - beta_w grad B div v + b = 0,
    i.e. this term joins beta_v A v in the reduced gradient and in the
    Hessian; it is the first variation of (beta_w / 2) ||div v||^2_{H1}.
    Written out step by step with the operators above: w = div v (Nyquist
    zeroed), B w = w - Lap w with the Laplacian's symbol -|k|^2, then
    -beta_w grad(B w).
    """
    n2, n1 = v.shape[1:]
    w = div(v)
    lap_w = ifft2_real(-reg_symbol(n1, n2, "H1") * fft2(w))
    return -beta_w * grad(w - lap_w)


def apply_regop(v, beta, reg_norm, beta_w=0.0):
    """The regularisation operator of the gradient and the Hessian:
    beta_v A v, plus -beta_w grad (I - Lap) div v for the near-incompressible
    problem (beta_w > 0)."""
    out = apply_reg(v, beta, reg_norm)
    if beta_w > 0.0:
        out = out + reg_w_term(v, beta_w)
    return out


def regop_power(v, beta, reg_norm, beta_w, s):
    """R^s for R = beta_v A - beta_w grad (I - Lap) div (the operator of
    apply_regop), with the zero weight of A at k = 0 replaced by 1 as in
    reg_power (s = 1 is R itself).

    R acts on each wavenumber k as the symmetric 2 x 2 matrix
        beta_v |k|^(2p) I + beta_w (1 + |k|^2) kd kd^T,
    kd the derivative wavenumbers of grad and div (Nyquist zeroed); its power
    is taken by the eigendecomposition of that matrix (numpy.linalg.eigh),
    mode by mode. With beta_w = 0 this is reg_power.
    """
    n2, n1 = v.shape[1:]
    gam = reg_symbol(n1, n2, reg_norm).astype(np.float64)
    if s != 1.0:
        gam[0, 0] = 1.0
    K1, K2 = _k_grids(n1, n2, zero_nyquist=True)
    ksq = reg_symbol(n1, n2, "H1").astype(np.float64)
    c = beta_w * (1.0 + ksq)
    M = np.empty((n2, n1, 2, 2))
    M[..., 0, 0] = beta * gam + c * K1 * K1
    M[..., 0, 1] = c * K1 * K2
    M[..., 1, 0] = c * K2 * K1
    M[..., 1, 1] = beta * gam + c * K2 * K2
    lam, Q = np.linalg.eigh(M)
    Ms = np.einsum("...ij,...j,...kj->...ik", Q, lam ** s, Q)
    vh = np.stack([fft2(v[0]), fft2(v[1])], axis=-1)
    oh = np.einsum("...ij,...j->...i", Ms, vh)
    return np.stack([ifft2_real(oh[..., 0]), ifft2_real(oh[..., 1])])


def near_inc_K(b, beta, reg_norm, beta_w):
    """The operator K of eq. control-elim for the near-incompressible problem.

    With w = div v and p = -beta_w (I - Lap) w eliminated (see reg_w_term)
    the control equation reads M v + b = 0 with
    M = beta A - beta_w grad (I - Lap) div (apply_regop). Writing it in the
    paper's form beta A v + K[b] = 0 (eq. control-elim) gives
    K = beta A M^-1 on every mode where M is invertible; on the mean (k = 0),
    where both regularisation terms vanish, K is the identity (as the Leray
    projection is there). Written out as that definition: M^-1 b by
    regop_power(s = -1), then beta A of it, plus the mean of b.
    """
    n2, n1 = b.shape[1:]
    x = regop_power(b, beta, reg_norm, beta_w, -1.0)
    out = apply_reg(x, beta, reg_norm)
    return out + b.mean(axis=(1, 2), keepdims=True)


def reg_power(v, beta, reg_norm, s):
    """(beta * A)^s componentwise, with the zero weight at k = 0 replaced by 1.

    eq. reg-precond: P_REG = beta*A = beta W Gamma W^-1 with the zero entries
    of Gamma replaced by one so that it can be inverted. s = -1 is the
    P_REG^-1 of eq. reg-precond-hessian; s = -1/2, +1/2 are the split
    preconditioner factors of §3.4.2 ("Spectral Preconditioning").
    """
    n2, n1 = v.shape[1:]
    gam = reg_symbol(n1, n2, reg_norm).astype(np.float64)
    gam[0, 0] = 1.0
    mult = (beta * gam) ** s
    return np.stack([ifft2_real(mult * fft2(v[c])) for c in range(v.shape[0])])


def lowpass_mask(n1, n2):
    """Ideal cut-off filter at half the fine frequency (§3.4.2 "Filters").

    Keeps the modes with |k_1| < n_1/4 and |k_2| < n_2/4, i.e. exactly the
    modes that the coarse grid of n/2 points represents without its own
    Nyquist mode.
    """
    K1, K2 = _k_grids(n1, n2, zero_nyquist=False)
    return (np.abs(K1) < n1 / 4) & (np.abs(K2) < n2 / 4)


def lowpass(u):
    n2, n1 = u.shape
    return ifft2_real(lowpass_mask(n1, n2) * fft2(u))


def highpass(u):
    n2, n1 = u.shape
    return ifft2_real((~lowpass_mask(n1, n2)) * fft2(u))


def restrict(u):
    """Spectral restriction from an (n2, n1) grid to (n2/2, n1/2) (§3.4.2).

    The coarse field is the trigonometric interpolant of the modes kept by
    ``lowpass``: same function, coarser samples. With numpy's normalised
    inverse transform this scales the kept coefficients by N_c / N_f.
    """
    n2, n1 = u.shape
    c2, c1 = n2 // 2, n1 // 2
    uh = fft2(u)
    ch = np.zeros((c2, c1), dtype=complex)
    kf1, kf2 = wavenumbers(n1), wavenumbers(n2)
    kc1, kc2 = wavenumbers(c1), wavenumbers(c2)
    for jc in range(c2):
        if not abs(kc2[jc]) < n2 / 4:
            continue
        jf = int(kc2[jc]) % n2
        assert kf2[jf] == kc2[jc]
        for ic in range(c1):
            if not abs(kc1[ic]) < n1 / 4:
                continue
            i_f = int(kc1[ic]) % n1
            assert kf1[i_f] == kc1[ic]
            ch[jc, ic] = uh[jf, i_f]
    return ifft2_real(ch * (c1 * c2) / (n1 * n2))


def prolong(u):
    """Spectral prolongation from (n2, n1) to (2*n2, 2*n1) by zero padding.

    The coarse Nyquist modes are dropped (they have no unique fine-grid
    counterpart), so that restrict(prolong(u)) = u on fields without them and
    prolong(restrict(u)) = lowpass(u).
    """
    c2, c1 = u.shape
    n2, n1 = 2 * c2, 2 * c1
    ch = fft2(u)
    fh = np.zeros((n2, n1), dtype=complex)
    kc1, kc2 = wavenumbers(c1), wavenumbers(c2)
    for jc in range(c2):
        if not abs(kc2[jc]) < n2 / 4:
            continue
        jf = int(kc2[jc]) % n2
        for ic in range(c1):
            if not abs(kc1[ic]) < n1 / 4:
                continue
            fh[jf, int(kc1[ic]) % n1] = ch[jc, ic]
    return ifft2_real(fh * (n1 * n2) / (c1 * c2))


def restrict_vec(v):
    return np.stack([restrict(v[c]) for c in range(v.shape[0])])


def prolong_vec(v):
    return np.stack([prolong(v[c]) for c in range(v.shape[0])])


def spline_prefilter_symbol(n1, n2):
    """Fourier symbol of sampling a periodic cubic B-spline series.

    The centred cubic B-spline takes the values 2/3 at 0 and 1/6 at +-1, so
    sampling sum_m c[m] beta3(x - m) at the nodes multiplies the DFT of c by
    (2 + cos(2 pi k / n)) / 3 per axis. Dividing by it yields the C2 cubic
    spline coefficients that interpolate the samples (§3.5 "Interpolation").
    """
    k1 = wavenumbers(n1)
    k2 = wavenumbers(n2)
    s1 = (2.0 + np.cos(2.0 * np.pi * k1 / n1)) / 3.0
    s2 = (2.0 + np.cos(2.0 * np.pi * k2 / n2)) / 3.0
    return s2[:, None] * s1[None, :]


def spline_prefilter(u):
    """Periodic cubic B-spline coefficients c of the samples u (exact inverse
    of the B-spline sampling operator on the torus)."""
    n2, n1 = u.shape
    return ifft2_real(fft2(u) / spline_prefilter_symbol(n1, n2))
