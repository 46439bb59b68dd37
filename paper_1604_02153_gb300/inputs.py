"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module only synthesises images and velocity fields; it holds none of the
registration method's arithmetic (no transport, no gradient, no Hessian).
Every generator is deterministic given its arguments (numpy PCG64 via
``default_rng(seed)``). Fields are float64 arrays in the library layout:
scalar ``u[j, i]`` (x_1 fastest), vector ``v[c, j, i]``, on the periodic grid
x = (i h_1, j h_2), h_k = 2 pi / n_k.

Workloads (the paper's own images and analytic test problems are not
available; these stand in for them at the paper's scale: smooth images with
intensities in [0, 1] and velocities of magnitude up to 0.5):
* ``sinusoid_pair``     - the analytic template and ground-truth velocity of
                          the 64^2 plain-method problem;
* ``random_field``      - band-limited Gaussian random field, Fourier modes
                          0 < |k| <= kmax with amplitude |k|^-2 and uniform
                          random phases, rescaled to [0, 1];
* ``random_velocity``   - two such fields with modes 0 < |k| <= 4, scaled so
                          that max_x |v(x)|_2 equals a given value;
* ``ellipse_phantoms``  - a pair of piecewise-smooth phantoms made of seeded
                          random ellipses, blurred and normalised to [0, 1];
* ``he_normal``         - seeded He-normal initial weights (zero biases) for
                          a stack of 3x3 convolutions given their channel
                          counts, in the flat parameter layout of the
                          warm-start network.
"""

import numpy as np


def grid_coordinates(n1, n2):
    """Physical node coordinates X1, X2 of shape (n2, n1)."""
    x1 = 2.0 * np.pi * np.arange(n1) / n1
    x2 = 2.0 * np.pi * np.arange(n2) / n2
    X2, X1 = np.meshgrid(x2, x1, indexing="ij")
    return X1, X2


def sinusoid_pair(n1, n2=None):
    """m_T = (sin^2 x1 + sin^2 x2)/2 and v* = (0.5 sin x1 cos x2, 0.5 cos x1 sin x2)."""
    n2 = n1 if n2 is None else n2
    X1, X2 = grid_coordinates(n1, n2)
    m_T = 0.5 * (np.sin(X1) ** 2 + np.sin(X2) ** 2)
    v = np.stack([0.5 * np.sin(X1) * np.cos(X2), 0.5 * np.cos(X1) * np.sin(X2)])
    return m_T, v


def vortex_pair(n1, n2=None):
    """m_T as in sinusoid_pair and the divergence-free v* = (-0.5 sin x1 cos x2,
    0.5 cos x1 sin x2) (stream function 0.5 sin x1 sin x2), for the
    incompressible problem."""
    n2 = n1 if n2 is None else n2
    X1, X2 = grid_coordinates(n1, n2)
    m_T = 0.5 * (np.sin(X1) ** 2 + np.sin(X2) ** 2)
    v = np.stack([-0.5 * np.sin(X1) * np.cos(X2), 0.5 * np.cos(X1) * np.sin(X2)])
    return m_T, v


def _half_plane_modes(kmax):
    modes = []
    for k2 in range(0, kmax + 1):
        for k1 in range(-kmax, kmax + 1):
            if k2 == 0 and k1 <= 0:
                continue
            r2 = k1 * k1 + k2 * k2
            if 0 < r2 <= kmax * kmax:
                modes.append((k1, k2))
    return modes


def _cosine_series(n1, n2, kmax, rng):
    """sum over a half plane of |k|^-2 cos(k . x + phi_k), phi_k ~ U[0, 2 pi).

    Evaluated on the grid as the real part of an inverse DFT of the sparse
    coefficient array (identical to summing the cosines node by node, modes
    with |k_i| >= n_i/2 aliasing the same way).
    """
    C = np.zeros((n2, n1), dtype=complex)
    for (k1, k2) in _half_plane_modes(kmax):
        phi = rng.uniform(0.0, 2.0 * np.pi)
        amp = 1.0 / float(k1 * k1 + k2 * k2)
        C[k2 % n2, k1 % n1] += amp * np.exp(1j * phi)
    return np.real(np.fft.ifft2(C)) * (n1 * n2)


def rescale01(u):
    lo, hi = float(np.min(u)), float(np.max(u))
    return (u - lo) / (hi - lo)


def random_field(n1, n2=None, seed=0, kmax=16):
    """Band-limited Gaussian random field rescaled to [0, 1]."""
    n2 = n1 if n2 is None else n2
    rng = np.random.default_rng(seed)
    return rescale01(_cosine_series(n1, n2, kmax, rng))


def random_velocity(n1, n2=None, seed=0, kmax=4, vmax=0.2):
    """Smooth random velocity, modes 0 < |k| <= kmax, max |v(x)|_2 = vmax."""
    n2 = n1 if n2 is None else n2
    rng = np.random.default_rng(seed)
    v = np.stack([_cosine_series(n1, n2, kmax, rng), _cosine_series(n1, n2, kmax, rng)])
    vn = float(np.max(np.sqrt(v[0] ** 2 + v[1] ** 2)))
    return v * (vmax / vn)


def _cosine_series3(n1, n2, n3, kmax, rng):
    """The 3D analogue of _cosine_series: |k|^-2 cos(k . x + phi_k) summed
    over the modes 0 < |k| <= kmax of a half space (k3 > 0, or k3 = 0 and
    the 2D half plane), shape (n3, n2, n1)."""
    C = np.zeros((n3, n2, n1), dtype=complex)
    for k3 in range(0, kmax + 1):
        for k2 in range(-kmax, kmax + 1):
            for k1 in range(-kmax, kmax + 1):
                if k3 == 0 and (k2 < 0 or (k2 == 0 and k1 <= 0)):
                    continue
                r2 = k1 * k1 + k2 * k2 + k3 * k3
                if 0 < r2 <= kmax * kmax:
                    phi = rng.uniform(0.0, 2.0 * np.pi)
                    C[k3 % n3, k2 % n2, k1 % n1] += np.exp(1j * phi) / float(r2)
    return np.real(np.fft.ifftn(C)) * (n1 * n2 * n3)


def random_field3(n1, n2, n3, seed=0, kmax=4):
    """Band-limited random field on an n1 x n2 x n3 grid rescaled to [0, 1]."""
    rng = np.random.default_rng(seed)
    return rescale01(_cosine_series3(n1, n2, n3, kmax, rng))


def random_velocity3(n1, n2, n3, seed=0, kmax=3, vmax=0.2):
    """Smooth random 3-component velocity, max |v(x)|_2 = vmax, shape
    (3, n3, n2, n1)."""
    rng = np.random.default_rng(seed)
    v = np.stack([_cosine_series3(n1, n2, n3, kmax, rng) for _ in range(3)])
    vn = float(np.max(np.sqrt(np.sum(v * v, axis=0))))
    return v * (vmax / vn)


def gaussian_blur(u, sigma_px):
    """Periodic Gaussian blur with standard deviation sigma_px grid points."""
    n2, n1 = u.shape
    k1 = np.fft.fftfreq(n1, d=1.0 / n1)
    k2 = np.fft.fftfreq(n2, d=1.0 / n2)
    s1 = sigma_px * 2.0 * np.pi / n1
    s2 = sigma_px * 2.0 * np.pi / n2
    mult = np.exp(-0.5 * ((s2 * k2[:, None]) ** 2 + (s1 * k1[None, :]) ** 2))
    return np.real(np.fft.ifft2(np.fft.fft2(u) * mult))


def _paint(n1, n2, ellipses):
    X1, X2 = grid_coordinates(n1, n2)
    img = np.zeros((n2, n1))
    two_pi = 2.0 * np.pi
    for (c1, c2, a, b, th, inten) in ellipses:
        d1 = np.mod(X1 - c1 + np.pi, two_pi) - np.pi     # nearest periodic image
        d2 = np.mod(X2 - c2 + np.pi, two_pi) - np.pi
        ct, st = np.cos(th), np.sin(th)
        r1 = ct * d1 + st * d2
        r2 = -st * d1 + ct * d2
        inside = (r1 / a) ** 2 + (r2 / b) ** 2 <= 1.0
        img[inside] = inten
    return img


def ellipse_phantoms(n1, n2=None, seed=100, count=12, sigma_px=2.0):
    """Template/reference phantom pair of ``count`` random ellipses each.

    Centres U[0, 2 pi)^2, semi-axes U[0.05, 0.25] * 2 pi, angle U[0, pi),
    intensity U[0, 1], painted in order (later ellipses overwrite earlier
    ones). The second image moves each centre by U[-0.1, 0.1] times the
    semi-axes and scales each semi-axis by U[0.9, 1.1]. Both are blurred with
    a periodic Gaussian of sigma_px grid points and rescaled to [0, 1].
    Returns (m_R, m_T).
    """
    n2 = n1 if n2 is None else n2
    rng = np.random.default_rng(seed)
    first, second = [], []
    for _ in range(count):
        c1, c2 = rng.uniform(0.0, 2.0 * np.pi, size=2)
        a, b = rng.uniform(0.05, 0.25, size=2) * 2.0 * np.pi
        th = rng.uniform(0.0, np.pi)
        inten = rng.uniform(0.0, 1.0)
        first.append((c1, c2, a, b, th, inten))
        e1, e2 = rng.uniform(-0.1, 0.1, size=2)
        s1, s2 = rng.uniform(0.9, 1.1, size=2)
        second.append((c1 + e1 * a, c2 + e2 * b, a * s1, b * s2, th, inten))
    m_T = rescale01(gaussian_blur(_paint(n1, n2, first), sigma_px))
    m_R = rescale01(gaussian_blur(_paint(n1, n2, second), sigma_px))
    return m_R, m_T


def splitmix64_uniform(count, seed):
    """``count`` numbers in [-1, 1) from the SplitMix64 generator.

    SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): state s_i = seed + i*G
    with G = 0x9E3779B97F4A7C15, output z = mix(s_i) for i = 1..count, mix
    being two xor-shift-multiply rounds and a final xor-shift. The top 53
    bits map to [0, 1), then to [-1, 1). Used for the Lanczos start vector,
    which the library draws with its own copy of this generator.
    """
    mask = np.uint64(0xFFFFFFFFFFFFFFFF)
    G = np.uint64(0x9E3779B97F4A7C15)
    idx = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (np.uint64(seed) + idx * G) & mask
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) * 2.0 - 1.0


def he_normal(shapes, seed):
    """Flat parameters for 3x3 convolutions shapes = [(Cin, Cout), ...]:
    per layer Cout*9*Cin weights ~ N(0, 2 / (9 Cin)), then Cout zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co in shapes:
        parts.append(rng.standard_normal(co * 9 * ci) * np.sqrt(2.0 / (9 * ci)))
        parts.append(np.zeros(co))
    return np.concatenate(parts)
