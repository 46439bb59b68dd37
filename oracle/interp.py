"""Periodic cubic interpolation at off-grid points (FP64 oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

§3.2 and §3.5 ("Interpolation"): the semi-Lagrangian scheme evaluates fields
at departure points with a C2 cubic spline model, the data extended
periodically. On the torus the periodic extension is exact modular wrap
(equivalent to padding by at least the largest displacement plus the stencil
support, which is what the paper does).

Points are given in index units: p_1 = x_1 / h_1, p_2 = x_2 / h_2. With
i0 = floor(p), t = p - i0 the value is the tensor sum over offsets
a, b in {-1, 0, 1, 2} of c[(j0 + b) mod n2, (i0 + a) mod n1] w_a(t_1) w_b(t_2).

Two weight families:
* "spline"   (the paper's model, the default): centred cubic B-spline weights
  applied to the prefiltered coefficients c = spectral.spline_prefilter(u);
* "lagrange" (a variant): cubic Lagrange weights on the nodes -1, 0, 1, 2
  applied to the raw samples c = u.
"""

import numpy as np

from . import spectral


def bspline3_weights(t):
    """Cubic B-spline weights at offsets -1, 0, 1, 2 for fractional t in [0,1)."""
    s = 1.0 - t
    return (
        s * s * s / 6.0,
        (3.0 * t * t * t - 6.0 * t * t + 4.0) / 6.0,
        (-3.0 * t * t * t + 3.0 * t * t + 3.0 * t + 1.0) / 6.0,
        t * t * t / 6.0,
    )


def lagrange3_weights(t):
    """Cubic Lagrange weights on nodes -1, 0, 1, 2 evaluated at t."""
    return (
        -t * (t - 1.0) * (t - 2.0) / 6.0,
        (t + 1.0) * (t - 1.0) * (t - 2.0) / 2.0,
        -(t + 1.0) * t * (t - 2.0) / 2.0,
        (t + 1.0) * t * (t - 1.0) / 6.0,
    )


def coefficients(u, kind):
    """Coefficients that the 4x4 stencil is applied to."""
    if kind == "spline":
        return spectral.spline_prefilter(u)
    if kind == "lagrange":
        return np.array(u, dtype=np.float64, copy=True)
    raise ValueError(kind)


def evaluate(c, p1, p2, kind):
    """Evaluate the interpolant with coefficients c at index-space points.

    c: (n2, n1) coefficients; p1, p2: arrays of equal shape (any shape).
    """
    n2, n1 = c.shape
    wfun = bspline3_weights if kind == "spline" else lagrange3_weights
    f1 = np.floor(p1)
    f2 = np.floor(p2)
    t1 = p1 - f1
    t2 = p2 - f2
    i0 = f1.astype(np.int64)
    j0 = f2.astype(np.int64)
    w1 = wfun(t1)
    w2 = wfun(t2)
    out = np.zeros(np.shape(p1), dtype=np.float64)
    for b in range(4):
        jj = np.mod(j0 + (b - 1), n2)
        for a in range(4):
            ii = np.mod(i0 + (a - 1), n1)
            out += c[jj, ii] * w1[a] * w2[b]
    return out


def interp(u, p1, p2, kind):
    """Interpolate the samples u at index-space points (p1, p2)."""
    return evaluate(coefficients(u, kind), p1, p2, kind)


def node_coordinates(n1, n2):
    """Index-space coordinates of every grid node, shapes (n2, n1)."""
    J, I = np.meshgrid(np.arange(n2, dtype=np.float64),
                       np.arange(n1, dtype=np.float64), indexing="ij")
    return I, J
