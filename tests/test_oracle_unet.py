"""Pins of the U-Net warm-start oracle (oracle/unet.py) against what fixes it
independently of its own formulas: scipy's periodic correlation, adjoint
identities, central finite differences of the loss, the closed form of the
first Adam step and torch's bfloat16 rounding."""

import numpy as np
import pytest
from scipy import ndimage

from oracle import unet
from paper_1604_02153_gb300 import inputs


def test_conv_forward_is_periodic_cross_correlation():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 3, 8, 12))
    W = rng.standard_normal((4, 9, 3))
    b = rng.standard_normal(4)
    out = unet.conv_forward(x, W, b)
    for n in range(2):
        for co in range(4):
            ref = np.full((8, 12), b[co])
            for ci in range(3):
                ref += ndimage.correlate(x[n, ci], W[co, :, ci].reshape(3, 3), mode="wrap")
            assert np.allclose(out[n, co], ref, rtol=0, atol=1e-12)


def test_conv_backward_is_the_adjoint():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 5, 8, 8))
    W = rng.standard_normal((3, 9, 5))
    y = rng.standard_normal((2, 3, 8, 8))
    lin = unet.conv_forward(x, W, np.zeros(3))
    dx, dW, db = unet.conv_backward(x, W, y)
    # <conv(x), y> = <x, conv^T(y)> = <W, dW>  (bilinear in x and W)
    assert np.isclose(np.sum(lin * y), np.sum(x * dx), rtol=1e-12)
    assert np.isclose(np.sum(lin * y), np.sum(W * dW), rtol=1e-12)
    assert np.allclose(db, y.sum(axis=(0, 2, 3)))


def test_pool_and_upsample_adjoints():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 3, 8, 8))
    y = rng.standard_normal((2, 3, 4, 4))
    assert np.isclose(np.sum(unet.pool(x) * y), np.sum(x * unet.pool_backward(y)))
    assert np.isclose(np.sum(unet.upsample(y) * x), np.sum(y * unet.upsample_backward(x)))
    # pooling a replicated field returns it
    assert np.allclose(unet.pool(unet.upsample(y)), y)


def test_param_layout():
    assert unet.param_count() == sum(co * 9 * ci + co for _, ci, co, _ in unet.LAYERS)
    theta = np.arange(unet.param_count(), dtype=np.float64)
    assert np.array_equal(unet.pack(unet.unpack(theta)), theta)


@pytest.fixture(scope="module")
def small_problem():
    rng = np.random.default_rng(3)
    theta = inputs.he_normal([(ci, co) for _, ci, co, _ in unet.LAYERS], seed=5)
    mR = rng.uniform(0, 1, (1, 16, 16))
    mT = rng.uniform(0, 1, (1, 16, 16))
    target = 0.2 * rng.standard_normal((1, 2, 16, 16))
    return theta, mR, mT, target


def test_backward_matches_central_differences(small_problem):
    theta, mR, mT, target = small_problem
    v, cache = unet.forward(theta, mR, mT, keep=True)
    g = unet.backward(theta, cache, v, target)
    rng = np.random.default_rng(4)
    # a few coordinates in every layer's weights and biases
    o = 0
    idx = []
    for _, ci, co, _ in unet.LAYERS:
        nW = co * 9 * ci
        idx += list(o + rng.integers(0, nW, 2)) + [o + nW + int(rng.integers(0, co))]
        o += nW + co
    loss = lambda th: unet.mse(unet.forward(th, mR, mT), target)
    for i in idx:
        h = 1e-6 * max(1.0, abs(theta[i]))
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (loss(tp) - loss(tm)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(g).max()), (i, fd, g[i])


def test_planted_mistakes_are_caught(small_problem):
    """A dropped skip gradient or a missing ReLU mask changes the gradient
    far beyond the finite-difference tolerance."""
    theta, mR, mT, target = small_problem
    v, cache = unet.forward(theta, mR, mT, keep=True)
    g = unet.backward(theta, cache, v, target)
    saved = unet.pool_backward
    try:
        unet.pool_backward = lambda d: 0.0 * saved(d)
        g_bad = unet.backward(theta, cache, v, target)
    finally:
        unet.pool_backward = saved
    assert np.linalg.norm(g_bad - g) > 1e-3 * np.linalg.norm(g)


def test_first_adam_step_closed_form():
    rng = np.random.default_rng(6)
    theta = rng.standard_normal(50)
    grad = rng.standard_normal(50)
    new, m, v = unet.adam_step(theta, grad, np.zeros(50), np.zeros(50), 1, lr=1e-3)
    # bias-corrected first step: lr * g / (|g| + eps)
    assert np.allclose(new, theta - 1e-3 * grad / (np.abs(grad) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * grad) and np.allclose(v, 0.001 * grad ** 2)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    x = np.concatenate([rng.standard_normal(10000) * 10.0 ** rng.integers(-8, 8, 10000),
                        [0.0, -0.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 65504.0]])
    ref = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(unet.round_bf16(x), ref)
