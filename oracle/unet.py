"""U-Net warm start: forward, backward and Adam (FP64 oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The learned warm start is not part of the paper: a small U-Net maps the
image pair (m_R, m_T) to a stationary velocity v_0 from which the
Gauss-Newton-Krylov solve of §3.4 starts; the solve, run to the same
gradient tolerance, still decides the result (the warm start is used
only if J(v_0) < J(0)). This module is the plain definition of that network,
of the mean-squared-error training loss, of its gradient (written out layer
by layer, checked against central finite differences in the tests) and of
one Adam step (Kingma & Ba 2015, Algorithm 1).

Architecture (fixed; the sizes of the learned-warm-start configuration):
* 4 levels with 32, 64, 128, 256 channels; at each level two 3x3
  convolutions with bias, each followed by ReLU.
* Levels 0-2 of the encoder end in 2x2 average pooling.
* The decoder at levels 2, 1, 0 upsamples the deeper output by nearest-
  neighbour replication, concatenates [upsampled, encoder output of the
  level] along channels and applies two 3x3 convolutions with ReLU.
* A last 3x3 convolution with bias maps 32 channels to the 2 velocity
  components (no activation).
* Every convolution is periodic (the images live on the torus of §3.2):
      out[co, h, w] = b[co] + sum_{a, b, ci} W[co, 3a + b, ci] in[ci, h + a - 1, w + b - 1]
  with indices mod (H, W) (a cross-correlation).

Arrays are channels-first float64: a batch is [B, C, H, W]. The parameter
vector is flat: per layer in LAYERS order, W[co, t, ci] (t = 3a + b), then b[co].

``bf16=True`` rounds to bfloat16 (round to nearest even) at the points where
the GPU stores a bfloat16 value: the inputs, the weights used by the
convolutions, every layer's output and every backpropagated activation
gradient. The arithmetic in between stays float64.
"""

import numpy as np

# (name, Cin, Cout, relu)
LAYERS = [
    ("enc0a", 2, 32, True), ("enc0b", 32, 32, True),
    ("enc1a", 32, 64, True), ("enc1b", 64, 64, True),
    ("enc2a", 64, 128, True), ("enc2b", 128, 128, True),
    ("enc3a", 128, 256, True), ("enc3b", 256, 256, True),
    ("dec2a", 384, 128, True), ("dec2b", 128, 128, True),
    ("dec1a", 192, 64, True), ("dec1b", 64, 64, True),
    ("dec0a", 96, 32, True), ("dec0b", 32, 32, True),
    ("out", 32, 2, False),
]


def param_count():
    return sum(co * 9 * ci + co for _, ci, co, _ in LAYERS)


def unpack(theta):
    """Flat parameter vector -> {name: (W [Cout, 9, Cin], b [Cout])}."""
    out, o = {}, 0
    for name, ci, co, _ in LAYERS:
        W = theta[o:o + co * 9 * ci].reshape(co, 9, ci)
        o += co * 9 * ci
        b = theta[o:o + co]
        o += co
        out[name] = (W, b)
    assert o == theta.size
    return out


def pack(params):
    return np.concatenate([np.concatenate([params[n][0].ravel(), params[n][1].ravel()])
                           for n, _, _, _ in LAYERS])


def round_bf16(x):
    """Round float64 values to the nearest bfloat16 (ties to even), as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _shift(x, a, b):
    """y[..., h, w] = x[..., (h + a - 1) mod H, (w + b - 1) mod W]."""
    return np.roll(x, shift=(1 - a, 1 - b), axis=(-2, -1))


def conv_forward(x, W, b):
    """Periodic 3x3 cross-correlation with bias; x [B, Cin, H, W], W [Cout, 9, Cin]."""
    out = np.zeros((x.shape[0], W.shape[0]) + x.shape[2:])
    for a in range(3):
        for bb in range(3):
            out += np.einsum("oc,nchw->nohw", W[:, 3 * a + bb, :], _shift(x, a, bb))
    return out + b[None, :, None, None]


def conv_backward(x, W, dout):
    """Gradients of conv_forward: (dx, dW, db) for the upstream gradient dout."""
    dW = np.zeros_like(W)
    dx = np.zeros_like(x)
    for a in range(3):
        for bb in range(3):
            xs = _shift(x, a, bb)
            dW[:, 3 * a + bb, :] = np.einsum("nohw,nchw->oc", dout, xs)
            # adjoint of the shift: roll back
            dx += np.roll(np.einsum("oc,nohw->nchw", W[:, 3 * a + bb, :], dout),
                          shift=(a - 1, bb - 1), axis=(-2, -1))
    db = dout.sum(axis=(0, 2, 3))
    return dx, dW, db


def pool(x):
    """2x2 average pooling."""
    B, C, H, W = x.shape
    return x.reshape(B, C, H // 2, 2, W // 2, 2).mean(axis=(3, 5))


def pool_backward(dout):
    return np.repeat(np.repeat(dout, 2, axis=2), 2, axis=3) * 0.25


def upsample(x):
    """Nearest-neighbour 2x upsampling."""
    return np.repeat(np.repeat(x, 2, axis=2), 2, axis=3)


def upsample_backward(dout):
    B, C, H, W = dout.shape
    return dout.reshape(B, C, H // 2, 2, W // 2, 2).sum(axis=(3, 5))


def forward(theta, mR, mT, bf16=False, keep=False):
    """v = net(m_R, m_T): mR, mT [B, H, W] -> v [B, 2, H, W].

    With keep=True also returns the cache of layer inputs and outputs that
    backward() needs.
    """
    P = unpack(theta)
    rnd = round_bf16 if bf16 else (lambda z: z)
    x = rnd(np.stack([mR, mT], axis=1).astype(np.float64))
    cache = {}

    def layer(name, inp):
        W, b = P[name]
        relu = dict((n, r) for n, _, _, r in LAYERS)[name]
        z = conv_forward(inp, rnd(W), b)
        y = np.maximum(z, 0.0) if relu else z
        y = rnd(y) if relu else y       # the last layer's output stays FP32 on the GPU
        cache[name] = (inp, y)
        return y

    e0 = layer("enc0b", layer("enc0a", x))
    e1 = layer("enc1b", layer("enc1a", rnd(pool(e0))))
    e2 = layer("enc2b", layer("enc2a", rnd(pool(e1))))
    e3 = layer("enc3b", layer("enc3a", rnd(pool(e2))))
    d2 = layer("dec2b", layer("dec2a", np.concatenate([upsample(e3), e2], axis=1)))
    d1 = layer("dec1b", layer("dec1a", np.concatenate([upsample(d2), e1], axis=1)))
    d0 = layer("dec0b", layer("dec0a", np.concatenate([upsample(d1), e0], axis=1)))
    v = layer("out", d0)
    return (v, cache) if keep else v


def mse(v, target):
    return float(np.mean((v - target) ** 2))


def backward(theta, cache, v, target, bf16=False):
    """Gradient of mse(forward(theta), target) with respect to theta (flat)."""
    P = unpack(theta)
    rnd = round_bf16 if bf16 else (lambda z: z)
    grads = {}

    def layer_back(name, dy, need_dx=True):
        """dy is the gradient with respect to the layer's output y."""
        W, _ = P[name]
        inp, y = cache[name]
        relu = dict((n, r) for n, _, _, r in LAYERS)[name]
        dz = dy * (y > 0) if relu else dy
        dx, dW, db = conv_backward(inp, rnd(W), dz)
        grads[name] = (dW, db)
        return rnd(dx) if need_dx else None

    dv = rnd(2.0 * (v - target) / v.size)
    g = layer_back("out", dv)
    g = layer_back("dec0a", layer_back("dec0b", g))
    c1 = P["dec1b"][0].shape[0]
    de0 = g[:, c1:]                                   # gradient into the level-0 skip
    g = rnd(upsample_backward(g[:, :c1]))
    g = layer_back("dec1a", layer_back("dec1b", g))
    c2 = P["dec2b"][0].shape[0]
    de1 = g[:, c2:]
    g = rnd(upsample_backward(g[:, :c2]))
    g = layer_back("dec2a", layer_back("dec2b", g))
    c3 = P["enc3b"][0].shape[0]
    de2 = g[:, c3:]
    g = rnd(upsample_backward(g[:, :c3]))
    g = layer_back("enc3a", layer_back("enc3b", g))   # gradient w.r.t. pool(e2)
    g = layer_back("enc2a", layer_back("enc2b", rnd(de2 + pool_backward(g))))
    g = layer_back("enc1a", layer_back("enc1b", rnd(de1 + pool_backward(g))))
    layer_back("enc0a", layer_back("enc0b", rnd(de0 + pool_backward(g))), need_dx=False)
    return pack(grads)


def adam_step(theta, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (bias-corrected first and second moments); step counts from 1."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v
