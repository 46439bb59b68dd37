"""GPU parity of the warm-start U-Net kernels (forward, gradients, Adam)
against the FP64 oracle (oracle/unet.py), through the C ABI.

The oracle runs in its bfloat16 mode: it rounds to bfloat16 exactly where
the GPU stores bfloat16 (inputs, convolution weights, layer outputs,
activation gradients), so what remains is FP32 versus FP64 accumulation
order. Through 15 layers that order decides some bfloat16 roundings (one
ulp, 2^-8 relative) and their effect compounds: perturbing the oracle's own
convolution outputs by 1e-7 relative noise before rounding moves its
bfloat16-mode output by 7e-3 relative L2, its gradient by 1.4e-2 (per layer
up to 3e-2) and its loss by 2.7e-3. The bars are about three times those
floors: forward 2e-2, gradient 5e-2 overall and 1e-1 per layer, loss 1e-2.
Structural mistakes (transposed or flipped taps, a wrong pooling) move the
output by 0.1 to 0.8 relative. Adam is checked exactly (to FP32 rounding)
against the oracle's update applied to the GPU's own gradient.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import unet
from paper_1604_02153_gb300 import inputs

pytestmark = pytest.mark.gpu

SHAPES = [(ci, co) for _, ci, co, _ in unet.LAYERS]


@pytest.fixture(scope="module")
def regnk():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1604_02153_gb300 import build, regnk as r
    build.build()
    r.load()
    return r


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def batch(S, B, seed):
    mR = np.stack([inputs.random_field(S, seed=seed + 10 * i + 1, kmax=8) for i in range(B)])
    mT = np.stack([inputs.random_field(S, seed=seed + 10 * i + 2, kmax=8) for i in range(B)])
    vt = np.stack([inputs.random_velocity(S, seed=seed + 10 * i + 3, vmax=0.2) for i in range(B)])
    return mR, mT, vt


def dev(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float32).ravel(), device="cuda")


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("S,B", [(32, 2), (64, 1)])
def test_forward_matches_oracle(regnk, S, B):
    theta = f32(inputs.he_normal(SHAPES, seed=11))
    mR, mT, _ = batch(S, B, 100)
    net = regnk.UNet(S, B)
    net.set_params(theta)
    assert np.array_equal(net.get_params(), theta.astype(np.float32))
    v = torch.empty(B * 2 * S * S, device="cuda")
    net.forward(B, dev(mR), dev(mT), v)
    ref = unet.forward(theta, f32(mR), f32(mT), bf16=True)
    got = v.cpu().numpy().reshape(B, 2, S, S)
    assert rel(got, ref) < 2e-2
    net.close()


def test_forward_selects_problems_by_index(regnk):
    S, B = 32, 2
    theta = f32(inputs.he_normal(SHAPES, seed=12))
    mR, mT, _ = batch(S, 4, 200)
    net = regnk.UNet(S, B)
    net.set_params(theta)
    idx = torch.tensor([3, 1], dtype=torch.int32, device="cuda")
    v = torch.empty(B * 2 * S * S, device="cuda")
    net.forward(B, dev(mR), dev(mT), v, idx=idx)
    v2 = torch.empty_like(v)
    net.forward(B, dev(mR[[3, 1]]), dev(mT[[3, 1]]), v2)
    assert torch.equal(v, v2)
    net.close()


def test_gradients_match_oracle(regnk):
    S, B = 32, 2
    theta = f32(inputs.he_normal(SHAPES, seed=13))
    mR, mT, vt = batch(S, B, 300)
    net = regnk.UNet(S, B)
    net.set_params(theta)
    loss, g = net.gradients(B, dev(mR), dev(mT), dev(vt))
    v, cache = unet.forward(theta, f32(mR), f32(mT), bf16=True, keep=True)
    g_ref = unet.backward(theta, cache, v, f32(vt), bf16=True)
    assert abs(loss - unet.mse(v, f32(vt))) <= 1e-2 * unet.mse(v, f32(vt))
    assert rel(g, g_ref) < 5e-2
    o = 0
    for name, ci, co, _ in unet.LAYERS:
        n = co * 9 * ci + co
        assert rel(g[o:o + n], g_ref[o:o + n]) < 1e-1, name
        o += n
    net.close()


def test_adam_step_and_training_lowers_the_loss(regnk):
    S, B = 32, 2
    theta = f32(inputs.he_normal(SHAPES, seed=14))
    mR, mT, vt = batch(S, B, 400)
    net = regnk.UNet(S, B)
    net.set_params(theta)
    _, g = net.gradients(B, dev(mR), dev(mT), dev(vt))
    l0 = net.train_step(B, dev(mR), dev(mT), dev(vt), lr=1e-3)
    # the step used the same gradient: compare with the oracle's Adam on it
    new, _, _ = unet.adam_step(theta, g.astype(np.float64), np.zeros_like(theta),
                               np.zeros_like(theta), 1, lr=1e-3)
    got = net.get_params().astype(np.float64)
    assert np.max(np.abs(got - new)) <= 1e-6 * max(1.0, np.abs(theta).max())
    losses = [l0] + [net.train_step(B, dev(mR), dev(mT), dev(vt), lr=1e-3) for _ in range(30)]
    assert losses[-1] < 0.5 * losses[0]
    net.close()


def test_rejected_arguments(regnk):
    net = regnk.UNet(32, 2)
    v = torch.empty(2 * 32 * 32 * 3, device="cuda")
    m = torch.zeros(3 * 32 * 32, device="cuda")
    with pytest.raises(regnk.RegError):
        net.forward(3, m, m, v)          # more problems than batch_max
    with pytest.raises(regnk.RegError):
        net.forward(1, m[1:1025], m[:1024], v[:2048])   # off a 16-byte boundary
    net.close()


def test_warm_start_rejects_a_velocity_that_does_not_lower_J(regnk):
    """With all parameters zero the network predicts v_0 = 0, so J(v_0) =
    J(0) is not lower and the warm start falls back to v = 0."""
    n = 64
    net = regnk.UNet(n, 1)
    net.set_params(np.zeros(unet.param_count()))
    R = regnk.Registration(n, n, 4, 1e-2)
    mR, mT, _ = batch(n, 1, 500)
    R.set_images(dev(mR[0]), dev(mT[0]))
    v = torch.full((2 * n * n,), 7.0, device="cuda")
    assert R.warm_start(net, v) is False
    assert float(v.abs().max()) == 0.0
    R.close()
    net.close()


def test_warm_start_prolongs_the_network_velocity(regnk):
    """On a 2x grid the kept velocity is the spectral prolongation of the
    network's output for the spectrally restricted images (checked against
    the oracle's restriction, network and prolongation)."""
    from oracle import spectral
    S, n = 32, 64
    theta = f32(inputs.he_normal(SHAPES, seed=15)) * 0.05
    net = regnk.UNet(S, 1)
    net.set_params(theta)
    R = regnk.Registration(n, n, 4, 1e-2)
    mT = inputs.random_field(n, seed=601, kmax=8)
    vstar = inputs.random_velocity(n, seed=602, vmax=0.2)
    # m_R: m_T moved by a smooth field, so that the network's v_0 is informative
    from oracle.problem import Problem
    P = Problem(np.zeros((n, n)), f32(mT), 4, 1e-2)
    P.state_solve(f32(vstar))
    mR = P.m[-1]
    R.set_images(dev(mR), dev(mT))
    v = torch.empty(2 * n * n, device="cuda")
    kept = R.warm_start(net, v)
    mRs = spectral.restrict(f32(mR))
    mTs = spectral.restrict(f32(mT))
    v0 = unet.forward(theta, mRs[None], mTs[None], bf16=True)[0]
    v_ref = np.stack([spectral.prolong(v0[0]), spectral.prolong(v0[1])])
    if kept:
        assert rel(v.cpu().numpy().reshape(2, n, n), v_ref) < 2e-2
    else:
        assert float(v.abs().max()) == 0.0
    R.close()
    net.close()


@pytest.mark.parametrize("S,B", [(32, 2), (64, 1)])
def test_tcgen05_convolutions_match_mma_sync_and_oracle(regnk, S, B):
    """The convolutions on tcgen05 (tensor memory accumulator) give the
    network of the mma.sync path up to accumulation order: the forward pass
    and the gradients against the oracle at the bars above, and against the
    mma.sync path at the same bars; a training step on that path lowers the
    loss like the other."""
    theta = f32(inputs.he_normal(SHAPES, seed=21))
    mR, mT, vt = batch(S, B, 600)
    out = {}
    for path in (0, 1):
        net = regnk.UNet(S, B)
        net.set_conv_path(path)
        net.set_params(theta)
        v = torch.empty(B * 2 * S * S, device="cuda")
        net.forward(B, dev(mR), dev(mT), v)
        loss, g = net.gradients(B, dev(mR), dev(mT), dev(vt))
        out[path] = (v.cpu().numpy().reshape(B, 2, S, S), loss, g)
        net.close()
    ref, cache = unet.forward(theta, f32(mR), f32(mT), bf16=True, keep=True)
    g_ref = unet.backward(theta, cache, ref, f32(vt), bf16=True)
    v1, loss1, g1 = out[1]
    assert rel(v1, ref) < 2e-2
    assert rel(v1, out[0][0]) < 2e-2
    assert abs(loss1 - unet.mse(ref, f32(vt))) <= 1e-2 * unet.mse(ref, f32(vt))
    assert rel(g1, g_ref) < 5e-2
    assert rel(g1, out[0][2]) < 5e-2
    net = regnk.UNet(S, B)
    net.set_conv_path(1)
    net.set_params(theta)
    losses = [net.train_step(B, dev(mR), dev(mT), dev(vt), lr=1e-3) for _ in range(31)]
    assert losses[-1] < 0.5 * losses[0]
    net.close()
