"""What the trained warm-start network gains over the method without it.

Held-out pairs of the learned-warm-start configuration (seeds 30000..,
never seen in training), solved at 256^2 to ||g||rel <= 1e-2 from v = 0 and
from the network's velocity: every warm start is kept (it lowers J below
J(0)), both solves converge to the same tolerance and end at nearly the same
velocity, and the warm solves need fewer Newton iterations and matvecs.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def regnk():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1604_02153_gb300 import build, regnk as r
    build.build()
    r.load()
    return r


def test_trained_network_saves_newton_iterations(regnk):
    from paper_1604_02153_gb300 import warmstart
    theta, record = warmstart.load_params()
    assert record["pairs"] >= 10000 and record["loss_per_epoch"][-1] < 1e-3
    net = regnk.UNet(warmstart.S, 1)
    net.set_params(theta)
    n = warmstart.S
    pairs = 8
    seeds = np.arange(warmstart.HELD_OUT_SEED0, warmstart.HELD_OUT_SEED0 + pairs)
    mR, mT, _ = warmstart.make_pairs(n, seeds, procs=1)
    R = regnk.Registration(n, n, warmstart.NT, warmstart.BETA)
    cold, warm = [], []
    for i in range(pairs):
        R.set_images(mR[i], mT[i])
        vc = torch.zeros(2 * n * n, device="cuda")
        ic = R.solve(vc, warmstart.GTOL)
        vw = torch.empty_like(vc)
        assert R.warm_start(net, vw)
        iw = R.solve(vw, warmstart.GTOL)
        assert ic["gnorm_rel"] <= warmstart.GTOL and iw["gnorm_rel"] <= warmstart.GTOL
        d = float(torch.linalg.vector_norm(vw - vc) / torch.linalg.vector_norm(vc))
        assert d < 0.1, d
        cold.append((ic["newton_iters"], ic["matvecs"]))
        warm.append((iw["newton_iters"], iw["matvecs"]))
    R.close()
    net.close()
    cold, warm = np.array(cold), np.array(warm)
    assert warm[:, 0].mean() < cold[:, 0].mean()
    assert warm[:, 1].mean() < cold[:, 1].mean()
    assert np.all(warm[:, 0] <= cold[:, 0])
