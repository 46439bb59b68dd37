"""Batches of independent problems (reg_batch) on the GPU.

Every problem of a concurrent batch must give what a solve of that problem
alone gives (same kernels, same order within the problem): the batched
results are compared with single-context solves of the same problems, and
one problem with the FP64 oracle's solve within the final-velocity bar.
"""

import numpy as np
import pytest

from oracle.problem import Problem
from oracle.solver import Solver
from paper_1604_02153_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def regnk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1604_02153_gb300 import regnk as r
    return r


def dev(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float32).ravel(), device="cuda")


def test_batch_matches_single_solves_and_oracle(regnk):
    sizes = [64, 128, 64, 192, 256, 128, 64, 384]
    nt, beta, gtol = 4, 1e-2, 1e-2
    data = {}
    for n in set(sizes):
        m_T, vstar = inputs.sinusoid_pair(n)
        m_R = Problem(np.zeros((n, n)), m_T, nt, beta).state_solve(vstar)
        data[n] = (m_R, m_T)
    batch = regnk.Batch([(n, n) for n in sizes], nt, [beta] * len(sizes))
    batch.set_images([dev(data[n][0]) for n in sizes], [dev(data[n][1]) for n in sizes])
    vs = [torch.zeros(2 * n * n, device="cuda") for n in sizes]
    infos = batch.solve(vs, gtol)
    torch.cuda.synchronize()
    for i, n in enumerate(sizes):
        assert infos[i]["status_name"] == "REG_OK" and infos[i]["gnorm_rel"] <= gtol
        R = regnk.Registration(n, n, nt, beta)
        R.set_images(dev(data[n][0]), dev(data[n][1]))
        v1 = torch.zeros(2 * n * n, device="cuda")
        info1 = R.solve(v1, gtol)
        torch.cuda.synchronize()
        assert info1["newton_iters"] == infos[i]["newton_iters"]
        assert torch.equal(v1, vs[i]), i          # bitwise: same kernels, same order
        R.close()
    # the 64^2 problem against the oracle's solve
    n = 64
    seed = regnk.default_options().lanczos_seed
    v0 = inputs.splitmix64_uniform(2 * (n // 2) ** 2, seed)
    S = Solver(Problem(data[n][0], data[n][1], nt, beta), precond="2L", lanczos_v0=v0)
    vo, _ = S.solve(np.zeros((2, n, n)), gtol)
    got = vs[0].cpu().numpy().astype(np.float64).reshape(2, n, n)
    assert np.linalg.norm(got - vo) / np.linalg.norm(vo) < 1e-3
    # batched matvecs equal single matvecs
    us = [dev(inputs.random_velocity(n, seed=40 + i, vmax=1.0)) for i, n in enumerate(sizes)]
    Hs = [torch.empty(2 * n * n, device="cuda") for n in sizes]
    batch.hessian_matvec(vs, us, Hs)
    torch.cuda.synchronize()
    for k in (3, 4):
        m = sizes[k]
        R = regnk.Registration(m, m, nt, beta)
        R.set_images(dev(data[m][0]), dev(data[m][1]))
        H1 = torch.empty_like(Hs[k])
        R.hessian_matvec(vs[k], us[k], H1)
        torch.cuda.synchronize()
        assert torch.equal(H1, Hs[k])
        R.close()
    batch.close()
