"""Lockstep batches (reg_lockstep) on the GPU: one launch per transport step
over every problem of a batch of uneven grids.

Each problem's objective, gradient, Hessian matvec and whole Newton-Krylov
solve must be bitwise those of a one-problem context with the same options
(P_REG): the batched kernels run the same per-tile bodies, the segmented
reductions use the one-problem partition and order, and the lockstep solver
takes each problem through its own iteration. One problem is also checked
against the FP64 oracle's solve within the final-velocity bar.
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


def pair(n, nt, beta):
    m_T, vstar = inputs.sinusoid_pair(n)
    m_R = Problem(np.zeros((n, n)), m_T, nt, beta).state_solve(vstar)
    return m_R, m_T


def random_pair(n1, n2, seed):
    m_T = inputs.random_field(n1, n2, seed=seed, kmax=6)
    m_R = np.roll(m_T, 2, axis=-1)
    return m_R, m_T


# uneven grids: powers of two and 3 * 2^k, a non-square grid, repeated sizes
# (one FFT launch per run), two betas on one size (two runs of that size)
GRIDS = [(128, 128), (64, 64), (192, 192), (64, 64), (96, 96), (128, 64), (256, 256), (64, 64)]
BETAS = [1e-2, 1e-2, 1e-2, 3e-2, 1e-2, 1e-2, 1e-2, 1e-2]


def test_lockstep_matches_single_contexts(regnk):
    """J, g and H v~ of every problem bitwise equal to a one-problem context,
    the matvec through its first (eager), second (captured) and third
    (replayed graph) call."""
    nt = 4
    data = [random_pair(a, b, 10 + i) for i, (a, b) in enumerate(GRIDS)]
    vs = [dev(0.4 * np.stack([np.sin(np.arange(a * b).reshape(b, a) * 0.01 + i),
                              np.cos(np.arange(a * b).reshape(b, a) * 0.013 - i)]))
          for i, (a, b) in enumerate(GRIDS)]
    vts = [dev(np.random.default_rng(50 + i).standard_normal((2, b, a)) * 0.1)
           for i, (a, b) in enumerate(GRIDS)]
    L = regnk.Lockstep(GRIDS, nt, BETAS)
    L.set_images([dev(d[0]) for d in data], [dev(d[1]) for d in data])
    gs = [torch.empty(2 * a * b, device="cuda") for a, b in GRIDS]
    J = L.objective_gradient(vs, gs)
    Hs = []
    for call in range(3):
        H = [torch.empty(2 * a * b, device="cuda") for a, b in GRIDS]
        L.hessian_matvec(vs, vts, H)
        Hs.append(H)
    torch.cuda.synchronize()
    for i, (a, b) in enumerate(GRIDS):
        R = regnk.Registration(a, b, nt, BETAS[i], precond=regnk.REG_PC_REG)
        R.set_images(dev(data[i][0]), dev(data[i][1]))
        g1 = torch.empty(2 * a * b, device="cuda")
        J1 = R.objective_gradient(vs[i], g1)
        H1 = torch.empty(2 * a * b, device="cuda")
        R.hessian_matvec(vs[i], vts[i], H1)
        torch.cuda.synchronize()
        assert J1 == J[i], i
        assert torch.equal(g1, gs[i]), i
        for call in range(3):
            assert torch.equal(H1, Hs[call][i]), (i, call)
        R.close()
    L.close()


def test_lockstep_solve_matches_single_solves_and_oracle(regnk):
    """reg_lockstep_solve: every problem's iterate, counts and objective
    bitwise those of reg_solve with P_REG; the problems stop after different
    numbers of Newton and PCG iterations, so the masks are exercised. The
    64^2 problem against the oracle's solve (final velocity <= 1e-3)."""
    sizes = [64, 128, 192, 64, 256, 96, 128, 64]
    betas = [1e-2, 1e-2, 1e-2, 5e-2, 1e-2, 1e-2, 2e-2, 1e-2]
    nt, gtol = 4, 1e-2
    data = [pair(n, nt, b) for n, b in zip(sizes, betas)]
    L = regnk.Lockstep([(n, n) for n in sizes], nt, betas)
    L.set_images([dev(d[0]) for d in data], [dev(d[1]) for d in data])
    vs = [torch.zeros(2 * n * n, device="cuda") for n in sizes]
    infos = L.solve(vs, gtol)
    torch.cuda.synchronize()
    newton = set()
    for i, n in enumerate(sizes):
        R = regnk.Registration(n, n, nt, betas[i], precond=regnk.REG_PC_REG)
        R.set_images(dev(data[i][0]), dev(data[i][1]))
        v1 = torch.zeros(2 * n * n, device="cuda")
        info1 = R.solve(v1, gtol)
        torch.cuda.synchronize()
        for k in ("status", "newton_iters", "pcg_iters", "matvecs", "line_search_steps", "J", "J0",
                  "gnorm_rel", "gnorm_inf", "gref_inf"):
            assert info1[k] == infos[i][k], (i, k, info1[k], infos[i][k])
        assert torch.equal(v1, vs[i]), i
        newton.add((info1["newton_iters"], info1["pcg_iters"]))
        R.close()
    assert len(newton) > 1   # the problems do take different paths
    n, nt, beta = 64, 4, 1e-2
    S = Solver(Problem(data[0][0], data[0][1], nt, beta), precond="REG")
    vo, oinfo = S.solve(np.zeros((2, n, n)), gtol)
    got = vs[0].cpu().numpy().astype(np.float64).reshape(2, n, n)
    assert infos[0]["newton_iters"] == oinfo["newton_iters"]
    assert np.linalg.norm(got - vo) / np.linalg.norm(vo) < 1e-3
    assert abs(infos[0]["J"] - oinfo["J"]) / oinfo["J"] < 1e-4
    L.close()


def test_lockstep_single_problem_and_large_displacement(regnk):
    """A batch of one problem equals the one-problem context; a velocity
    whose displacement per step exceeds the fused kernels' 14 cells is
    refused with REG_EINVAL and the batch stays usable."""
    n, nt, beta = 128, 4, 1e-2
    m_R, m_T = pair(n, nt, beta)
    L = regnk.Lockstep([(n, n)], nt, [beta])
    L.set_images([dev(m_R)], [dev(m_T)])
    v = dev(inputs.random_velocity(n, seed=3, vmax=0.5))
    g = torch.empty(2 * n * n, device="cuda")
    J = L.objective_gradient([v], [g])
    R = regnk.Registration(n, n, nt, beta, precond=regnk.REG_PC_REG)
    R.set_images(dev(m_R), dev(m_T))
    g1 = torch.empty_like(g)
    assert R.objective_gradient(v, g1) == J[0]
    torch.cuda.synchronize()
    assert torch.equal(g, g1)
    # 20 cells per step: h_t |v| / h = 20 with h = 2 pi / n, h_t = 1 / nt
    big = dev(np.full((2, n, n), 20 * nt * 2 * np.pi / n))
    with pytest.raises(regnk.RegError) as e:
        L.objective_gradient([big], [g])
    assert e.value.status == regnk.REG_EINVAL
    J2 = L.objective_gradient([v], [g])
    torch.cuda.synchronize()
    assert J2 == J and torch.equal(g, g1)
    R.close()
    L.close()
