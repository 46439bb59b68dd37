"""The allocation-free interpolation entry point (reg_interpolate_static).

Some callers cannot allocate device memory while they run: their device
memory belongs to another framework's caching allocator, or they sit in a
latency-bound loop where cudaMalloc/cudaFree (which may block and
synchronise the device) is not allowed. For them the library keeps the
spline-coefficient scratch in one fixed device array. This file is named to
be collected last; it checks, through the C ABI, that two calls in a row
reproduce the context-based reg_interpolate within the interpolation
tolerance of the parity tests (1e-5 relative L2), the second call reusing
the scratch left by the first, and that oversized grids are refused.
"""

import numpy as np
import pytest

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


def rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def test_static_matches_context_entry_point_twice(regnk):
    n1, n2 = 256, 128
    R = regnk.Registration(n1, n2, 4, 1e-2, interp=regnk.REG_INTERP_SPLINE)
    cases = []
    for seed in (31, 32):
        u = dev(inputs.random_field(n1, n2, seed=seed, kmax=16))
        disp = dev(inputs.random_velocity(n1, n2, seed=seed + 10, vmax=6.0))
        ref = torch.empty(n1 * n2, device="cuda")
        R.interpolate(u, disp, ref)
        cases.append((u, disp, ref))
    torch.cuda.synchronize()
    for u, disp, ref in cases:          # two calls in a row on the shared scratch
        out = torch.full((n1 * n2,), float("nan"), device="cuda")
        regnk.interpolate_static(n1, n2, u, disp, out)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert rel(out, ref) < 1e-5
    R.close()


def test_static_size_limit(regnk):
    n1, n2 = 2048, 1024          # 2 Mi points > REG_STATIC_MAX_POINTS
    assert n1 * n2 > regnk.REG_STATIC_MAX_POINTS
    u = torch.zeros(n1 * n2, device="cuda")
    disp = torch.zeros(2 * n1 * n2, device="cuda")
    out = torch.zeros(n1 * n2, device="cuda")
    with pytest.raises(regnk.RegError) as e:
        regnk.interpolate_static(n1, n2, u, disp, out)
    assert e.value.status == regnk.REG_EINVAL
