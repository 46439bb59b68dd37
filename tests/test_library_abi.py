"""The C-ABI library builds, loads and exports every declared entry point
(CPU only: no call here launches a kernel).

* every ``reg_*`` function declared in include/reg.h is exported by
  libregnk.so and bound by the Python binding;
* reg_default_options returns the documented defaults;
* argument validation happens on the host (REG_EINVAL), and without a GPU
  reg_create fails with REG_ECUDA: there is no CPU fallback.
"""

import ctypes
import os
import re

import pytest

from paper_1604_02153_gb300 import build as libbuild
from paper_1604_02153_gb300 import regnk


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(regnk.LIB_PATH):
        libbuild.build()
    return regnk.load()


def declared_functions(repo_root):
    src = open(os.path.join(repo_root, "include", "reg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(reg_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib, repo_root):
    names = declared_functions(repo_root)
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
        assert name in regnk._SIGNATURES, name


def test_default_options(lib):
    o = regnk.default_options()
    assert o.reg_norm == regnk.REG_H1
    assert o.interp == regnk.REG_INTERP_SPLINE
    assert o.precond == regnk.REG_PC_2L
    assert o.pc_solver == regnk.REG_PCSOLVER_CHEB
    assert o.cheb_iters == 10 and abs(o.pc_eps - 0.1) < 1e-15
    assert abs(o.gabs - 1e-5) < 1e-20 and o.lanczos_steps == 30
    assert o.max_backtracks == 10 and abs(o.armijo_c1 - 1e-4) < 1e-20
    assert o.persistent_matvec == 0 and o.programmatic_launch == 1 and o.fused_transport == 1
    assert o.coarse_nt == 0 and o.coarse_interp == -1 and o.step_tile == -1
    assert o.incompressible == 0 and o.hessian == regnk.REG_HESSIAN_GN
    assert o.precision == regnk.REG_PRECISION_FP64 and o.use_graphs == 1


def _create(lib, n1, n2, nt, beta, **kw):
    h = ctypes.c_void_p()
    o = regnk.default_options(**kw)
    return lib.reg_create(regnk.reg_grid(n1, n2), nt, beta, ctypes.byref(o), ctypes.byref(h)), h


@pytest.mark.parametrize("n1,n2,nt,beta,kw", [
    (48, 64, 4, 1e-2, {}),           # not a multiple of 32
    (160, 64, 4, 1e-2, {}),          # 5 * 32: no FFT for this length
    (96, 96, 4, 1e-2, {"precond": 1}),  # coarse grid 48 is not a supported size
    (64, 16, 4, 1e-2, {}),           # below the minimum size
    (64, 64, 0, 1e-2, {}),           # no time steps
    (64, 64, 4, 0.0, {}),            # beta must be positive
    (64, 64, 4, 1e-2, {"reg_norm": 4}),
    (64, 64, 4, 1e-2, {"interp": 2}),
    (32, 32, 4, 1e-2, {"precond": 1}),  # two-level needs a 32^2 coarse grid at least
    (64, 64, 4, 1e-2, {"coarse_nt": -1}),
    (64, 64, 4, 1e-2, {"coarse_interp": 2}),
    (64, 64, 4, 1e-2, {"step_tile": 10}),
    (64, 64, 4, 1e-2, {"step_tile": -2}),
    (64, 64, 4, 1e-2, {"incompressible": 2}),
    (64, 64, 4, 1e-2, {"hessian": 2}),
    (64, 64, 4, 1e-2, {"hessian": 1, "persistent_matvec": 1}),   # full Newton runs per step
    (64, 64, 4, 1e-2, {"precision": 2}),
    (64, 64, 4, 1e-2, {"use_graphs": 2}),
])
def test_invalid_arguments_rejected_on_host(lib, n1, n2, nt, beta, kw):
    s, h = _create(lib, n1, n2, nt, beta, **kw)
    assert s == regnk.REG_EINVAL
    assert not h.value


def test_null_handles(lib):
    assert lib.reg_set_images(None, None, None) == regnk.REG_EINVAL
    assert lib.reg_destroy(None) == regnk.REG_OK
    assert lib.reg_last_error(None) == b"null context"
    assert lib.reg_step_tiles(None, (ctypes.c_int * 4)()) == regnk.REG_EINVAL
    assert lib.reg_transport_rk2a(None, None, None, None, 4) == regnk.REG_EINVAL
    assert lib.reg_deformation_map(None, None, None, None) == regnk.REG_EINVAL
    assert lib.reg_adjoint_rk2a(None, None, None, None, 4) == regnk.REG_EINVAL


def test_no_cpu_fallback(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    s, h = _create(lib, 64, 64, 4, 1e-2)
    assert s == regnk.REG_ECUDA and not h.value


def test_static_interpolation_rejects_unaligned_buffers(lib):
    # checked on the host before any device work: the addresses are never used
    ok, off = ctypes.c_void_p(1 << 20), ctypes.c_void_p((1 << 20) + 4)
    for u, d, o in [(off, ok, ok), (ok, off, ok), (ok, ok, off)]:
        assert lib.reg_interpolate_static(64, 64, u, d, o, None) == regnk.REG_EINVAL


def test_unet_arguments_and_no_cpu_fallback(lib):
    import torch
    h = ctypes.c_void_p()
    assert lib.reg_unet_create(48, 1, ctypes.byref(h)) == regnk.REG_EINVAL      # not a multiple of 32
    assert lib.reg_unet_create(256, 0, ctypes.byref(h)) == regnk.REG_EINVAL
    assert lib.reg_unet_create(1024, 128, ctypes.byref(h)) == regnk.REG_EINVAL  # over 2^26 pixels
    assert lib.reg_unet_param_count() == 1947138
    assert lib.reg_warm_start(None, None, None, None) == regnk.REG_EINVAL
    if not torch.cuda.is_available():
        assert lib.reg_unet_create(32, 1, ctypes.byref(h)) == regnk.REG_ECUDA and not h.value


def test_lockstep_arguments_and_no_cpu_fallback(lib):
    """reg_lockstep_create validates its grids and options on the host: the
    lockstep form needs P_REG, the spline model, the Gauss-Newton matvec and
    FP64 reductions; without a GPU a valid request fails with REG_ECUDA."""
    import torch
    G = (regnk.reg_grid * 2)(regnk.reg_grid(64, 64), regnk.reg_grid(128, 128))
    beta = (ctypes.c_double * 2)(1e-2, 1e-2)
    h = ctypes.c_void_p()

    def create(grids=G, B=2, nt=4, b=beta, **kw):
        kw.setdefault("precond", regnk.REG_PC_REG)
        o = regnk.default_options(**kw)
        return lib.reg_lockstep_create(grids, B, nt, b, ctypes.byref(o), ctypes.byref(h))

    assert create(precond=regnk.REG_PC_2L) == regnk.REG_EINVAL
    assert create(interp=regnk.REG_INTERP_LAGRANGE) == regnk.REG_EINVAL
    assert create(hessian=regnk.REG_HESSIAN_FULL) == regnk.REG_EINVAL
    assert create(precision=regnk.REG_PRECISION_FP32) == regnk.REG_EINVAL
    assert create(incompressible=1) == regnk.REG_EINVAL
    assert create(beta_w=1e-3) == regnk.REG_EINVAL
    assert create(B=0) == regnk.REG_EINVAL
    assert create(nt=0) == regnk.REG_EINVAL
    bad = (regnk.reg_grid * 2)(regnk.reg_grid(64, 64), regnk.reg_grid(100, 100))
    assert create(grids=bad) == regnk.REG_EINVAL
    assert create(b=(ctypes.c_double * 2)(1e-2, 0.0)) == regnk.REG_EINVAL
    assert lib.reg_lockstep_solve(None, None, 1e-2, None) == regnk.REG_EINVAL
    assert lib.reg_lockstep_set_images(None, None, None) == regnk.REG_EINVAL
    if not torch.cuda.is_available():
        assert create() == regnk.REG_ECUDA and not h.value
