"""The registration path on 3D grids (reg3_*) against the 3D FP64 oracle.

Bars: the spectral operators within 1e-5 relative L2 (FP32 FFTs of smooth
fields); transported images, the gradient and the Gauss-Newton matvec within
the stated 1e-4 relative L2; J within 1e-5; the solve with the oracle's
Newton and PCG iteration counts and the final velocity within 1e-3. A problem
constant along x_3 also reproduces the 2D GPU path.
"""

import numpy as np
import pytest

from oracle import d3
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


def host(t, shape):
    return t.cpu().numpy().astype(np.float64).reshape(shape)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


N1, N2, N3 = 32, 64, 32


def test_spectral_operators(regnk):
    u = f32(inputs.random_field3(N1, N2, N3, seed=1, kmax=6))
    v = f32(inputs.random_velocity3(N1, N2, N3, seed=2, kmax=5, vmax=1.0))
    # a nonzero mean per component exercises the k = 0 weight beta^s of the
    # negative powers (beta A discards the mean, so s = 1 takes v itself)
    vm = f32(v + np.array([0.3, -0.2, 0.1])[:, None, None, None])
    R = regnk.Registration3(N1, N2, N3, 4, 2e-2)
    g = torch.empty(3 * R.N, device="cuda")
    R.spectral(regnk.REG_SPEC_GRAD, dev(u), g)
    assert rel(host(g, (3, N3, N2, N1)), d3.grad(u)) < 1e-5
    dv = torch.empty(R.N, device="cuda")
    R.spectral(regnk.REG_SPEC_DIV, dev(v), dv)
    assert rel(host(dv, (N3, N2, N1)), d3.div(v)) < 1e-5
    for s in (1.0, -1.0, -0.5):
        x = v if s == 1.0 else vm
        o = torch.empty(3 * R.N, device="cuda")
        R.spectral(regnk.REG_SPEC_REGPOW, dev(x), o, s=s)
        assert rel(host(o, (3, N3, N2, N1)), d3.reg_power(x, 2e-2, "H1", s)) < 1e-5, s
    R.close()


@pytest.mark.parametrize("interp", ["spline", "lagrange"])
def test_transport(regnk, interp):
    nt = 4
    m0 = f32(inputs.random_field3(N1, N2, N3, seed=3, kmax=4))
    v = f32(inputs.random_velocity3(N1, N2, N3, seed=4, kmax=3, vmax=0.5))
    R = regnk.Registration3(N1, N2, N3, nt, 1e-2,
                            interp=regnk.REG_INTERP_SPLINE if interp == "spline"
                            else regnk.REG_INTERP_LAGRANGE)
    m1 = torch.empty(R.N, device="cuda")
    R.transport(dev(v), dev(m0), m1)
    P = d3.Problem3(np.zeros_like(m0), m0, nt, 1e-2, kind=interp)
    ref = P.state_solve(v)
    assert rel(host(m1, (N3, N2, N1)), ref) < 1e-4
    R.close()


@pytest.mark.parametrize("interp", ["spline", "lagrange"])
def test_objective_gradient_and_gauss_newton_matvec(regnk, interp):
    nt, beta = 4, 1e-2
    m_T = f32(inputs.random_field3(N1, N2, N3, seed=5, kmax=4))
    m_R = f32(inputs.random_field3(N1, N2, N3, seed=6, kmax=4))
    v = f32(inputs.random_velocity3(N1, N2, N3, seed=7, kmax=3, vmax=0.3))
    u = f32(inputs.random_velocity3(N1, N2, N3, seed=8, kmax=3, vmax=1.0))
    kind = regnk.REG_INTERP_SPLINE if interp == "spline" else regnk.REG_INTERP_LAGRANGE
    R = regnk.Registration3(N1, N2, N3, nt, beta, interp=kind)
    R.set_images(dev(m_R), dev(m_T))
    g = torch.empty(3 * R.N, device="cuda")
    J = R.objective_gradient(dev(v), g)
    H = torch.empty(3 * R.N, device="cuda")
    R.hessian_matvec(dev(v), dev(u), H)
    P = d3.Problem3(m_R, m_T, nt, beta, kind=interp)
    J_ref, g_ref = P.objective_gradient(v)
    H_ref = P.hessian_matvec(u)
    assert abs(J - J_ref) < 1e-5 * abs(J_ref)
    assert rel(host(g, (3, N3, N2, N1)), g_ref) < 1e-4
    assert rel(host(H, (3, N3, N2, N1)), H_ref) < 1e-4
    R.close()


def test_solve_matches_oracle(regnk):
    n, nt, beta, gtol = 32, 4, 1e-2, 1e-2
    m_T = f32(inputs.random_field3(n, n, n, seed=9, kmax=3))
    vstar = f32(inputs.random_velocity3(n, n, n, seed=10, kmax=2, vmax=0.3))
    m_R = f32(d3.Problem3(np.zeros_like(m_T), m_T, nt, beta).state_solve(vstar))
    R = regnk.Registration3(n, n, n, nt, beta)
    R.set_images(dev(m_R), dev(m_T))
    v = torch.zeros(3 * R.N, device="cuda")
    info = R.solve(v, gtol)
    vo, oinfo = d3.Problem3(m_R, m_T, nt, beta).solve(np.zeros((3, n, n, n)), gtol)
    assert info["gnorm_rel"] <= gtol
    assert info["newton_iters"] == oinfo["newton_iters"]
    assert info["pcg_iters"] == oinfo["pcg_iters"]
    assert rel(host(v, (3, n, n, n)), vo) < 1e-3
    assert abs(info["J"] - oinfo["J"]) < 1e-4 * oinfo["J"]
    R.close()


def test_constant_along_x3_gives_the_2d_path(regnk):
    """Fields constant along x_3 and v_3 = 0: the 3D gradient and matvec
    equal the 2D GPU path's (tiled), J the 2D J times 2 pi."""
    n, n3, nt, beta = 64, 32, 4, 1e-2
    m_T = f32(inputs.random_field(n, seed=11, kmax=6))
    m_R = f32(inputs.random_field(n, seed=12, kmax=6))
    v2 = f32(inputs.random_velocity(n, seed=13, vmax=0.3))
    u2 = f32(inputs.random_velocity(n, seed=14, vmax=1.0))
    tile = lambda a: np.repeat(a[None], n3, axis=0)
    v3 = np.stack([tile(v2[0]), tile(v2[1]), np.zeros((n3, n, n))])
    u3 = np.stack([tile(u2[0]), tile(u2[1]), np.zeros((n3, n, n))])
    R2 = regnk.Registration(n, n, nt, beta, precond=regnk.REG_PC_REG)
    R2.set_images(dev(m_R), dev(m_T))
    g2 = torch.empty(2 * n * n, device="cuda")
    J2 = R2.objective_gradient(dev(v2), g2)
    H2 = torch.empty(2 * n * n, device="cuda")
    R2.hessian_matvec(dev(v2), dev(u2), H2)
    R3 = regnk.Registration3(n, n, n3, nt, beta)
    R3.set_images(dev(tile(m_R)), dev(tile(m_T)))
    g3 = torch.empty(3 * R3.N, device="cuda")
    J3 = R3.objective_gradient(dev(v3), g3)
    H3 = torch.empty(3 * R3.N, device="cuda")
    R3.hessian_matvec(dev(v3), dev(u3), H3)
    assert abs(J3 - 2 * np.pi * J2) < 1e-5 * abs(J3)
    G2, G3 = host(g2, (2, n, n)), host(g3, (3, n3, n, n))
    K2, K3 = host(H2, (2, n, n)), host(H3, (3, n3, n, n))
    for c in range(2):
        assert rel(G3[c], np.repeat(G2[c][None], n3, axis=0)) < 1e-5
        assert rel(K3[c], np.repeat(K2[c][None], n3, axis=0)) < 1e-5
    assert np.max(np.abs(G3[2])) < 1e-5 * np.max(np.abs(G2))
    R2.close()
    R3.close()


@pytest.mark.parametrize("interp", ["spline", "lagrange"])
@pytest.mark.parametrize("vmax", [0.3, 6.0])
def test_box_and_global_gathers(regnk, interp, vmax):
    """The tricubic gathers from shared-memory boxes (fused_transport 1 when
    the displacements fit a box: at vmax 0.3 the reach is under one cell, a
    box of about 36 x 12 x 12 floats) and from global memory (fused_transport
    0, and the fallback of fused_transport 1 at vmax 6, a reach of about 15
    cells along x_2 that needs a box of over 200 KB): transported image, gradient
    and GN matvec against the oracle at the stated bars, and the two forms
    against each other (the same stencil arithmetic) within 1e-6."""
    nt, beta = 4, 1e-2
    kind = regnk.REG_INTERP_SPLINE if interp == "spline" else regnk.REG_INTERP_LAGRANGE
    m_T = f32(inputs.random_field3(N1, N2, N3, seed=15, kmax=4))
    m_R = f32(inputs.random_field3(N1, N2, N3, seed=16, kmax=4))
    v = f32(inputs.random_velocity3(N1, N2, N3, seed=17, kmax=3, vmax=vmax))
    u = f32(inputs.random_velocity3(N1, N2, N3, seed=18, kmax=3, vmax=1.0))
    P = d3.Problem3(m_R, m_T, nt, beta, kind=interp)
    m1_ref = P.state_solve(v)
    J_ref, g_ref = P.objective_gradient(v)
    H_ref = P.hessian_matvec(u)
    out = {}
    for fused in (0, 1):
        R = regnk.Registration3(N1, N2, N3, nt, beta, interp=kind, fused_transport=fused)
        m1 = torch.empty(R.N, device="cuda")
        R.transport(dev(v), dev(m_T), m1)
        R.set_images(dev(m_R), dev(m_T))
        g = torch.empty(3 * R.N, device="cuda")
        J = R.objective_gradient(dev(v), g)
        H = torch.empty(3 * R.N, device="cuda")
        R.hessian_matvec(dev(v), dev(u), H)
        o = (host(m1, (N3, N2, N1)), host(g, (3, N3, N2, N1)), host(H, (3, N3, N2, N1)))
        assert rel(o[0], m1_ref) < 1e-4
        assert abs(J - J_ref) < 1e-5 * abs(J_ref)
        assert rel(o[1], g_ref) < 1e-4
        assert rel(o[2], H_ref) < 1e-4
        out[fused] = o
        R.close()
    for a, b in zip(out[0], out[1]):
        assert rel(b, a) < 1e-6


@pytest.mark.parametrize("interp", ["spline", "lagrange"])
def test_deformation_map(regnk, interp):
    """u = y - x and det grad y against the oracle (the composed gathers
    within 1e-4 relative L2, the determinant within 1e-4 of the oracle's at
    every node); the shear flow v = (a sin x_2, 0, 0) gives u = (-a sin x_2,
    0, 0) and det = 1 to FP32 rounding."""
    nt = 4
    kind = regnk.REG_INTERP_SPLINE if interp == "spline" else regnk.REG_INTERP_LAGRANGE
    v = f32(inputs.random_velocity3(N1, N2, N3, seed=31, kmax=3, vmax=0.5))
    R = regnk.Registration3(N1, N2, N3, nt, 1e-2, interp=kind)
    u = torch.empty(3 * R.N, device="cuda")
    det = torch.empty(R.N, device="cuda")
    R.deformation_map(dev(v), u, det)
    u_ref = d3.deformation_map(v, nt, interp)
    assert rel(host(u, (3, N3, N2, N1)), u_ref) < 1e-4
    assert np.max(np.abs(host(det, (N3, N2, N1)) - d3.det_grad_map(u_ref))) < 1e-4
    K, J, I = np.meshgrid(*(np.arange(n) * 2 * np.pi / n for n in (N3, N2, N1)), indexing="ij")
    a = 0.3
    vs = np.stack([a * np.sin(J), np.zeros_like(J), np.zeros_like(J)])
    R.deformation_map(dev(vs), u, det)
    us = host(u, (3, N3, N2, N1))
    assert np.max(np.abs(us[0] + a * np.sin(J))) < 1e-5
    assert np.max(np.abs(us[1])) < 1e-6 and np.max(np.abs(us[2])) < 1e-6
    assert np.max(np.abs(host(det, (N3, N2, N1)) - 1.0)) < 1e-5
    R.close()


def two_level_problem(n, nt, beta):
    m_T = f32(inputs.random_field3(n, n, n, seed=51, kmax=3))
    vstar = f32(inputs.random_velocity3(n, n, n, seed=52, kmax=2, vmax=0.3))
    m_R = f32(d3.Problem3(np.zeros_like(m_T), m_T, nt, beta).state_solve(vstar))
    return m_R, m_T


def test_two_level_preconditioner(regnk):
    """P_2L on a 64^3 grid (coarse 32^3): the Chebyshev bounds against the
    oracle's (e_min analytic to rounding; e_max the largest Ritz value of 30
    Lanczos steps from the same SplitMix64 vector: the GPU recurrence keeps
    FP32 vectors and does not reorthogonalise, the oracle's does, so the two
    differ beyond the operator's 1e-4, and the bound enters CHEB(k) with a
    5 % margin), and P_2L^-1 r at a velocity against the oracle's with the
    GPU's bounds at the stated 1e-4."""
    n, nt, beta = 64, 4, 1e-2
    m_R, m_T = two_level_problem(n, nt, beta)
    R = regnk.Registration3(n, n, n, nt, beta, precond=regnk.REG_PC_2L)
    R.set_images(dev(m_R), dev(m_T))
    emin, emax = R.eigen_bounds()
    nc = n // 2
    v0 = inputs.splitmix64_uniform(3 * nc ** 3, regnk.default_options().lanczos_seed)
    S = d3.Solver3(d3.Problem3(m_R, m_T, nt, beta), precond="2L",
                   lanczos_v0=v0.reshape(3, nc, nc, nc))
    e = S.estimate_eigenvalues()
    assert abs(emin - e["emin"]) < 1e-12 * e["emin"]
    assert abs(emax - e["emax"]) / e["emax"] < 1e-3
    v = f32(inputs.random_velocity3(n, n, n, seed=53, kmax=2, vmax=0.2))
    r = f32(inputs.random_velocity3(n, n, n, seed=54, kmax=8, vmax=1.0))
    z = torch.empty(3 * R.N, device="cuda")
    R.precond_apply(dev(v), dev(r), z)
    S.eig = {"emin": emin, "emax": emax}
    S.coarse.state_solve(d3.restrict_vec3(v))
    assert rel(host(z, (3, n, n, n)), S.apply_precond(r)) < 1e-4
    R.close()


@pytest.mark.parametrize("pc", ["cheb", "pcg"])
def test_two_level_solve_matches_oracle(regnk, pc):
    """The Newton-Krylov solve with P_2L (CHEB(10), or nested PCG(0.1 eta))
    on 64^3 against the oracle's (the same Lanczos start vector): the same
    Newton iterations, PCG iterations within one, v within the stated 1e-3
    and J within 1e-4; P_2L needs fewer fine-grid matvecs than P_REG on the
    same problem."""
    n, nt, beta, gtol = 64, 4, 1e-2, 1e-2
    m_R, m_T = two_level_problem(n, nt, beta)
    R = regnk.Registration3(n, n, n, nt, beta, precond=regnk.REG_PC_2L,
                            pc_solver=regnk.REG_PCSOLVER_CHEB if pc == "cheb"
                            else regnk.REG_PCSOLVER_PCG)
    R.set_images(dev(m_R), dev(m_T))
    v = torch.zeros(3 * R.N, device="cuda")
    info = R.solve(v, gtol)
    nc = n // 2
    v0 = inputs.splitmix64_uniform(3 * nc ** 3, regnk.default_options().lanczos_seed)
    S = d3.Solver3(d3.Problem3(m_R, m_T, nt, beta), precond="2L",
                   lanczos_v0=v0.reshape(3, nc, nc, nc), pc_solver=pc)
    vo, oinfo = S.solve(np.zeros((3, n, n, n)), gtol)
    assert info["gnorm_rel"] <= gtol
    assert info["newton_iters"] == oinfo["newton_iters"]
    assert abs(info["pcg_iters"] - oinfo["pcg_iters"]) <= 1
    assert info["coarse_matvecs"] > 0
    assert rel(host(v, (3, n, n, n)), vo) < 1e-3
    assert abs(info["J"] - oinfo["J"]) < 1e-4 * oinfo["J"]
    Rr = regnk.Registration3(n, n, n, nt, beta)
    Rr.set_images(dev(m_R), dev(m_T))
    vr = torch.zeros(3 * R.N, device="cuda")
    ir = Rr.solve(vr, gtol)
    assert info["matvecs"] < ir["matvecs"]
    R.close()
    Rr.close()


def test_rejected_arguments_3d(regnk):
    """reg3_create refuses axis lengths it has no FFT or tiles for, P_2L
    whose coarse grid would not be one or whose nested PCG has no tolerance,
    and the variants the 3D context does not run; a P_REG context has no Chebyshev bounds; a gradient before the
    images is a state error; the binding checks tensor sizes."""
    with pytest.raises(regnk.RegError):
        regnk.Registration3(48, 64, 64, 4, 1e-2)
    with pytest.raises(regnk.RegError):
        regnk.Registration3(32, 64, 64, 4, 1e-2, precond=regnk.REG_PC_2L)
    with pytest.raises(regnk.RegError):
        regnk.Registration3(64, 64, 64, 4, 1e-2, precond=regnk.REG_PC_2L,
                            pc_solver=regnk.REG_PCSOLVER_PCG, pc_eps=0.0)
    with pytest.raises(regnk.RegError):
        regnk.Registration3(64, 64, 64, 4, 1e-2, incompressible=1)
    R = regnk.Registration3(32, 32, 32, 4, 1e-2)
    with pytest.raises(regnk.RegError):
        R.eigen_bounds()
    v = torch.zeros(3 * R.N, device="cuda")
    g = torch.empty(3 * R.N, device="cuda")
    with pytest.raises(regnk.RegError):
        R.objective_gradient(v, g)
    with pytest.raises(ValueError):
        R.spectral(regnk.REG_SPEC_GRAD, torch.empty(R.N + 4, device="cuda"), g)
    R.close()
