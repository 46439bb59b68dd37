"""Small fixed workloads for kernel profiling (ncu) of libregnk.

    python profcase.py --n 1024 --nt 8 --matvecs 3

sets up the phantom pair at n^2 (seed 100), evaluates the objective and
gradient at a smooth velocity (max |v| = 0.2) and applies the GN Hessian
`--matvecs` times; `--precond` also applies the two-level preconditioner
once and times a PCG solve with it; `--pcg` times a PCG solve with the
spectral preconditioner P_REG (graph replay of the matvec alone). Prints
the wall time per matvec. The workload holds a few hundred MB
on the device at 1024^2.

    python profcase.py --lockstep 1

instead solves the bench's batch64 workload (64 problems of uneven size,
the analytic pair, nt = 4, beta = 1e-2, P_REG) with one lockstep batch that
many times and prints the wall time per batch (about 1.5 GB on the device).

    python profcase.py --d3 128 --nt 4 --matvecs 3

instead sets up a 3D problem on an n^3 grid (band-limited random images,
seeds 9 and 10, a smooth velocity with max |v| = 0.3), evaluates J and the
gradient, then times the GN matvec, J and the gradient at a new velocity
(two velocities in turn) and the transport with CUDA events (median);
(74 + 7 nt) n^3 floats on the device (0.9 GB at 128^3, 6.8 GB at 256^3).
"""

import argparse
import os
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--nt", type=int, default=8)
    ap.add_argument("--matvecs", type=int, default=3)
    ap.add_argument("--lagrange", action="store_true")
    ap.add_argument("--precond", action="store_true")
    ap.add_argument("--persistent", type=int, default=0)
    ap.add_argument("--pcg", action="store_true")
    ap.add_argument("--pdl", type=int, default=1, help="programmatic_launch option (0 or 1)")
    ap.add_argument("--fused", type=int, default=1, help="fused_transport option (0 or 1)")
    ap.add_argument("--step-tile", type=int, default=-1,
                    help="step_tile option (-1: timed at creation, 0: built-in, 1..9: fixed)")
    ap.add_argument("--flow", type=int, default=0, help="flow_matvec option (0 or 1)")
    ap.add_argument("--graph-pdl", type=int, default=0, help="graph_pdl option (0, 1 or 2)")
    ap.add_argument("--coarse-nt", type=int, default=0, help="coarse_nt option (0: the problem's)")
    ap.add_argument("--coarse-lagrange", action="store_true",
                    help="cubic Lagrange on P_2L's coarse grid (the bench's chosen form)")
    ap.add_argument("--unet", type=int, default=0,
                    help="instead: this many warm-start network training steps (batch 8, 256^2)")
    ap.add_argument("--conv-path", type=int, default=0,
                    help="with --unet: 0 mma.sync convolutions, 1 tcgen05 convolutions")
    ap.add_argument("--batch", type=int, default=8, help="with --unet: pairs per step")
    ap.add_argument("--lockstep", type=int, default=0,
                    help="instead: this many lockstep solves of the 64-problem batch workload")
    ap.add_argument("--d3", type=int, default=0,
                    help="instead: the 3D path on a d3^3 grid (GN matvec, gradient, transport)")
    a = ap.parse_args()
    if a.d3:
        return d3_case(a.d3, a.nt, a.matvecs, a.lagrange)
    if a.unet:
        return unet_case(a.unet, a.conv_path, a.batch)
    if a.lockstep:
        return lockstep_case(a.lockstep)
    import numpy as np
    import torch

    from paper_1604_02153_gb300 import inputs, regnk
    n = a.n
    m_R, m_T = inputs.ellipse_phantoms(n, seed=100)
    v = inputs.random_velocity(n, seed=7, vmax=0.2)
    u = inputs.random_velocity(n, seed=8, vmax=1.0)
    f = lambda x: torch.tensor(np.ascontiguousarray(x, dtype=np.float32).ravel(), device="cuda")
    pc = {} if a.precond else {"precond": regnk.REG_PC_REG}
    R = regnk.Registration(n, n, a.nt, 1e-2,
                           interp=regnk.REG_INTERP_LAGRANGE if a.lagrange else regnk.REG_INTERP_SPLINE,
                           persistent_matvec=a.persistent, programmatic_launch=a.pdl,
                           fused_transport=a.fused, step_tile=a.step_tile, flow_matvec=a.flow,
                           graph_pdl=a.graph_pdl, coarse_nt=a.coarse_nt,
                           coarse_interp=regnk.REG_INTERP_LAGRANGE if a.coarse_lagrange else -1,
                           **pc)
    R.set_images(f(m_R), f(m_T))
    vd, ud = f(v), f(u)
    g = torch.empty_like(vd)
    R.objective_gradient(vd, g)
    H = torch.empty_like(vd)
    R.hessian_matvec(vd, ud, H)          # first use: module loading, attributes
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(a.matvecs):
        R.hessian_matvec(vd, ud, H)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / max(1, a.matvecs)
    # device time per matvec: CUDA events around each call on the launching
    # stream, median
    st = torch.cuda.current_stream()
    dev_ms = []
    for _ in range(max(3, a.matvecs)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        R.hessian_matvec(vd, ud, H)
        e1.record(st)
        torch.cuda.synchronize()
        dev_ms.append(e0.elapsed_time(e1))
    tiles = " ".join(f"{l}/{k}={t[0]}x{t[1]}" for (l, k), t in R.step_tiles().items())
    print(f"n={n} nt={a.nt} persistent={a.persistent} pdl={a.pdl} fused={a.fused} flow={a.flow} "
          f"step tiles {tiles}: matvec {1e3 * dt:.3f} ms (wall, incl. host), "
          f"{1e3 * float(np.median(dev_ms)):.1f} us (CUDA events, median of {len(dev_ms)})")
    if a.pcg and not a.precond:
        x = torch.empty_like(vd)
        R.kkt_solve(vd, g, 1e-12, a.matvecs, x)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = R.kkt_solve(vd, g, 1e-12, a.matvecs, x)
        torch.cuda.synchronize()
        dk = time.perf_counter() - t0
        print(f"n={n} PCG (P_REG) {info['pcg_iters']} iterations "
              f"{1e3 * dk / max(1, info['pcg_iters']):.3f} ms per iteration (graph replay of the matvec)")
    if a.precond:
        z = torch.empty_like(vd)
        R.precond_apply(g, z)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(a.matvecs):
            R.precond_apply(g, z)
        torch.cuda.synchronize()
        dp = (time.perf_counter() - t0) / max(1, a.matvecs)
        print(f"n={n} P_2L apply {1e3 * dp:.3f} ms (wall, eager launches, incl. host)")
        x = torch.empty_like(vd)
        info = R.kkt_solve(vd, g, 1e-12, a.matvecs, x)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = R.kkt_solve(vd, g, 1e-12, a.matvecs, x)
        torch.cuda.synchronize()
        dk = time.perf_counter() - t0
        print(f"n={n} PCG {info['pcg_iters']} iterations {1e3 * dk / max(1, info['pcg_iters']):.3f} "
              f"ms per iteration (graph replay of matvec and P_2L)")
    R.close()


def d3_case(n, nt, reps, lagrange):
    import numpy as np
    import torch

    from paper_1604_02153_gb300 import inputs, regnk
    f = lambda x: torch.tensor(np.ascontiguousarray(x, dtype=np.float32).ravel(), device="cuda")
    m_T = f(inputs.random_field3(n, n, n, seed=9, kmax=4))
    m_R = f(inputs.random_field3(n, n, n, seed=11, kmax=4))
    v = f(inputs.random_velocity3(n, n, n, seed=10, kmax=3, vmax=0.3))
    u = f(inputs.random_velocity3(n, n, n, seed=8, kmax=3, vmax=1.0))
    R = regnk.Registration3(n, n, n, nt, 1e-2,
                            interp=regnk.REG_INTERP_LAGRANGE if lagrange else regnk.REG_INTERP_SPLINE)
    R.set_images(m_R, m_T)
    g = torch.empty_like(v)
    H = torch.empty_like(v)
    m1 = torch.empty_like(m_T)
    R.objective_gradient(v, g)
    R.hessian_matvec(v, u, H)
    R.transport(v, m_T, m1)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()

    def timed(fn):
        ms = []
        for _ in range(max(3, reps)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            fn()
            e1.record(st)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return float(np.median(ms))

    # two velocities in turn: every J + gradient call solves the state anew
    v2 = v * 1.001
    vs = [v, v2]
    k = [0]

    def new_velocity():
        k[0] ^= 1
        R.objective_gradient(vs[k[0]], g)

    t_mv = timed(lambda: R.hessian_matvec(v, u, H))
    t_g = timed(new_velocity)
    t_tr = timed(lambda: R.transport(v, m_T, m1))
    print(f"3D n={n}^3 nt={nt} {'lagrange' if lagrange else 'spline'}: GN matvec {t_mv:.3f} ms, "
          f"J + gradient at a new velocity (state solve included) {t_g:.3f} ms, "
          f"transport {t_tr:.3f} ms (CUDA events, median of {max(3, reps)})")
    R.close()


def lockstep_case(solves):
    """The batch of bench.py's batch64 workload (grids drawn with seed 200
    from BATCH_SIZES^2, m_R = m_T transported by v* on the GPU) solved by a
    lockstep batch with P_REG from v = 0 to ||g||rel 1e-2."""
    import numpy as np
    import torch
    import bench
    from paper_1604_02153_gb300 import inputs, regnk
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(200)
    sizes = [int(x) for x in rng.choice(bench.BATCH_SIZES, size=bench.BATCH_B)]
    f = lambda x: torch.tensor(np.ascontiguousarray(x, dtype=np.float32).ravel(), device=dev)
    cache, mR, mT = {}, [], []
    for n in sizes:
        if n not in cache:
            m_T, vstar = inputs.sinusoid_pair(n)
            R = regnk.Registration(n, n, bench.BATCH_NT, bench.BATCH_BETA, step_tile=0)
            m1 = torch.empty(n * n, device=dev)
            R.transport(f(vstar), f(m_T), m1)
            torch.cuda.synchronize()
            R.close()
            cache[n] = (m1.clone(), f(m_T))
        mR.append(cache[n][0])
        mT.append(cache[n][1])
    L = regnk.Lockstep([(n, n) for n in sizes], bench.BATCH_NT, [bench.BATCH_BETA] * len(sizes))
    L.set_images(mR, mT)
    vs = [torch.zeros(2 * n * n, device=dev) for n in sizes]
    for _ in range(solves):
        for v in vs:
            v.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        infos = L.solve(vs, bench.GTOL)
        torch.cuda.synchronize()
        print(f"lockstep batch of {len(sizes)}: {1e3 * (time.perf_counter() - t0):.2f} ms, "
              f"{sum(i['matvecs'] for i in infos)} matvecs, "
              f"max PCG iterations {max(i['pcg_iters'] for i in infos)}", flush=True)
    L.close()


def unet_case(steps, conv_path=0, B=8):
    """Forward passes and training steps of the warm-start network on a batch
    of B random 256^2 pairs (He-normal weights); prints the time per step."""
    import torch
    from paper_1604_02153_gb300 import inputs, regnk, warmstart
    S = warmstart.S
    net = regnk.UNet(S, B)
    net.set_conv_path(conv_path)
    net.set_params(inputs.he_normal(warmstart.SHAPES, seed=1))
    g = torch.Generator(device="cuda").manual_seed(0)
    mR = torch.rand(B * S * S, device="cuda", generator=g)
    mT = torch.rand(B * S * S, device="cuda", generator=g)
    vt = 0.1 * torch.randn(B * 2 * S * S, device="cuda", generator=g)
    v = torch.empty(B * 2 * S * S, device="cuda")
    net.forward(B, mR, mT, v)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        net.train_step(B, mR, mT, vt, 1e-4)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    print(f"U-Net S={S} B={B} conv path {conv_path}: {1e3 * dt:.3f} ms per training step (wall)")
    net.close()


if __name__ == "__main__":
    main()
