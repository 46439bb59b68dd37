#!/usr/bin/env python
"""Benchmark of the semi-Lagrangian Gauss-Newton-Krylov registration hot path.

One step is one complete registration solve, i.e. one pass through every row
of the hot path: departure points, cubic interpolation, state and adjoint
transport, pseudospectral operators, objective and reduced gradient,
incremental state and adjoint (GN Hessian matvec), PCG with the two-level
preconditioner (spectral restriction/prolongation, Chebyshev(10) on the
512^2 coarse grid), Armijo line search and the Newton loop.

Workload: 1024^2 piecewise-smooth phantom pair (12 seeded random ellipses per
image, Gaussian blur sigma = 2 px, second image with perturbed centres and
axes), nt = 8, H1 regularisation with beta continuation 1e-1 -> 1e-2 -> 1e-3
(warm started), stopping at ||g||_inf / ||g(0)||_inf <= 1e-2 per stage. FP32
fields, FP64 reductions. The two-level preconditioner's 512^2 coarse problem
uses nt/2 = 4 time steps (the same displacement per step in coarse cells) and
cubic Lagrange interpolation (no prefilter): §3.4.2 expects the
preconditioner's PDE solves to need little accuracy. The solve still runs to
the same gradient tolerance on the fine problem; against nt = 8 and splines
on the coarse grid this takes 1-2 % more fine matvecs and 40 % less time. Inputs are resident in HBM when timing starts; L2 is
flushed between steps (256 MB write, untimed).

value     = fine-grid GN Hessian matvecs per second of solve time (all ranks).
e2e       = the same through the C-ABI with host buffers: pinned-host images
            copied in, the velocity copied out, inside the timed region.
roofline  = the kernel class with the largest device time: algorithmic
            bytes / its CUDA-event time, from a profiled repeat of the timed
            steps (every launch bracketed by events on the launching stream,
            event nodes inside the replayed graphs), against the measured HBM
            copy bandwidth. Algorithmic bytes per grid point: 24 per
            incremental state step, 16 per adjoint step (+16 for the first of
            each solve, +8 for the last incremental state step: the
            per-velocity inputs and the handover of b~), 4 N (10 nt + 16) per
            GN matvec.
roofline_gn_matvec = the fine GN matvec as one unit (the library call,
            replayed from its CUDA graph) against 4 N (10 nt + 16) bytes.
step_tiles = (threads per block, points per thread) of the unfused
            adjoint and incremental-state step kernels on each grid level, as
            reg_create's timing of the nine shapes chose them.
cpu_baseline / --impl reference = the FP64 numpy oracle on the host cores,
            timed on a bounded sample: one GN Hessian matvec at 1024^2, nt = 8
            on one core; one such matvec per core at once (process pool); and
            the 64^2 analytic problem solved to ||g||rel 1e-2 on one core.
            The ratio of the two arms' values compares solve-level GPU
            matvecs/s (gradients, line search and the coarse level included
            in the time) with bare oracle matvecs/s: a deliberately slow
            program, not a like-for-like rate.
plain_form = the same solve with FP32 reductions, no CUDA graphs and plain
            launches (as many timed solves as the chosen form, after one
            warm-up, CUDA events): the "plain FP32" form the chosen one is
            compared against.
solver_arms = the coarse solver of P_2L as nested PCG(0.1 eta) against
            CHEB(10), and the coarse problem at the problem's nt and splines.
fft_comparator = the hand-written spectral operator (beta A)^-1 on two fields
            against cuFFT doing the same (torch.fft), 512^2 and 1024^2.
config_256_512 = the 256^2 / 512^2 random-field configuration at nt 4, 8, 16:
            GN matvecs/s, transport solves/s and gradients/s through the C ABI.
batch64 = 64 problems of uneven size, 5 batches per arm: the lockstep batch
            (one launch per transport step over all problems, one CUDA
            graph per matvec, FP64-accurate reductions, P_REG) against
            concurrent contexts, the same contexts one by one and the plain
            FP32 method one by one (P_REG), and concurrent contexts and the
            plain FP32 method with P_2L; the lockstep matvec of all 64
            problems timed alone against its algorithmic bytes.
learned_warm_start = the trained warm-start network (weights committed with
            the package) measured outside the timed region: cold versus warm
            time to ||g||rel 1e-2 on held-out pairs of the learned-warm-start
            configuration at 1024^2 (nt = 4, beta = 1e-2), and one
            warm-started solve of the phantom workload above.
"""

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Hessian matvecs/s & time-to-‖g‖rel 1e-2 at 1024² 2D; chosen form vs plain FP32"
UNIT = "matvecs/s"
N_GRID = 1024
NT = 8
BETAS = (1e-1, 1e-2, 1e-3)
GTOL = 1e-2
FALLBACK_HBM_GBS = 6800.0
CLASS_NAMES = ["fft_rows", "fft_cols", "prefilter", "departure", "gather",
               "adjoint_step", "incstate_step", "reduce", "vector", "matvec"]
# source file of each kernel class (a traffic figure is only valid for the
# source it was captured from)
CLASS_SOURCES = {"fft_rows": ("fft.cu",), "fft_cols": ("fft.cu",),
                 "prefilter": ("transport.cu", "interp.cuh"),
                 "departure": ("transport.cu", "interp.cuh"),
                 "gather": ("transport.cu", "interp.cuh"),
                 "adjoint_step": ("transport.cu", "interp.cuh"),
                 "incstate_step": ("transport.cu", "interp.cuh"),
                 "reduce": ("reduce.cu",), "vector": ("reduce.cu",),
                 "matvec": ("matvec.cu", "interp.cuh")}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--coarse-interp", choices=["lagrange", "spline"], default=None,
                    help="interpolation model of the P_2L coarse problem (default: cubic "
                         "Lagrange for phantom1024, the problems' spline for batch64)")
    ap.add_argument("--coarse-nt", type=int, default=-1,
                    help="time steps of the P_2L coarse problem (0: the problem's nt; default "
                         "-1: nt/2, the fine grid's displacement per step in coarse cells, for "
                         "phantom1024, and the problems' nt for batch64)")
    ap.add_argument("--hessian", choices=["gn", "full"], default="gn",
                    help="Gauss-Newton (the workload's) or full-Newton Hessian matvec")
    ap.add_argument("--incompressible", action="store_true",
                    help="the incompressible problem (div v = 0, K the Leray projection)")
    ap.add_argument("--graph-pdl", type=int, choices=[0, 1, 2], default=0,
                    help="programmatic edges inside the library's CUDA graphs: 0 none, 1 coarse "
                         "grid, 2 all")
    ap.add_argument("--beta-w", type=float, default=0.0,
                    help="near-incompressible problem: weight of ||div v||^2_H1 (0: off)")
    ap.add_argument("--no-plain-form", action="store_true",
                    help="skip the plain-form solve (FP32 reductions, no graphs)")
    ap.add_argument("--no-arms", action="store_true",
                    help="skip the coarse-solver arms (nested PCG, coarse problem at nt and splines)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the cuFFT comparator, the 256^2/512^2 measurements and the batch64 "
                         "comparison")
    ap.add_argument("--no-warm-start", action="store_true",
                    help="skip the learned warm-start measurement")
    ap.add_argument("--precond", choices=["2l-cheb", "2l-pcg", "reg"], default="2l-cheb",
                    help="preconditioner of the solve (the workload's is 2l-cheb)")
    ap.add_argument("--persistent", type=int, choices=[0, 1], default=0,
                    help="1: GN data term as one persistent cooperative kernel")
    ap.add_argument("--workload", choices=["phantom1024", "batch64"], default="phantom1024",
                    help="phantom1024: the 1024^2 continuation solve (default); batch64: "
                         "64 independent problems of uneven size")
    args = ap.parse_args()
    # batch64: the cheaper coarse problem raises matvecs per solve as much as
    # it lowers their cost there, so the batch keeps the problems' own model
    batch = args.workload == "batch64"
    if args.coarse_nt < 0:
        args.coarse_nt = 0 if batch else NT // 2
    if args.coarse_interp is None:
        args.coarse_interp = "spline" if batch else "lagrange"
    return args


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def source_hash(fnames):
    h = hashlib.sha256()
    for fname in fnames:
        h.update(open(os.path.join(ROOT, "paper_1604_02153_gb300", "csrc", fname), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(level, cls):
    """Per-launch DRAM traffic of a kernel class on a grid level from the
    committed ncu summary, or None if absent or captured from a different
    source."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(f"{level}/{cls}")
    if not e or e.get("source_sha256_16") != source_hash(CLASS_SOURCES[cls]):
        return None
    return e.get("dram_bytes_per_launch_full_size")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the raw samples go to the directory named by REGNK_CLOCKS_DIR (kept for
        # inspection), else to the system's temporary directory
        import tempfile
        d = os.environ.get("REGNK_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"clocks_bench_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# the oracle timed on the host (cpu_baseline and --impl reference)

def oracle_matvec_sample(incompressible=False, hessian="gn", beta_w=0.0):
    """Set up the 1024^2 workload in the FP64 oracle (untimed state solve at
    a smooth velocity) and return a callable doing one GN Hessian matvec."""
    from oracle.problem import Problem
    from paper_1604_02153_gb300 import inputs
    m_R, m_T = inputs.ellipse_phantoms(N_GRID, seed=100)
    P = Problem(m_R, m_T, NT, BETAS[-1], incompressible=incompressible, hessian=hessian,
                beta_w=beta_w)
    P.state_solve(inputs.random_velocity(N_GRID, seed=7, vmax=0.2))
    if hessian == "full":
        P.adjoint_solve()          # the full-Newton matvec needs the adjoint history
    P.ensure_adjoint_characteristic()
    vt = inputs.random_velocity(N_GRID, seed=8, vmax=1.0)
    return lambda: P.hessian_matvec(vt)


def _oracle_matvec_worker(args):
    """One oracle matvec in a worker process (set-up untimed); returns its
    start and end on the shared monotonic clock."""
    incompressible, hessian, beta_w = args
    f = oracle_matvec_sample(incompressible, hessian, beta_w)
    t0 = time.perf_counter()
    f()
    return t0, time.perf_counter()


def host_cpu():
    """Core count and model of the host that runs the oracle."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.TimeoutExpired):
        pass
    return {"nproc": os.cpu_count(), "model": model}


def oracle_c1_solve():
    """The 64^2 plain-method configuration solved by the oracle (P_2L CHEB(10),
    ||g||rel 1e-2): seconds and iterations, single-threaded."""
    from oracle.problem import Problem
    from oracle.solver import Solver
    from paper_1604_02153_gb300 import inputs
    n, nt, beta = 64, 4, 1e-2
    m_T, vstar = inputs.sinusoid_pair(n)
    m_R = Problem(np.zeros((n, n)), m_T, nt, beta).state_solve(vstar)
    t0 = time.perf_counter()
    S = Solver(Problem(m_R, m_T, nt, beta), precond="2L", pc_solver="cheb")
    _, info = S.solve(np.zeros((2, n, n)), GTOL)
    return {"seconds": time.perf_counter() - t0, "newton_iters": info["newton_iters"],
            "matvecs": info["matvecs"], "grid": [n, n], "nt": nt,
            "what": "FP64 oracle full solve of the 64^2 analytic problem, P_2L CHEB(10), "
                    "||g||rel 1e-2, one core"}


def cpu_baseline(incompressible=False, hessian="gn", beta_w=0.0, all_cores=True):
    """The oracle on the host: one GN matvec at 1024^2 on one core, then one
    independent matvec per core at once (process pool started with spawn),
    and the 64^2 oracle full solve."""
    f = oracle_matvec_sample(incompressible, hessian, beta_w)
    t0 = time.perf_counter()
    f()
    dt = time.perf_counter() - t0
    cpu = host_cpu()
    what = f"{'full-Newton' if hessian == 'full' else 'GN'} Hessian matvec"
    line = {"value": 1.0 / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"1 {what} of the FP64 numpy oracle at {N_GRID}^2, nt={NT} "
                      f"({dt:.1f} s, single-threaded numpy)",
            "host": cpu}
    if all_cores and (cpu["nproc"] or 1) > 1:
        import multiprocessing as mp
        k = int(cpu["nproc"])
        with mp.get_context("spawn").Pool(k) as pool:
            spans = pool.map(_oracle_matvec_worker, [(incompressible, hessian, beta_w)] * k)
        wall = max(e for _, e in spans) - min(s0 for s0, _ in spans)
        line["all_cores"] = {"value": k / wall, "unit": UNIT, "cores": k,
                             "sample": f"{k} independent {what}s at {N_GRID}^2, one per core "
                                       f"(process pool), {wall:.1f} s from the first start to "
                                       f"the last end"}
    line["c1_full_solve"] = oracle_c1_solve()
    return line


def run_reference(args, rank):
    if rank != 0:
        return
    f = oracle_matvec_sample(args.incompressible, args.hessian, args.beta_w)
    for _ in range(args.warmup):
        f()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f()
    dt = time.perf_counter() - t0
    value = args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.precond, args.coarse_nt, args.coarse_interp, args.incompressible,
                                  args.hessian, args.beta_w),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"one FP64 oracle GN Hessian matvec per step at "
                                       f"{N_GRID}^2, nt={NT}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(precond="2l-cheb", coarse_nt=0, coarse_interp="spline", incompressible=False,
                    hessian="gn", beta_w=0.0):
    pc = {"2l-cheb": "P_2L CHEB(10) 512^2 coarse", "2l-pcg": "P_2L PCG(1e-1) 512^2 coarse",
          "reg": "P_REG"}[precond]
    if coarse_nt and precond != "reg":
        pc += f" nt={coarse_nt}"
    if coarse_interp == "lagrange" and precond != "reg":
        pc += " cubic-Lagrange"
    return {"workload": f"phantom pair {N_GRID}x{N_GRID} (12 random ellipses, sigma 2 px), "
                        f"nt={NT}, H1, beta 1e-1->1e-2->1e-3, {pc}, "
                        f"||g||rel 1e-2, cubic B-spline SL"
                        + (", incompressible (K = Leray projection)" if incompressible else "")
                        + (f", near-incompressible (beta_w = {beta_w:g})" if beta_w > 0 else "")
                        + (", full-Newton Hessian" if hessian == "full" else ""),
            "grid": [N_GRID, N_GRID], "nt": NT, "betas": list(BETAS), "gtol": GTOL,
            "precond": pc, "interp": "spline", "reg_norm": "H1",
            "incompressible": bool(incompressible), "beta_w": float(beta_w),
            "hessian": {"gn": "Gauss-Newton", "full": "full Newton"}[hessian],
            "l2": "flushed between steps (256 MB write, untimed)"}


# ---------------------------------------------------------------------------
# measurements beside the headline (outside the timed region, rank 0)

def _median_ms(fn, reps=7, inner=20, warm=5):
    """Median over `reps` of the device time of `inner` back-to-back calls,
    divided by `inner` (CUDA events on the current stream; warm caches)."""
    import torch
    st = torch.cuda.current_stream()
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(inner):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) / inner)
    return float(np.median(ts))


def _graph_ms(fn, inner=20, reps=7):
    """Device time per call of fn: `inner` calls captured in one CUDA graph
    (no host launch overhead in the timing), replayed `reps` times between
    CUDA events; median. Falls back to eager calls if capture fails."""
    import torch
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(3):
            fn()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    try:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for _ in range(inner):
                fn()
    except RuntimeError:
        return _median_ms(fn, reps=reps, inner=inner), "eager"
    st = torch.cuda.current_stream()
    g.replay()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        g.replay()
        e1.record(st)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) / inner)
    return float(np.median(ts)), "graph"


def fft_comparator(dev, hbm, sizes=(512, 1024), beta=1e-2):
    """The hand-written spectral operator (beta A)^-1 v on a vector field (a
    row R2C pass, the column pass with the multiplier, a row C2R pass) timed
    beside cuFFT doing the same operator (torch.fft.rfft2, multiply by the
    same symbol, torch.fft.irfft2); both results are compared. Each side runs
    20 calls captured in one CUDA graph, so host launch overhead is not
    timed. GB/s counts the operator's algorithmic bytes: both components read
    and written once (16 B per grid point)."""
    import torch
    from paper_1604_02153_gb300 import inputs, regnk
    rows = []
    for n in sizes:
        R = regnk.Registration(n, n, 4, beta, precond=regnk.REG_PC_REG)
        v = torch.tensor(inputs.random_velocity(n, seed=9, kmax=n // 4, vmax=1.0)
                         .astype(np.float32).ravel(), device=dev)
        ours = torch.empty_like(v)
        k1 = torch.fft.rfftfreq(n, d=1.0 / n, device=dev).to(torch.float64)
        k2 = torch.fft.fftfreq(n, d=1.0 / n, device=dev).to(torch.float64)
        gam = k2[:, None] ** 2 + k1[None, :] ** 2
        gam[0, 0] = 1.0                     # the k = 0 weight of (beta A)^s is 1
        sym = (1.0 / (beta * gam)).to(torch.float32)
        V = v.view(2, n, n)
        theirs = torch.empty(2, n, n, device=dev)

        def run_ours():
            R.spectral(regnk.REG_SPEC_REGPOW, v, ours, -1.0)

        def run_cufft():
            torch.fft.irfft2(torch.fft.rfft2(V) * sym, s=(n, n), out=theirs)

        t_ours, mode_o = _graph_ms(run_ours)
        t_cu, mode_c = _graph_ms(run_cufft)
        run_ours()
        run_cufft()
        torch.cuda.synchronize()
        agree = float(torch.linalg.norm(ours.view(2, n, n) - theirs) / torch.linalg.norm(theirs))
        by = 16.0 * n * n
        rows.append({"grid": [n, n], "operator": "(beta A)^-1 on 2 fields",
                     "ours_us": 1e3 * t_ours, "cufft_us": 1e3 * t_cu, "timing": [mode_o, mode_c],
                     "ours_gbs": by / (t_ours / 1e3) / 1e9, "cufft_gbs": by / (t_cu / 1e3) / 1e9,
                     "ours_frac": by / (t_ours / 1e3) / 1e9 / hbm,
                     "speedup_vs_cufft": t_cu / t_ours, "rel_diff": agree})
        R.close()
    return {"what": "hand-written FFT + multiplier (3 kernels) vs cuFFT R2C -> multiply -> C2R "
                    "(torch.fft), 20 calls per CUDA graph, median of 7 replays, warm caches",
            "rows": rows}


def measurement_c2(dev, hbm, l2_bytes):
    """The 256^2 / 512^2 random-field configuration at nt = 4, 8, 16: GN
    Hessian matvecs/s, state transport solves/s and objective+gradient
    evaluations (state + adjoint) per second through the C ABI, CUDA events,
    with the algorithmic bytes of each unit and whether the matvec's working
    set fits the L2 cache (then the HBM fraction does not bound it)."""
    import torch
    from paper_1604_02153_gb300 import inputs, regnk
    f = lambda a: torch.tensor(np.ascontiguousarray(a, dtype=np.float32).ravel(), device=dev)
    out = []
    for n in (256, 512):
        m_T = inputs.random_field(n, seed=1, kmax=16)
        vstar = inputs.random_velocity(n, seed=3, kmax=4, vmax=0.2)
        for nt in (4, 8, 16):
            R = regnk.Registration(n, n, nt, 1e-2)
            m_T_d, v_d = f(m_T), f(vstar)
            m_R_d = torch.empty(n * n, device=dev)
            R.transport(v_d, m_T_d, m_R_d)
            R.set_images(m_R_d, m_T_d)
            u = f(inputs.random_velocity(n, seed=8, vmax=1.0))
            H = torch.empty_like(u)
            g = torch.empty_like(u)
            R.objective_gradient(v_d, g)
            m1 = torch.empty(n * n, device=dev)
            N = n * n
            t_mv = _median_ms(lambda: R.hessian_matvec(v_d, u, H))
            t_tr = _median_ms(lambda: R.transport(v_d, m_T_d, m1))
            # a new velocity every call (alternating), so the state solve is redone
            va, vb = v_d, v_d * (1.0 + 1e-3)
            flip = [0]

            def grad():
                flip[0] ^= 1
                R.objective_gradient(va if flip[0] else vb, g)
            t_gr = _median_ms(grad, reps=5, inner=10)
            b_mv = 4.0 * N * (10 * nt + 16)                 # GN matvec, stored grad m_j
            b_tr = 4.0 * N * (2 * nt + 4)                   # state transport solve
            b_gr = 4.0 * N * (2 * nt + 4 * nt + 2 * (nt + 1) + 16)
            # fields a matvec touches: dX, dY, v~, v~(X_D), div v, div v(Y_D),
            # b~, two transported fields (14 N), G_1..G_nt and grad m_0..grad m_nt
            ws = 4.0 * N * (16 + 4 * nt)
            row = {"grid": [n, n], "nt": nt,
                   "matvecs_per_s": 1e3 / t_mv, "transport_solves_per_s": 1e3 / t_tr,
                   "gradients_per_s": 1e3 / t_gr,
                   "matvec_us": 1e3 * t_mv, "matvec_algorithmic_bytes": b_mv,
                   "roofline_matvec": {"achieved": b_mv / (t_mv / 1e3) / 1e9, "peak": hbm,
                                       "unit": "GB/s",
                                       "frac": b_mv / (t_mv / 1e3) / 1e9 / hbm,
                                       "l2_resident": bool(ws < l2_bytes)},
                   "roofline_transport": {"achieved": b_tr / (t_tr / 1e3) / 1e9,
                                          "frac": b_tr / (t_tr / 1e3) / 1e9 / hbm},
                   "roofline_gradient": {"achieved": b_gr / (t_gr / 1e3) / 1e9,
                                         "frac": b_gr / (t_gr / 1e3) / 1e9 / hbm}}
            out.append(row)
            R.close()
    return {"what": "random-field pairs (m_T k <= 16, v* k <= 4, max |v| 0.2, m_R = m_T "
                    "transported by v*), beta 1e-2, spline SL, eager calls through the C ABI, "
                    "median of CUDA-event timings; algorithmic bytes per unit: matvec "
                    "4N(10nt+16), transport solve 4N(2nt+4), gradient 4N(8nt+18)",
            "rows": out}


def d3_bytes_per_point(nt, lagrange=False):
    """Algorithmic bytes per grid point of one 3D GN matvec, summed over its
    kernels (each kernel's inputs read once, outputs written once): the
    prefilter of v~ (3 fields x 3 axis passes x 8 B), the first incremental
    state step (76 B), nt - 1 more with their prefilters (68 + 24 B),
    lambda~_nt with the first term of b~ (32 B), nt adjoint steps with their
    prefilters (64 + 24 B), and beta A v~ + b~ on two packed complex fields
    (pack 28 B, six FFT passes 192 B, multiply 32 B, unpack and add 40 B).
    Cubic Lagrange has no prefilter passes."""
    pre = 0 if lagrange else 24
    return 3 * pre + 76 + (nt - 1) * (68 + pre) + 32 + nt * (64 + pre) + 292


def measurement_3d(dev, hbm, sizes=(128, 256), nt=4):
    """The 3D path (row f4): GN matvec, J + gradient at a new velocity (state
    solve included) and state transport at n^3 through the C ABI (CUDA
    events, median), the matvec's roofline in the algorithmic bytes of its
    kernels, and one Newton-Krylov solve at the smallest size."""
    import torch
    from paper_1604_02153_gb300 import inputs, regnk
    f = lambda a: torch.tensor(np.ascontiguousarray(a, dtype=np.float32).ravel(), device=dev)
    rows = []
    for n in sizes:
        for lagrange in ((False, True) if n == max(sizes) else (False,)):
            m_T = f(inputs.random_field3(n, n, n, seed=9, kmax=4))
            vstar = f(inputs.random_velocity3(n, n, n, seed=10, kmax=3, vmax=0.3))
            u = f(inputs.random_velocity3(n, n, n, seed=8, kmax=3, vmax=1.0))
            R = regnk.Registration3(n, n, n, nt, 1e-2, interp=regnk.REG_INTERP_LAGRANGE
                                    if lagrange else regnk.REG_INTERP_SPLINE)
            m_R = torch.empty_like(m_T)
            R.transport(vstar, m_T, m_R)
            R.set_images(m_R, m_T)
            v = 0.5 * vstar
            g = torch.empty_like(v)
            H = torch.empty_like(v)
            m1 = torch.empty_like(m_T)
            R.objective_gradient(v, g)
            t_mv = _median_ms(lambda: R.hessian_matvec(v, u, H), reps=5, inner=10, warm=3)
            va, vb = v, v * (1.0 + 1e-3)
            flip = [0]

            def grad():
                flip[0] ^= 1
                R.objective_gradient(va if flip[0] else vb, g)
            t_gr = _median_ms(grad, reps=5, inner=4, warm=2)
            t_tr = _median_ms(lambda: R.transport(v, m_T, m1), reps=5, inner=10, warm=3)
            N = n ** 3
            b_mv = float(N) * d3_bytes_per_point(nt, lagrange)
            row = {"grid": [n, n, n], "nt": nt, "interp": "lagrange" if lagrange else "spline",
                   "matvec_ms": t_mv, "gradient_at_new_velocity_ms": t_gr, "transport_ms": t_tr,
                   "matvec_algorithmic_bytes": b_mv,
                   "roofline_matvec": {"achieved": b_mv / (t_mv / 1e3) / 1e9, "peak": hbm,
                                       "unit": "GB/s", "frac": b_mv / (t_mv / 1e3) / 1e9 / hbm}}
            if n == min(sizes) and not lagrange:
                row["solve"] = {}
                for name, Rs in (("P_REG", R), ("P_2L", None)):
                    if Rs is None:   # the two-level preconditioner, CHEB(10)
                        Rs = regnk.Registration3(n, n, n, nt, 1e-2, precond=regnk.REG_PC_2L)
                        Rs.set_images(m_R, m_T)
                    x = torch.zeros_like(v)
                    torch.cuda.synchronize()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                    info = Rs.solve(x, 1e-2)
                    e1.record()
                    torch.cuda.synchronize()
                    row["solve"][name] = {"gtol": 1e-2, "beta": 1e-2,
                                          "seconds": e0.elapsed_time(e1) / 1e3,
                                          "newton_iters": info["newton_iters"],
                                          "pcg_iters": info["pcg_iters"],
                                          "matvecs": info["matvecs"],
                                          "coarse_matvecs": info["coarse_matvecs"],
                                          "gnorm_rel": info["gnorm_rel"]}
                    if Rs is not R:
                        Rs.close()
            rows.append(row)
            R.close()
            del m_T, vstar, u, m_R, v, g, H, m1
    return {"what": "3D random-field pair (m_T k <= 4, v* k <= 3, max |v*| 0.3, m_R = m_T "
                    "transported by v*), evaluated at v = v*/2, beta 1e-2, P_REG, CUDA events "
                    "(median); matvec bytes per point summed over its kernels "
                    "(380 + 180 nt with splines)", "rows": rows}


def aggregate_ranks(dist, device, total_ms, matvecs, e2e_ms, e2e_matvecs):
    """Whole-job figures over replicas: time = max over ranks, work = sum.

    Returns (value, e2e_value) in matvecs/s. dist may be None (one rank).
    """
    if dist is None:
        return matvecs / (total_ms / 1e3), e2e_matvecs / (e2e_ms / 1e3)
    import torch
    t = torch.tensor([total_ms, e2e_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    w = torch.tensor([float(matvecs), float(e2e_matvecs)], dtype=torch.float64, device=device)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(w[0]) / (float(t[0]) / 1e3), float(w[1]) / (float(t[1]) / 1e3)


BATCH_SIZES = (128, 192, 256, 384, 512)
BATCH_B = 64
BATCH_NT = 4
BATCH_BETA = 1e-2


def batch_comparison(args, samples, warmup):
    """64 independent problems, grids drawn (seed 200) from BATCH_SIZES^2,
    each the analytic template/velocity pair with m_R = m_T transported by
    v* (nt = 4, computed on the GPU), H1, beta = 1e-2, solved to ||g||rel
    1e-2 from v = 0. Arms with the spectral preconditioner P_REG:
    lockstep (reg_lockstep: one launch per transport step over all 64
    problems, one CUDA graph for the matvec, FP64-accurate reductions),
    concurrent contexts (reg_batch: one context and stream per problem,
    CUDA graphs, FP64-accurate reductions), the same contexts one by one,
    and the plain FP32 method one by one (FP32 reductions, no CUDA graphs,
    plain launches). Arms with P_2L-CHEB(10) (coarse problem as --coarse-nt
    / --coarse-interp): concurrent contexts and plain FP32 one by one. Wall
    time per batch between device synchronisations, `samples` batches per
    arm after `warmup`. The lockstep matvec of all 64 problems is also
    timed alone (graph replays, CUDA events) against its algorithmic bytes
    sum_p 4 N_p (10 nt + 16)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1604_02153_gb300 import inputs, regnk
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(200)
    sizes = [int(x) for x in rng.choice(BATCH_SIZES, size=BATCH_B)]
    f = lambda a: torch.tensor(np.ascontiguousarray(a, dtype=np.float32).ravel(), device=dev)
    mR, mT = [], []
    cache = {}
    for n in sizes:
        if n not in cache:
            m_T, vstar = inputs.sinusoid_pair(n)
            R = regnk.Registration(n, n, BATCH_NT, BATCH_BETA)
            m1 = torch.empty(n * n, device=dev)
            R.transport(f(vstar), f(m_T), m1)
            torch.cuda.synchronize()
            R.close()
            cache[n] = (m1.clone(), f(m_T))
        mR.append(cache[n][0])
        mT.append(cache[n][1])
    grids = [(n, n) for n in sizes]
    betas = [BATCH_BETA] * BATCH_B
    ci = {"lagrange": regnk.REG_INTERP_LAGRANGE, "spline": regnk.REG_INTERP_SPLINE}[args.coarse_interp]
    vs = [torch.zeros(2 * n * n, device=dev) for n in sizes]

    def arm(solve):
        for _ in range(max(1, warmup)):
            for v in vs:
                v.zero_()
            solve()
        torch.cuda.synchronize()
        times, mv, infos = [], 0, None
        for _ in range(samples):
            for v in vs:
                v.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            infos = solve()
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
            mv += sum(i["matvecs"] for i in infos)
        return times, mv, infos

    def stats(t, mv, infos, per_problem):
        d = {"samples": len(t), "seconds_per_batch_mean": float(np.mean(t)),
             "seconds_per_batch_min": float(np.min(t)), "seconds_per_batch_std": float(np.std(t)),
             "matvecs_per_s": mv / sum(t), "matvecs_per_batch": mv // len(t),
             "newton_iters": int(sum(i["newton_iters"] for i in infos)),
             "status": sorted(set(i["status_name"] for i in infos))}
        if per_problem:
            d["mean_time_to_solution_s"] = float(np.mean([i["seconds"] for i in infos]))
        return d

    reg = dict(precond=regnk.REG_PC_REG)
    plain = dict(precision=regnk.REG_PRECISION_FP32, use_graphs=0, programmatic_launch=0)
    out = {}
    L = regnk.Lockstep(grids, BATCH_NT, betas)
    L.set_images(mR, mT)
    r = arm(lambda: L.solve(vs, GTOL))
    out["lockstep_reg"] = dict(stats(*r, per_problem=False), kernels_per_matvec=L.info()["matvec_graph_kernels"])
    v_lock = [v.clone() for v in vs]
    # the batched matvec alone at the solutions, against its algorithmic bytes
    us = [f(inputs.random_velocity(n, seed=40 + i, vmax=0.2)) for i, n in enumerate(sizes)]
    Hs = [torch.empty(2 * n * n, device=dev) for n in sizes]
    L.hessian_matvec(v_lock, us, Hs)
    L.hessian_matvec(v_lock, us, Hs)
    ms = min(L.matvec_time(20) for _ in range(3))
    algo = float(sum(4.0 * n * n * (10 * BATCH_NT + 16) for n in sizes))
    peak, peak_kind = peaks()
    out["lockstep_matvec"] = {"ms": ms, "algorithmic_bytes": algo, "achieved_gbs": algo / ms / 1e6,
                              "peak_gbs": peak, "peak_kind": peak_kind,
                              "frac": algo / ms / 1e6 / peak,
                              "points": L.info()["points"], "tiles": L.info()["tiles"],
                              "unit": "one GN matvec of all 64 problems (graph replay, CUDA events, "
                                      "best of 3 means of 20)"}
    L.close()
    B = regnk.Batch(grids, BATCH_NT, betas, **reg)
    B.set_images(mR, mT)
    out["contexts_reg"] = stats(*arm(lambda: B.solve(vs, GTOL, threads=0)), per_problem=True)
    out["one_by_one_reg"] = stats(*arm(lambda: B.solve(vs, GTOL, threads=1)), per_problem=True)
    same = all(torch.equal(a, b) for a, b in zip(vs, v_lock))
    B.close()
    P = regnk.Batch(grids, BATCH_NT, betas, **reg, **plain)
    P.set_images(mR, mT)
    out["plain_fp32_reg"] = dict(stats(*arm(lambda: P.solve(vs, GTOL, threads=1)), per_problem=True),
                                 options="P_REG one by one, FP32 reductions, no CUDA graphs, plain launches")
    P.close()
    B2 = regnk.Batch(grids, BATCH_NT, betas, coarse_nt=args.coarse_nt, coarse_interp=ci)
    B2.set_images(mR, mT)
    out["contexts_2l"] = stats(*arm(lambda: B2.solve(vs, GTOL, threads=0)), per_problem=True)
    B2.close()
    P2 = regnk.Batch(grids, BATCH_NT, betas, coarse_nt=args.coarse_nt, coarse_interp=ci, **plain)
    P2.set_images(mR, mT)
    out["plain_fp32_2l"] = dict(stats(*arm(lambda: P2.solve(vs, GTOL, threads=1)), per_problem=True),
                                options="P_2L one by one, FP32 reductions, no CUDA graphs, plain launches")
    P2.close()
    t = {k: out[k]["seconds_per_batch_mean"] for k in out if "seconds_per_batch_mean" in out[k]}
    return {"workload": f"{BATCH_B} problems, grids from {list(BATCH_SIZES)}^2 (seed 200), analytic "
                        f"pair, nt={BATCH_NT}, H1, beta={BATCH_BETA}, ||g||rel 1e-2; P_REG arms and "
                        f"P_2L CHEB(10) arms (coarse nt={args.coarse_nt or BATCH_NT} {args.coarse_interp})",
            "sizes": sizes, **out,
            "lockstep_equals_one_by_one_bitwise": bool(same),
            "speedup_lockstep_vs_one_by_one_reg": t["one_by_one_reg"] / t["lockstep_reg"],
            "speedup_lockstep_vs_contexts_reg": t["contexts_reg"] / t["lockstep_reg"],
            "speedup_lockstep_vs_plain_fp32_reg": t["plain_fp32_reg"] / t["lockstep_reg"],
            "speedup_lockstep_vs_plain_fp32_2l": t["plain_fp32_2l"] / t["lockstep_reg"],
            "speedup_lockstep_vs_contexts_2l": t["contexts_2l"] / t["lockstep_reg"],
            "learned_warm_start": "not applied: the network's input grid is 256^2 and it was "
                                  "trained on random-field pairs; the batch's analytic problems "
                                  "converge from v = 0 in a few Newton steps"}


def run_batch(args):
    """The batch workload as its own bench line (--workload batch64)."""
    c = batch_comparison(args, max(1, args.steps), args.warmup)
    line = {"metric": "aggregate Hessian matvecs/s, 64 independent problems of uneven size "
                      "(lockstep batch, P_REG)",
            "value": c["lockstep_reg"]["matvecs_per_s"], "unit": "matvecs/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * c["lockstep_reg"]["seconds_per_batch_mean"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": c["workload"], "sizes": c["sizes"]},
            "comparison": c}
    print(json.dumps(line), flush=True)


def learned_warm_start(R, v, ok, dev, pairs=4):
    """Cold versus warm start (see the module doc). Each solve is timed alone
    between device synchronisations and starts on freshly set images, so both
    pay for the reference gradient at v = 0."""
    import torch
    from paper_1604_02153_gb300 import regnk, warmstart
    theta, record = warmstart.load_params()
    net = regnk.UNet(warmstart.S, 1)
    net.set_params(theta)
    n = 4 * warmstart.S
    seeds = np.arange(warmstart.HELD_OUT_SEED0, warmstart.HELD_OUT_SEED0 + pairs)
    mR, mT, _ = warmstart.make_pairs(n, seeds, procs=1)
    Rh = regnk.Registration(n, n, warmstart.NT, warmstart.BETA)
    vh = torch.empty(2 * n * n, device=dev)
    rows = {"cold": [], "warm": []}
    accepted = 0
    for i in range(pairs):
        for mode in ("cold", "warm", "cold", "warm"):     # second pass is measured
            Rh.set_images(mR[i], mT[i])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if mode == "warm":
                acc = Rh.warm_start(net, vh)
            else:
                vh.zero_()
            info = Rh.solve(vh, warmstart.GTOL, allow=ok)
            torch.cuda.synchronize()
            rows[mode].append((time.perf_counter() - t0, info["newton_iters"], info["matvecs"]))
        accepted += int(acc)
    Rh.close()
    held = {"pairs": pairs, "grid": [n, n], "nt": warmstart.NT, "beta": warmstart.BETA,
            "warm_start_accepted": accepted}
    for mode in ("cold", "warm"):
        r = np.array(rows[mode][1::2])
        held[mode] = {"time_to_solution_s": float(r[:, 0].mean()),
                      "newton_iters": float(r[:, 1].mean()), "matvecs": float(r[:, 2].mean())}
    held["speedup_wall"] = held["cold"]["time_to_solution_s"] / held["warm"]["time_to_solution_s"]
    # the phantom workload, warm started at the first beta
    stats = {"matvecs": 0, "newton": 0}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    acc = False
    for b in BETAS:
        R.set_beta(b)
        if b == BETAS[0]:
            acc = R.warm_start(net, v)
        info = R.solve(v, GTOL, allow=ok)
        stats["matvecs"] += info["matvecs"]
        stats["newton"] += info["newton_iters"]
    torch.cuda.synchronize()
    ph = {"warm_start_accepted": bool(acc), "time_to_solution_s": time.perf_counter() - t0,
          "newton_iters_per_solve": stats["newton"], "matvecs_per_solve": stats["matvecs"]}
    net.close()
    return {"network": "U-Net 4 levels, 32 base channels, BF16 (weights/unet256.npz)",
            "training": {k: record[k] for k in ("pairs", "epochs", "batch", "seconds_training",
                                                "train_steps_per_second")},
            "final_training_loss": record["loss_per_epoch"][-1],
            "heldout_1024": held, "phantom1024": ph}


def main():
    args = parse()
    rank, local_rank, world = dist_env()
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.workload == "batch64":
        if rank == 0:
            run_batch(args)
        return
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if dist is not None:
        dist.barrier()
    from paper_1604_02153_gb300 import inputs, regnk
    regnk.load()

    n = N_GRID
    m_R, m_T = inputs.ellipse_phantoms(n, seed=100 + rank)
    h_mR = torch.tensor(m_R.astype(np.float32).ravel()).pin_memory()
    h_mT = torch.tensor(m_T.astype(np.float32).ravel()).pin_memory()
    d_mR, d_mT = h_mR.to(dev), h_mT.to(dev)
    pc_opts = {"2l-cheb": dict(precond=regnk.REG_PC_2L, pc_solver=regnk.REG_PCSOLVER_CHEB),
               "2l-pcg": dict(precond=regnk.REG_PC_2L, pc_solver=regnk.REG_PCSOLVER_PCG),
               "reg": dict(precond=regnk.REG_PC_REG)}[args.precond]
    R = regnk.Registration(n, n, NT, BETAS[0], persistent_matvec=args.persistent,
                           incompressible=int(args.incompressible), beta_w=args.beta_w,
                           graph_pdl=args.graph_pdl,
                           hessian={"gn": regnk.REG_HESSIAN_GN, "full": regnk.REG_HESSIAN_FULL}[args.hessian],
                           coarse_nt=args.coarse_nt,
                           coarse_interp={"lagrange": regnk.REG_INTERP_LAGRANGE,
                                          "spline": regnk.REG_INTERP_SPLINE}[args.coarse_interp],
                           **pc_opts)
    R.set_images(d_mR, d_mT)
    v = torch.zeros(2 * n * n, device=dev)
    h_v = torch.empty(2 * n * n).pin_memory()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    ok = (regnk.REG_OK, regnk.REG_ENOTCONV, regnk.REG_ELINESEARCH)

    def step(stats):
        v.zero_()
        for b in BETAS:
            R.set_beta(b)
            info = R.solve(v, GTOL, allow=ok)
            stats["matvecs"] += info["matvecs"]
            stats["newton"] += info["newton_iters"]
            stats["pcg"] += info["pcg_iters"]
            stats["coarse_matvecs"] += info["coarse_matvecs"]
            stats["status"].append(info["status_name"])
            stats["gnorm_rel"] = info["gnorm_rel"]

    def new_stats():
        return {"matvecs": 0, "newton": 0, "pcg": 0, "coarse_matvecs": 0, "status": [],
                "gnorm_rel": None}

    for _ in range(args.warmup):
        step(new_stats())
    torch.cuda.synchronize()

    # ---- timed region: K solves, inputs resident, L2 flushed between steps
    stats = new_stats()
    launches0 = regnk.launch_count()
    st = torch.cuda.current_stream()
    step_ms = []
    with ClockSampler(dev.index) as clocks:
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            step(stats)
            e1.record(st)
            torch.cuda.synchronize()
            step_ms.append(e0.elapsed_time(e1))
        if dist is not None:
            dist.barrier()
    launches = regnk.launch_count() - launches0
    total_ms = float(sum(step_ms))

    # ---- the same K solves again with per-kernel-class CUDA events (inside
    # the replayed graphs each kernel is bracketed by event nodes)
    R.profile_enable(True)
    for _ in range(args.steps):
        flush.fill_(1.0)
        step(new_stats())
    prof = R.profile_read()
    R.profile_enable(False)

    # ---- end to end through the C ABI with host buffers
    e2e_ms = 0.0
    e2e_mv = 0
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d_mR.copy_(h_mR, non_blocking=True)
        d_mT.copy_(h_mT, non_blocking=True)
        R.set_images(d_mR, d_mT)
        s2 = new_stats()
        step(s2)
        h_v.copy_(v, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms += 1e3 * (time.perf_counter() - t0)
        e2e_mv += s2["matvecs"]
    value, e2e_value = aggregate_ranks(dist, dev, total_ms, stats["matvecs"], e2e_ms, e2e_mv)

    def solve_samples(K, **opts):
        """K timed solves (CUDA events) of the workload with other options,
        after one untimed solve; contexts are created and closed here."""
        base = dict(persistent_matvec=args.persistent, incompressible=int(args.incompressible),
                    beta_w=args.beta_w, graph_pdl=args.graph_pdl,
                    hessian={"gn": regnk.REG_HESSIAN_GN, "full": regnk.REG_HESSIAN_FULL}[args.hessian],
                    coarse_nt=args.coarse_nt,
                    coarse_interp={"lagrange": regnk.REG_INTERP_LAGRANGE,
                                   "spline": regnk.REG_INTERP_SPLINE}[args.coarse_interp])
        base.update(pc_opts)
        base.update(opts)
        nonlocal R
        Rx = regnk.Registration(n, n, NT, BETAS[0], **base)
        Rx.set_images(d_mR, d_mT)
        R, Rmain = Rx, R
        try:
            step(new_stats())
            times, sp = [], new_stats()
            for _ in range(K):
                flush.fill_(1.0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(st)
                step(sp)
                e1.record(st)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1) / 1e3)
        finally:
            R = Rmain
            Rx.close()
        return {"samples": K, "time_to_solution_s": float(np.mean(times)),
                "time_to_solution_min_s": float(np.min(times)),
                "time_to_solution_std_s": float(np.std(times)),
                "matvecs_per_solve": sp["matvecs"] / K, "newton_iters_per_solve": sp["newton"] / K,
                "coarse_matvecs_per_solve": sp["coarse_matvecs"] / K,
                "solve_status": sorted(set(sp["status"])), "final_gnorm_rel": sp["gnorm_rel"]}

    # ---- the plain form of the same solve: FP32 reductions, no CUDA graphs,
    # plain launches, one launch per transport step (cold start, as above),
    # as many timed solves as the chosen form
    plain = None
    arms = None
    if not args.no_plain_form and rank == 0:
        plain = solve_samples(args.steps, precision=regnk.REG_PRECISION_FP32, use_graphs=0,
                              programmatic_launch=0, flow_matvec=0)
        plain["options"] = ("FP32 reductions, no CUDA graphs, plain launches, per-step transport "
                            "kernels, cold start")
        plain["speedup_of_chosen_form"] = plain["time_to_solution_s"] / (total_ms / args.steps / 1e3)
    if not args.no_arms and rank == 0 and args.precond == "2l-cheb":
        # the coarse solver of P_2L: nested PCG(0.1 eta) against CHEB(10), and
        # the coarse problem at the problem's nt and model (the library default)
        arms = {"pcg_coarse": solve_samples(2, pc_solver=regnk.REG_PCSOLVER_PCG),
                "coarse_problem_nt_and_spline": solve_samples(2, coarse_nt=0,
                                                              coarse_interp=regnk.REG_INTERP_SPLINE)}
        arms["pcg_coarse"]["what"] = "P_2L with nested PCG(0.1 eta) on the coarse grid"
        arms["coarse_problem_nt_and_spline"]["what"] = (
            "P_2L CHEB(10) with the coarse problem at nt = 8 and splines (library default)")

    # ---- the fine GN Hessian matvec as one unit: CUDA events around the
    # library call at the final velocity (replayed from its CUDA graph),
    # against its algorithmic bytes 4 N (10 nt + 16) (every field read or
    # written once; grad m_j stored, X_D, Y_D, div v computed once per velocity)
    u_dir = torch.tensor(inputs.random_velocity(n, seed=8, vmax=1.0).astype(np.float32).ravel(), device=dev)
    Hu = torch.empty_like(u_dir)
    for _ in range(3):
        R.hessian_matvec(v, u_dir, Hu)
    torch.cuda.synchronize()
    mv_ms = []
    for _ in range(20):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        R.hessian_matvec(v, u_dir, Hu)
        e1.record(st)
        torch.cuda.synchronize()
        mv_ms.append(e0.elapsed_time(e1))
    b_mv = 4.0 * n * n * (10 * NT + 16)

    # ---- roofline of the dominant kernel class (per grid level)
    dom = max(prof, key=lambda k: prof[k][0])
    ms, nl, by = prof[dom]
    hbm, how = peaks()
    achieved = (by / (ms / 1e3)) / 1e9 if ms > 0 else None
    per_launch = by / nl if nl else None
    total_prof_ms = sum(p[0] for p in prof.values())
    level, cls = dom
    # DRAM bytes per launch with warm caches from the committed ncu summary;
    # below the algorithmic bytes the class runs out of L2 (the 512^2 coarse
    # working set fits the 129 MB L2), so the HBM fraction understates it
    traffic = ncu_traffic(level, cls)
    roof = {"bound": "hbm", "kernel_class": cls, "grid_level": level,
            "grid": [n, n] if level == "fine" else [n // 2, n // 2],
            "achieved": achieved, "peak": hbm,
            "peak_source": f"{how} HBM copy bandwidth", "unit": "GB/s",
            "frac": (achieved / hbm) if achieved else None,
            "traffic": traffic,
            "l2_resident": (traffic < per_launch) if (traffic is not None and per_launch) else None,
            "algorithmic_bytes_per_launch": per_launch, "launches": nl,
            "share_of_device_time": ms / total_prof_ms,
            "classes_ms": {f"{k[0]}/{k[1]}": round(p[0], 3) for k, p in prof.items() if p[1]}}
    t_mv = float(np.median(mv_ms)) / 1e3
    roof_mv = {"unit": "GN Hessian matvec at 1024^2, nt = 8 (fine grid, graph replay, CUDA events, "
                       "median of 20)",
               "time_us": 1e6 * t_mv, "algorithmic_bytes": b_mv,
               "achieved": b_mv / t_mv / 1e9, "peak": hbm, "unit_bw": "GB/s",
               "frac": b_mv / t_mv / 1e9 / hbm}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": workload_config(args.precond, args.coarse_nt, args.coarse_interp, args.incompressible,
                                  args.hessian, args.beta_w),
                "time_to_solution_s": total_ms / args.steps / 1e3,
                "newton_iters_per_solve": stats["newton"] / args.steps,
                "matvecs_per_solve": stats["matvecs"] / args.steps,
                "pcg_iters_per_solve": stats["pcg"] / args.steps,
                "coarse_matvecs_per_solve": stats["coarse_matvecs"] / args.steps,
                "final_gnorm_rel": stats["gnorm_rel"],
                "solve_status": sorted(set(stats["status"])),
                "e2e": {"value": e2e_value, "unit": UNIT,
                        "h2d_bytes_per_step": int(h_mR.numel() * 4 + h_mT.numel() * 4),
                        "d2h_bytes_per_step": int(h_v.numel() * 4)},
                "gpu_launches": int(launches),
                "roofline": roof,
                "roofline_gn_matvec": roof_mv,
                "step_tiles": {f"{lvl}/{ker}": list(t) for (lvl, ker), t in R.step_tiles().items()},
                "plain_form": plain,
                "solver_arms": arms,
                "clocks": clocks.summary()}
        if world == 1 and not args.no_extras:
            l2 = torch.cuda.get_device_properties(dev).L2_cache_size
            line["fft_comparator"] = fft_comparator(dev, hbm)
            line["config_256_512"] = measurement_c2(dev, hbm, l2)
            try:
                line["grids_3d"] = measurement_3d(dev, hbm)
            except Exception as exc:   # the 2D line stands without it
                line["grids_3d"] = {"error": f"{type(exc).__name__}: {exc}"}
            # the batch workload's own coarse model (the problems' nt and splines)
            bargs = argparse.Namespace(**vars(args))
            bargs.coarse_nt, bargs.coarse_interp = 0, "spline"
            line["batch64"] = batch_comparison(bargs, 5, 2)
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.incompressible, args.hessian, args.beta_w)
        if not args.no_warm_start:
            line["learned_warm_start"] = learned_warm_start(R, v, ok, dev)
        print(json.dumps(line), flush=True)
    R.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
