"""Training data, training and evaluation of the warm-start U-Net.

    python -m paper_1604_02153_gb300.warmstart train --pairs 20000 --epochs 20
    python -m paper_1604_02153_gb300.warmstart evaluate --held-out 512

Learned warm start (no counterpart in the paper): the network of
``reg_unet_*`` maps (m_R, m_T) on a 256^2 grid to a stationary velocity from
which the Gauss-Newton-Krylov solve starts; the solve runs to the same
gradient tolerance from there, and ``reg_warm_start`` keeps the network's
velocity only if it lowers the objective below J(0).

Data. Pair s (seed s) is built like the 256^2 configuration: m_T is the
band-limited random field ``inputs.random_field(256, seed=s, kmax=16)``,
v* the smooth random velocity ``inputs.random_velocity(256, seed=s + 10**6,
kmax=4, vmax=0.2)``, and m_R is m_T transported by v* (nt = 4, the library's
state solve). Training pairs use seeds 10000..29999, held-out pairs
30000..30511. Targets are the solver's velocities at beta = 1e-2 (H1, nt = 4,
P_2L with CHEB(10), ||g||rel <= 1e-2), computed by batched solves.

Training runs entirely in the library's kernels (forward, backward, Adam;
reg_unet_train_step) on minibatches drawn from device-resident arrays by
index. The parameters are saved as bfloat16 bits (the precision the network
computes in) in an .npz file with the training record.
"""

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

S = 256
NT = 4
BETA = 1e-2
GTOL = 1e-2
TRAIN_SEED0 = 10000
HELD_OUT_SEED0 = 30000
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "unet256.npz")

# (Cin, Cout) of the network's convolutions, in parameter order
SHAPES = [(2, 32), (32, 32), (32, 64), (64, 64), (64, 128), (128, 128), (128, 256), (256, 256),
          (384, 128), (128, 128), (192, 64), (64, 64), (96, 32), (32, 32), (32, 2)]


def _pair_fields(args):
    n, seed = args
    from paper_1604_02153_gb300 import inputs
    mT = inputs.random_field(n, seed=seed, kmax=16)
    vs = inputs.random_velocity(n, seed=seed + 10 ** 6, kmax=4, vmax=0.2)
    return mT.astype("float32"), vs.astype("float32")


def host_fields(n, seeds, procs):
    """(m_T, v*) for each seed, generated on `procs` host processes."""
    import numpy as np
    work = [(n, int(s)) for s in seeds]
    if procs > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(procs) as pool:
            out = pool.map(_pair_fields, work, chunksize=16)
    else:
        out = [_pair_fields(w) for w in work]
    return np.stack([o[0] for o in out]), np.stack([o[1] for o in out])


def make_pairs(n, seeds, procs=8, chunk=1024):
    """Device arrays m_R [P, n*n], m_T [P, n*n] and v* [P, 2*n*n] (float32),
    generated in chunks of `chunk` pairs."""
    import torch
    from paper_1604_02153_gb300 import regnk
    P = len(seeds)
    mT = torch.empty(P, n * n, device="cuda")
    vs = torch.empty(P, 2 * n * n, device="cuda")
    mR = torch.empty_like(mT)
    R = regnk.Registration(n, n, NT, BETA, precond=regnk.REG_PC_REG)
    for p0 in range(0, P, chunk):
        p1 = min(P, p0 + chunk)
        mT_h, vs_h = host_fields(n, seeds[p0:p1], procs)
        mT[p0:p1].copy_(torch.from_numpy(mT_h.reshape(p1 - p0, n * n)))
        vs[p0:p1].copy_(torch.from_numpy(vs_h.reshape(p1 - p0, 2 * n * n)))
        if p0 == 0:
            R.set_images(mT[0], mT[0])
        for i in range(p0, p1):
            R.transport(vs[i], mT[i], mR[i])
    torch.cuda.synchronize()
    R.close()
    return mR, mT, vs


def solve_targets(mR, mT, n, batch=64):
    """Solver velocities at beta = 1e-2 for every pair (batched solves)."""
    import torch
    from paper_1604_02153_gb300 import regnk
    P = mR.shape[0]
    v = torch.zeros(P, 2 * n * n, device="cuda")
    stats = []
    B = None
    for p0 in range(0, P, batch):
        p1 = min(P, p0 + batch)
        if B is None or B.B != p1 - p0:
            if B is not None:
                B.close()
            B = regnk.Batch([(n, n)] * (p1 - p0), NT, [BETA] * (p1 - p0))
        B.set_images([mR[i] for i in range(p0, p1)], [mT[i] for i in range(p0, p1)])
        stats += B.solve([v[i] for i in range(p0, p1)], GTOL)
    B.close()
    return v, stats


def train(args):
    import numpy as np
    import torch
    from paper_1604_02153_gb300 import inputs, regnk
    t0 = time.time()
    seeds = np.arange(TRAIN_SEED0, TRAIN_SEED0 + args.pairs)
    mR, mT, _ = make_pairs(S, seeds, args.procs)
    t_pairs = time.time() - t0
    v, stats = solve_targets(mR, mT, S)
    torch.cuda.synchronize()
    t_targets = time.time() - t0 - t_pairs
    conv = sum(1 for s in stats if s["status_name"] == "REG_OK")
    print(f"{args.pairs} pairs in {t_pairs:.1f} s, targets in {t_targets:.1f} s "
          f"({conv} converged, mean {np.mean([s['newton_iters'] for s in stats]):.2f} Newton iterations)",
          flush=True)
    net = regnk.UNet(S, args.batch)
    net.set_params(inputs.he_normal(SHAPES, seed=args.seed))
    P = mR.shape[0]
    steps_per_epoch = P // args.batch
    total = steps_per_epoch * args.epochs
    g = torch.Generator(device="cuda").manual_seed(args.seed)
    history = []
    step = 0
    t1 = time.time()
    for ep in range(args.epochs):
        perm = torch.randperm(P, device="cuda", generator=g).to(torch.int32)
        acc = 0.0
        for k in range(steps_per_epoch):
            lr = args.lr * 0.5 * (1.0 + np.cos(np.pi * step / total))    # cosine decay
            idx = perm[k * args.batch:(k + 1) * args.batch].contiguous()
            acc += net.train_step(args.batch, mR, mT, v, lr, idx=idx)
            step += 1
        history.append(acc / steps_per_epoch)
        print(f"epoch {ep + 1}/{args.epochs}: mean loss {history[-1]:.4e} "
              f"({time.time() - t1:.1f} s)", flush=True)
    t_train = time.time() - t1
    theta = net.get_params()
    bits = (theta.view(np.uint32).astype(np.uint64) + 0x7FFF + ((theta.view(np.uint32) >> 16) & 1)) >> 16
    record = {"pairs": int(P), "epochs": args.epochs, "batch": args.batch, "lr": args.lr,
              "seed": args.seed, "loss_per_epoch": history, "seconds_pairs": t_pairs,
              "seconds_targets": t_targets, "seconds_training": t_train,
              "train_steps_per_second": total / t_train,
              "target_newton_iters_mean": float(np.mean([s["newton_iters"] for s in stats])),
              "target_matvecs_mean": float(np.mean([s["matvecs"] for s in stats]))}
    os.makedirs(os.path.dirname(args.out), exist_ok=True)
    np.savez_compressed(args.out, params_bf16=bits.astype(np.uint16), record=json.dumps(record))
    print(json.dumps(record), flush=True)
    net.close()


def load_params(path=WEIGHTS):
    """Saved parameters as float32 (bfloat16 values) and the training record."""
    import numpy as np
    z = np.load(path)
    bits = z["params_bf16"].astype(np.uint32) << 16
    return bits.view(np.float32), json.loads(str(z["record"]))


def evaluate(args):
    """Cold versus warm start on held-out pairs: Newton iterations, matvecs and
    wall time to ||g||rel <= 1e-2 (each solve timed alone, synchronised).

    Both solves of a pair start on freshly set images, so both pay for the
    reference gradient at v = 0 that the relative tolerance needs; the warm
    time includes the warm start itself. One untimed cold and warm solve of
    the first pair comes first (CUDA graph captures)."""
    import numpy as np
    import torch
    from paper_1604_02153_gb300 import regnk
    theta, record = load_params(args.weights)
    net = regnk.UNet(S, 1)
    net.set_params(theta)
    results = {}
    for n, count in ((S, args.held_out), (4 * S, args.held_out_1024)):
        if count <= 0:
            continue
        seeds = np.arange(HELD_OUT_SEED0, HELD_OUT_SEED0 + count)
        mR, mT, _ = make_pairs(n, seeds, args.procs)
        R = regnk.Registration(n, n, NT, BETA)
        v = torch.empty(2 * n * n, device="cuda")
        rows = {"cold": [], "warm": []}
        kept = []
        for i in [0] + list(range(count)):
            for mode in ("cold", "warm"):
                R.set_images(mR[i], mT[i])
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                if mode == "warm":
                    kept.append(R.warm_start(net, v))
                else:
                    v.zero_()
                info = R.solve(v, GTOL, allow=(regnk.REG_OK, regnk.REG_ENOTCONV, regnk.REG_ELINESEARCH))
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                rows[mode].append((info["newton_iters"], info["matvecs"], dt,
                                   info["status_name"] == "REG_OK"))
        rows = {mode: r[1:] for mode, r in rows.items()}   # drop the untimed first pair
        accepted = int(sum(kept[1:]))
        R.close()
        summ = {}
        for mode, r in rows.items():
            a = np.array([x[:3] for x in r], dtype=np.float64)
            summ[mode] = {"newton_iters": float(a[:, 0].mean()), "matvecs": float(a[:, 1].mean()),
                          "seconds": float(a[:, 2].mean()),
                          "converged": int(sum(x[3] for x in r))}
        summ["pairs"] = int(count)
        summ["warm_start_accepted"] = accepted
        summ["speedup_wall"] = summ["cold"]["seconds"] / summ["warm"]["seconds"]
        results[f"{n}x{n}"] = summ
        print(f"{n}^2: {json.dumps(summ)}", flush=True)
    results["training"] = record
    if args.json:
        with open(args.json, "w") as f:
            json.dump(results, f, indent=1)
    net.close()
    return results


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--pairs", type=int, default=20000)
    t.add_argument("--epochs", type=int, default=20)
    t.add_argument("--batch", type=int, default=32)
    t.add_argument("--lr", type=float, default=1e-3)
    t.add_argument("--seed", type=int, default=1)
    t.add_argument("--procs", type=int, default=8)
    t.add_argument("--out", default=WEIGHTS)
    e = sub.add_parser("evaluate")
    e.add_argument("--weights", default=WEIGHTS)
    e.add_argument("--held-out", type=int, default=512)
    e.add_argument("--held-out-1024", type=int, default=8)
    e.add_argument("--procs", type=int, default=8)
    e.add_argument("--json", default=None)
    a = ap.parse_args()
    train(a) if a.cmd == "train" else evaluate(a)


if __name__ == "__main__":
    main()
