"""Semi-Lagrangian transport against the RK2A comparator on the GPU.

    python -m paper_1604_02153_gb300.compare_transport [--nref 1024] [--json out.json]

The trend of the paper's transport experiments (§4.1.1-4.1.2: SL at CFL
numbers 0.2, 1 and 5 against the stabilised RK2 scheme RK2A at 0.2) on
synthetic data standing in for SMOOTH A: m0 = inputs.random_field(nref,
seed=1, kmax=6) and v = inputs.random_velocity(nref, seed=3, kmax=3,
vmax=0.5), spectrally restricted to each grid n. Reference: RK2A(0.2) state
solve on the nref^2 grid (512^2, the paper's reference grid). For each n and
scheme: relative L2 distance of m(1), spectrally prolonged to nref, from the
reference (the error measure of the paper's tables, "rel_err"), the same on
the modes the n-grid resolves ("rel_err_band"), and the time of one solve
through the C ABI (CUDA events on the current stream, best of 3 after a
warm-up). "ref_out_of_band" is the reference's relative L2 norm outside
that band: in FP32 the non-dissipative RK2 steps amplify the roundoff of
the highest modes (Heun grows a purely imaginary eigenvalue z by
sqrt(1 + z^4/4) per step, z up to pi c), so this floor grows with nref and
the number of steps. The restriction, prolongation and errors use numpy's
FFT: evaluation only, not part of the solves.
"""

import argparse
import json
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def truncate(uh, n):
    """Fourier coefficients of an (N, N) field kept on an (n, n) grid
    (|k_i| < n/2, the coarse Nyquist dropped), in numpy's normalisation for
    the (n, n) inverse."""
    N = uh.shape[0]
    k = np.fft.fftfreq(N, 1.0 / N).astype(int)
    keep = np.abs(k) < n / 2
    idx = np.where(k < 0, k + n, k)[keep]
    out = np.zeros((n, n), dtype=complex)
    out[np.ix_(idx, idx)] = uh[np.ix_(keep, keep)]
    return out * (n * n) / (N * N)


def restrict(u, n):
    return np.real(np.fft.ifft2(truncate(np.fft.fft2(u), n)))


def prolong(u, N):
    n = u.shape[0]
    uh = np.fft.fft2(u)
    k = np.fft.fftfreq(n, 1.0 / n)
    out = np.zeros((N, N), dtype=complex)
    idx = np.where(k < 0, k + N, k).astype(int)
    keep = np.abs(k) < n / 2
    out[np.ix_(idx[keep], idx[keep])] = uh[np.ix_(keep, keep)]
    return np.real(np.fft.ifft2(out * (N * N) / (n * n)))


def cfl_steps(v, c):
    n = v.shape[-1]
    h = 2.0 * math.pi / n
    return max(1, math.ceil(float(np.max(np.abs(v))) / (c * h)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nref", type=int, default=512)
    ap.add_argument("--grids", type=int, nargs="+", default=[64, 128, 256])
    ap.add_argument("--json", default=None)
    a = ap.parse_args()
    import torch
    from paper_1604_02153_gb300 import inputs, regnk
    regnk.load()
    m0f = inputs.random_field(a.nref, seed=1, kmax=6)
    vf = inputs.random_velocity(a.nref, seed=3, kmax=3, vmax=0.5)
    dev = lambda x: torch.tensor(np.ascontiguousarray(x, dtype=np.float32).ravel(), device="cuda")

    def timed(fn):
        fn()
        best = float("inf")
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best

    R = regnk.Registration(a.nref, a.nref, 4, 1e-2, precond=regnk.REG_PC_REG)
    nt_ref = cfl_steps(vf, 0.2)
    out = torch.empty(a.nref * a.nref, device="cuda")
    t_ref = timed(lambda: R.transport_rk2a(dev(vf), dev(m0f), out, nt_ref))
    ref = out.cpu().numpy().astype(np.float64).reshape(a.nref, a.nref)
    R.close()
    rows = [{"n": a.nref, "scheme": "RK2A", "cfl": 0.2, "nt": nt_ref, "ms": t_ref, "rel_err": 0.0}]
    print(json.dumps(rows[-1]), flush=True)
    for n in a.grids:
        m0 = restrict(m0f, n)
        v = np.stack([restrict(vf[0], n), restrict(vf[1], n)])
        R = regnk.Registration(n, n, 4, 1e-2, precond=regnk.REG_PC_REG)
        m1 = torch.empty(n * n, device="cuda")
        vd, m0d = dev(v), dev(m0)
        for scheme, c in (("SL", 0.2), ("SL", 1.0), ("SL", 5.0), ("RK2A", 0.2)):
            nt = cfl_steps(v, c)
            if scheme == "SL":
                R.close()
                R = regnk.Registration(n, n, nt, 1e-2, precond=regnk.REG_PC_REG)
                ms = timed(lambda: R.transport(vd, m0d, m1))
            else:
                ms = timed(lambda: R.transport_rk2a(vd, m0d, m1, nt))
            mh = m1.cpu().numpy().astype(np.float64).reshape(n, n)
            err = float(np.linalg.norm(prolong(mh, a.nref) - ref) / np.linalg.norm(ref))
            band = restrict(ref, n)
            err_band = float(np.linalg.norm(mh - band) / np.linalg.norm(band))
            oob = float(np.linalg.norm(ref - prolong(band, a.nref)) / np.linalg.norm(ref))
            rows.append({"n": n, "scheme": scheme, "cfl": c, "nt": nt, "ms": ms, "rel_err": err,
                         "rel_err_band": err_band, "ref_out_of_band": oob})
            print(json.dumps(rows[-1]), flush=True)
        R.close()
    if a.json:
        with open(a.json, "w") as f:
            json.dump(rows, f, indent=1)


if __name__ == "__main__":
    main()
