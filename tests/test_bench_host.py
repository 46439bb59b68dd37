"""Host logic of bench.py (CPU only): the whole-job aggregation over
replicas (max time, summed work) with two gloo ranks, and the single-rank
path."""

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r: 1000 + 500 r ms for 10 + r matvecs; e2e 2000 + 100 r ms for 10 + r
    v, e = bench.aggregate_ranks(dist, torch.device("cpu"), 1000.0 + 500.0 * rank, 10 + rank,
                                 2000.0 + 100.0 * rank, 10 + rank)
    q.put((rank, v, e))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, v, e in out:
        assert v == pytest.approx(21 / 1.5)       # 21 matvecs over max(1.0, 1.5) s
        assert e == pytest.approx(21 / 2.1)


def test_single_rank_aggregation():
    import bench
    v, e = bench.aggregate_ranks(None, None, 2000.0, 40, 4000.0, 40)
    assert v == pytest.approx(20.0) and e == pytest.approx(10.0)


def test_3d_matvec_bytes_count_each_kernel():
    """The algorithmic bytes per point of a 3D GN matvec add up its kernels:
    spline prefilter of v~ (3 fields x 3 axis passes x 8 B), the first
    incremental step (v~ and G at X_D, v~, grad m, m~ out: 76 B), nt - 1
    further steps with their prefilters, lambda~_nt with the first term of
    b~, nt adjoint steps with their prefilters, and the spectral beta A v~ +
    b~ on two packed complex fields (292 B); cubic Lagrange drops every
    prefilter pass."""
    import bench
    for nt in (1, 2, 4, 8):
        spline = 3 * 24 + 76 + (nt - 1) * (68 + 24) + 32 + nt * (64 + 24) + 292
        assert bench.d3_bytes_per_point(nt) == spline == 380 + 180 * nt
        lag = 76 + (nt - 1) * 68 + 32 + nt * 64 + 292
        assert bench.d3_bytes_per_point(nt, lagrange=True) == lag
