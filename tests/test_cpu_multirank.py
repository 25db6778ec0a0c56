"""The multi-rank path of bench.py on CPU: two processes over gloo.

bench.py runs one replica of the solve per rank (weak scaling, no data-path
collective); the only cross-rank steps are the barrier and the max-over-ranks
reduction of the timed region, which decides the whole-job rate.  These run
here with the gloo backend on 127.0.0.1; the reference arm on a rank other
than 0 must return without doing any work.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as tdist
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, ws, lr = bench.rank_info()
    slowest = bench.max_over_ranks(10.0 + 5.0 * rank)  # rank 1 is the slow one
    tdist.barrier()
    q.put((rank, r, ws, lr, slowest))
    tdist.destroy_process_group()


def test_two_rank_max_and_rate():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert [x[1] for x in res] == [0, 1] and all(x[2] == 2 for x in res)
    assert all(x[4] == 15.0 for x in res)  # both ranks see the slowest rank's time
    sys.path.insert(0, ROOT)
    import bench
    # 2 ranks x 10 steps x 1e6 units in 2 s (the slowest rank) -> 10 M units/s
    assert bench.job_rate(1e6, 10, 2, 2.0) == pytest.approx(10.0)
    assert bench.max_over_ranks(3.5) == 3.5  # no process group: the value itself
    del torch


def test_reference_arm_other_rank_does_no_work(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")

    class Args:
        steps, warmup = 1, 0

    def boom(*a, **k):
        raise AssertionError("rank 1 must not run the oracle")

    monkeypatch.setattr(bench, "cpu_oracle_rate", boom)
    monkeypatch.setattr(bench, "oracle_sampler", boom)
    monkeypatch.setattr(bench, "workload", boom)
    assert bench.bench_reference(Args()) == 0


def _replica_worker(rank, world, port, q):
    """One rank of the replica path: the rank builds the benchmarked workload (seeded, the
    same on every rank), runs its own replica of a small solve (the oracle's direct sum at a
    few targets stands in for the GPU solve on this CPU-only box), times it, and the job
    takes the slowest rank's time; no data crosses ranks."""
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import time
    import numpy as np
    import torch.distributed as tdist
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle as O
    from paper_1601_00035_gb300 import inputs
    f, src_c, dst_c, cfg = bench.workload()
    pts = inputs.block_points(src_c, bench.B)
    v = f[:, 0].reshape(-1).astype(np.float64)
    nz = v != 0
    tgt = inputs.block_points(dst_c, bench.B)[::4099][:64]
    tdist.barrier()
    t0 = time.perf_counter()
    u = O.direct_conv(O.lgf_cube(127), pts[nz], -v[nz], tgt)
    dt = time.perf_counter() - t0
    tdist.barrier()
    slowest = bench.max_over_ranks(dt)
    q.put((rank, float(np.abs(u).sum()), dt, slowest, bench.job_rate(len(tgt), 1, world, slowest)))
    tdist.destroy_process_group()


def test_two_rank_replicas():
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_replica_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][1] == res[1][1] > 0                      # identical replicas
    assert res[0][3] == res[1][3] == max(res[0][2], res[1][2])   # the job's time is the slowest rank's
    assert res[0][4] == pytest.approx(2 * 64 / res[0][3] / 1e6)  # both ranks' points over that time
