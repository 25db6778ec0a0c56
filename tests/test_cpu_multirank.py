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
