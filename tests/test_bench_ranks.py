"""The multi-rank path of bench.py on CPU: two gloo ranks (127.0.0.1) time different regions,
and the job's time is the slowest rank's; the job rate counts every rank's units (replicas,
weak scaling), and the serving replicas' rates add. The GPU runs use the same functions with
NCCL."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as tmp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    try:
        ms = bench.max_over_ranks(10.0 * (rank + 1), "cpu")      # rank r timed 10 (r + 1) ms
        total = bench.sum_over_ranks(1.0e9 * (rank + 1), "cpu")  # per-rank served rates
        q.put((rank, ms, bench.job_rate(1000.0, ws, ms), total))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_the_units():
    ws, port = 2, _free_port()
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(ws))
    for rank, ms, rate, total in got:
        assert ms == 20.0                       # the slower rank's 20 ms for both ranks
        assert rate == pytest.approx(2 * 1000.0 / 0.020)
        assert total == pytest.approx(3.0e9)    # replicas' rates add


def test_single_rank_rate():
    import bench
    assert bench.job_rate(5e9, 1, 1000.0) == pytest.approx(5e9)
