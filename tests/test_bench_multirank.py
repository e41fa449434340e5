"""The multi-rank path of bench.py (independent replicas, job time = slowest rank)
exercised with two gloo processes on the CPU."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    my_ms = 10.0 * (rank + 1)
    mx = bench.reduce_max(my_ms, dist, "cpu")
    value = bench.job_throughput(1000.0, 5, world, mx)
    q.put((rank, mx, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_timing_reduction():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [20.0, 20.0]      # both ranks see the slowest time
    assert all(abs(r[2] - 2 * 1000 * 5 / 0.020) < 1e-6 for r in res)
    _ = torch, os
