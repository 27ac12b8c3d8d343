"""The N > 1 path of bench.py (replicas: every rank runs the whole workload on its own GPU) on CPU
with two gloo ranks: the job time is the slowest rank's, on every rank, and the job value counts
every rank's cells over that time."""
import os
import socket
import sys

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    local_ms = [10.0, 25.0][rank]
    t = bench.job_time_ms(local_ms, world, "cpu")
    out.put((rank, t, bench.job_value(1000, 4, world, t)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [25.0, 25.0]
    assert all(abs(g[2] - 2 * 1000 * 4 / 0.025 / 1e6) < 1e-12 for g in got)


def test_single_rank_is_its_own_time():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_time_ms(7.5, 1, "cpu") == 7.5
    assert bench.job_value(100, 2, 1, 7.5) == 100 * 2 / 0.0075 / 1e6
