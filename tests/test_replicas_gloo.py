"""bench.py's replica path (one replica per rank, whole-job rate over the
slowest rank's time) on two gloo ranks on the CPU."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench

    ms = 100.0 + 25.0 * rank  # rank 1 is the slower one
    slow = bench.max_over_ranks(ms, torch.device("cpu"))
    rate = bench.whole_job_rate(world, 1000, 10, slow)
    out.put((rank, slow, rate))
    dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank():
    import socket

    import torch.multiprocessing as mp

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [125.0, 125.0]
    # 2 ranks x 1000 units x 10 steps in 0.125 s
    assert got[0][2] == pytest.approx(2 * 1000 * 10 / 0.125)
