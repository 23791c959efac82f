"""The multi-GPU path of bench.py is replicas only (one independent reduction per rank, no
collective on the data path); its host logic -- the step time is the maximum over the ranks and
the job rate counts every replica -- runs here on two gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(5.0 + 1.5 * rank, "cpu", world)
        q.put((rank, ms, bench.job_rate(ms, world)))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_step():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, rate in res:
        assert ms == pytest.approx(6.5)
        assert rate == pytest.approx(2 * 1000.0 / 6.5)


def test_one_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(4.0, "cpu", 1) == 4.0
    assert bench.job_rate(4.0, 1) == 250.0
