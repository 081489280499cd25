"""The N>1 bench path on CPU: two gloo ranks split the flight path into
per-rank frame schedules and take the max of their timed regions."""

import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    sched = bench.frame_schedule(120, 10, rank, world)
    m = bench.reduce_max(float(10 + rank * 5), world)
    dist.barrier()
    q.put((rank, sched, m))
    dist.destroy_process_group()


def test_two_rank_schedule_and_max():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, m0), (r1, s1, m1) = out
    assert m0 == m1 == 15.0
    assert s0 == list(range(0, 120, 12)) and s1 == list(range(6, 120, 12))
    assert not set(s0) & set(s1)


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
    assert bench.frame_schedule(120, 5, 0, 1) == [0, 24, 48, 72, 96]
    assert bench.frame_schedule(4, 6, 0, 1) == [0, 0, 1, 2, 2, 3]
    assert sorted(set(bench.frame_schedule(120, 1200, 0, 1))) == list(range(120))
