"""The N > 1 timing path of bench.py on two gloo ranks (CPU): the slowest
rank's time is what every rank reports, and the weak-scaling value counts all
ranks' work over that time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = 1.5 + rank                     # rank 1 is the slow one
        t = bench.reduce_max_over_ranks(local)
        out.put((rank, t, bench.weak_scaling_value(100.0, world, 4, t)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_weak_scaling_value():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2.5, 2.5]
    assert all(abs(r[2] - 100.0 * 2 * 4 / 2.5) < 1e-12 for r in res)


def test_single_process_passthrough():
    import bench
    assert bench.reduce_max_over_ranks(3.25) == 3.25
    assert bench.weak_scaling_value(10, 1, 2, 4.0) == 5.0
