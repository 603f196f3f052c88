"""Replica aggregation of bench.py on CPU: two gloo ranks, each with its own
time; the job rate uses the slowest rank and counts every replica's steps."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 * (rank + 1)  # rank 1 is slower
    m = bench.max_over_ranks(ms)
    q.put((rank, m, bench.job_rate(10, world, m)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [200.0, 200.0]
    assert out[0][2] == pytest.approx(10 * 2 / 0.2)


def test_single_process_identity():
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.job_rate(30, 1, 1000.0) == pytest.approx(30.0)
