"""Host-side logic of the multi-rank benchmark path, on CPU with gloo (world size 2).

Each rank steps its own replica (no data-path collective); the only exchange is
the max over ranks of the timed region, which these ranks exercise with
different local times.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = 0.10 + 0.05 * rank  # seconds; rank 1 is the slow one
    value, t = bench.throughput(10, local, world)
    q.put((rank, value, t, bench.max_over_ranks(float(rank), world)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
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
    for rank, value, t, mx in out:
        assert t == pytest.approx(0.15)
        assert value == pytest.approx(2 * 10 / 0.15)
        assert mx == 1.0


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    v, t = bench.throughput(20, 0.5, 1)
    assert t == 0.5 and v == pytest.approx(40.0)
