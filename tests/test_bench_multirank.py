"""bench.py's multi-rank timing: the time is the maximum over ranks, checked
with two gloo ranks on the CPU (the GPU benchmark runs one replica per rank
with no data exchange, so this is the only cross-rank step)."""
import multiprocessing as mp
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
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    got = bench.max_over_ranks(10.0 + 5.0 * rank)
    env = bench.dist_env()
    dist.destroy_process_group()
    q.put((rank, got, env))


def test_max_over_ranks_two_gloo_ranks():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [15.0, 15.0]
    assert [o[2][:2] for o in out] == [(0, 2), (1, 2)]


def test_max_over_ranks_without_group():
    pytest.importorskip("torch")
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
