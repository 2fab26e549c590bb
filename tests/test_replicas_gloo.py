"""The multi-GPU path of bench.py is replicas only (a single QP has no
data-parallel exchange): each rank times its own solves, and the job's figures
are the slowest rank's time and the QPs solved by all ranks.  Checked here with
two gloo processes on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r "took" 100 + 50 r ms and solved r + 1 QPs
    t, k = bench.reduce_over_ranks(100.0 + 50.0 * rank, rank + 1)
    q.put((rank, t, k))
    dist.destroy_process_group()


def test_reduce_over_ranks_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == [(0, 150.0, 3), (1, 150.0, 3)]


def test_reduce_over_ranks_single_process():
    pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(12.5, 4) == (12.5, 4)
