"""bench.py's multi-rank aggregation (sum of units, max of times) on two
CPU ranks over gloo: the N > 1 path without GPUs."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.dist_env()
    units, ms = bench.aggregate(1000.0 * (rank + 1), 10.0 + 5 * rank, w)
    q.put((r, w, lr, units, ms))
    dist.destroy_process_group()


def test_two_rank_aggregate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, (r, w, lr, units, ms) in enumerate(res):
        assert (r, w, lr) == (rank, 2, rank)
        assert units == 3000.0          # whole-job units: summed
        assert ms == 15.0               # slowest rank


def test_single_rank_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(12.0, 3.0, 1) == (12.0, 3.0)
