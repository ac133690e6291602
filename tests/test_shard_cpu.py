"""The multi-GPU split of one build (the parallel loop over hyperedges of
Section IV-F), on two CPU ranks over gloo: rows cut into contiguous ranges of
balanced wedge work, each rank computes its range (here with the CPU oracle,
standing in for slg_build_rows on its GPU), one all-gather of the pair
counts places every rank's pairs, and the concatenation equals the
single-rank list.  Unmeasured on GPU hardware: one GPU per run here."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import hypergen as hg  # noqa: E402
import oracle  # noqa: E402
from paper_2010_11448_gb300 import shard  # noqa: E402


def row_work_by_definition(h, s, dual):
    """Per row e with |e| >= s: the number of wedges e -> v -> f with f > e and
    |f| >= s (Algorithm 3's walk with degree-based pruning), by brute force
    over each row's vertices and their columns."""
    m, n, off, idx = oracle.side(h, dual)
    t_off, t_idx = oracle.transpose(m, n, off, idx)
    size = np.diff(off)
    work = np.zeros(m, np.int64)
    for e in range(m):
        if size[e] < s:
            continue
        for v in idx[off[e]:off[e + 1]]:
            col = t_idx[t_off[v]:t_off[v + 1]]
            col = col[col > e]
            work[e] += int(np.count_nonzero(size[col] >= s))
    return work


def test_balanced_ranges_properties():
    rng = np.random.default_rng(1)
    for parts in (1, 2, 3, 7):
        work = rng.integers(0, 1000, 500) * (rng.random(500) < 0.7)
        b = shard.balanced_ranges(work, parts)
        assert b[0] == 0 and b[-1] == 500 and len(b) == parts + 1
        assert all(x <= y for x, y in zip(b[:-1], b[1:]))
        total, biggest = int(work.sum()), int(work.max())
        for k in range(parts):
            part = int(work[b[k]:b[k + 1]].sum())
            assert abs(part - total / parts) <= biggest + 1
    assert shard.offsets_of([3, 0, 5]) == [0, 3, 3, 8]


def test_work_helper_matches_the_closed_form():
    h = hg.chung_lu(800, 1600, seed=3, size_cap=200)
    for dual in (False, True):
        m, n, off, idx = oracle.side(h, dual)
        for s in (1, 3):
            assert row_work_by_definition(h, s, dual).sum() == oracle.wedges(m, n, off, idx, s)


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import hypergen as hg2
    import oracle as orc
    from paper_2010_11448_gb300 import shard as sh
    dist.init_process_group("gloo", rank=rank, world_size=world)
    h = hg2.chung_lu(1500, 3000, seed=7, size_cap=300)  # the same replicated input
    out = []
    for dual, s in ((False, 2), (True, 2), (True, 3)):
        work = row_work_by_definition(h, s, dual)
        bounds = sh.balanced_ranges(work, world)
        a, b = bounds[rank], bounds[rank + 1]
        m, n, off, idx = orc.side(h, dual)
        mine = orc.canonical(*orc.line_graph(m, n, off, idx, s,
                                             rows=np.arange(a, b, dtype=np.int32)))
        cnt = torch.tensor([mine.shape[0]], dtype=torch.int64)
        allc = [torch.zeros_like(cnt) for _ in range(world)]
        dist.all_gather(allc, cnt)
        offs = sh.offsets_of([int(x) for x in allc])
        parts = [None] * world
        dist.all_gather_object(parts, (offs[rank], mine))
        out.append((dual, s, bounds, offs, parts, int(work.sum()), int(work.max())))
    q.put((rank, out))
    dist.destroy_process_group()


def test_two_rank_split_concatenates_to_the_whole_list():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 2
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    h = hg.chung_lu(1500, 3000, seed=7, size_cap=300)
    for k, (dual, s) in enumerate(((False, 2), (True, 2), (True, 3))):
        want = oracle.canonical(*oracle.line_graph_of(h, s, dual=dual))
        views = [res[r][k] for r in range(world)]
        assert views[0][2] == views[1][2] and views[0][3] == views[1][3]  # same plan everywhere
        _, _, bounds, offs, parts, total, biggest = views[0]
        whole = np.zeros((offs[-1], 3), np.int64)
        for off, piece in parts:
            whole[off:off + piece.shape[0]] = piece
        assert np.array_equal(whole, want), (dual, s)
        assert offs[-1] == want.shape[0]
        work = row_work_by_definition(h, s, dual)
        for r in range(world):  # balanced within one row's work
            assert abs(int(work[bounds[r]:bounds[r + 1]].sum()) - total / world) <= biggest + 1
