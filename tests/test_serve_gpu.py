"""Serving form: queries admitted as slots and memory free up, run
concurrently on their own streams; every result equals the same query run
alone (and the oracle)."""
import numpy as np
import pytest

import hypergen as hg
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
slg = pytest.importorskip("paper_2010_11448_gb300")


@pytest.fixture(scope="module")
def pool():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_11448_gb300 import build_lib
    build_lib.build()
    slg.load()
    hs = [hg.chung_lu(m, 2 * m, seed=40 + k, size_cap=600)
          for k, m in enumerate((3000, 8000, 15000, 30000))]
    return hs, [slg.to_device(h) for h in hs]


def as_np(t):
    i, j, w = t
    if i.shape[0] == 0:
        return np.zeros((0, 3), np.int64)
    return np.stack([i.cpu().numpy(), j.cpu().numpy(), w.cpu().numpy()], 1).astype(np.int64)


def test_mix_equals_alone(pool):
    from paper_2010_11448_gb300.serve import Server
    hs, dhs = pool
    rng = np.random.default_rng(0)
    reqs = [(int(rng.integers(0, 4)), int(rng.integers(1, 9)), bool(rng.integers(0, 2)))
            for _ in range(48)]
    srv = Server(dhs, slots=4, keep_results=True)
    qs = [srv.submit(*r) for r in reqs]
    for q in qs:
        assert q.wait(300)
    srv.close()
    for (gid, s, dual), q in zip(reqs, qs):
        assert q.error is None
        alone = as_np(slg.build(dhs[gid], s, dual=dual))
        assert np.array_equal(as_np(q.result), alone)
        if gid == 0:
            want = oracle.canonical(*oracle.line_graph_of(hs[gid], s, dual=dual))
            assert np.array_equal(alone, want)
    st = Server.summary(qs, 1.0)
    assert st["errors"] == 0 and st["p99_ms"] >= st["p50_ms"] > 0


def test_tiny_budget_admits_one_at_a_time(pool):
    from paper_2010_11448_gb300.serve import Server
    _, dhs = pool
    srv = Server(dhs, slots=4, memory_budget=1)
    qs = [srv.submit(k % 4, 2, False) for k in range(12)]
    for q in qs:
        assert q.wait(300)
    srv.close()
    spans = sorted((q.t_start, q.t_done) for q in qs)
    for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
        assert b0 >= a1 - 1e-6          # never two queries in flight
    assert all(q.error is None for q in qs)


def test_reuse_filters_equal_walks(pool):
    # with reuse, queries at larger thresholds are answered by filtering the
    # kept list of a smaller one; every result must still equal a fresh build
    from paper_2010_11448_gb300.serve import Server
    hs, dhs = pool
    reqs = [(g, s, d) for s in (1, 3, 2, 5, 8, 4) for g in (0, 2) for d in (False, True)]
    srv = Server(dhs, slots=2, keep_results=True, reuse=True, base_s=None)
    qs = []
    for r in reqs:
        q = srv.submit(*r)
        assert q.wait(300)  # one after another: each finds the lists kept so far
        qs.append(q)
    srv.close()
    for (gid, s, dual), q in zip(reqs, qs):
        assert q.error is None
        assert np.array_equal(as_np(q.result), as_np(slg.build(dhs[gid], s, dual=dual)))
    # s = 1 is built first for every graph and side; all later ones filter
    assert [q.reused for q in qs] == [False] * 4 + [True] * (len(reqs) - 4)
    assert Server.summary(qs, 1.0)["answered_by_filter"] == len(reqs) - 4


def test_eager_base_lists_equal_walks(pool):
    # base_s = 2: the first query with s >= 2 on a graph and side builds L_2
    # and keeps it; every query with s >= 2 is answered by filtering it, s = 1
    # walks; concurrent queries on the same graph wait for the one base build
    from paper_2010_11448_gb300.serve import Server
    hs, dhs = pool
    rng = np.random.default_rng(3)
    reqs = [(int(rng.integers(0, 4)), int(rng.integers(1, 12)), bool(rng.integers(0, 2)))
            for _ in range(60)]
    srv = Server(dhs, slots=4, keep_results=True, reuse=True, base_s=2)
    qs = [srv.submit(*r) for r in reqs]
    for q in qs:
        assert q.wait(300)
    srv.close()
    for (gid, s, dual), q in zip(reqs, qs):
        assert q.error is None
        assert np.array_equal(as_np(q.result), as_np(slg.build(dhs[gid], s, dual=dual)))
        assert q.reused == (s >= 2)
    st = Server.summary(qs, 1.0)
    keys = {(g, d) for g, s, d in reqs if s >= 2}
    ones = sum(1 for _, s, _ in reqs if s == 1)
    # one base build per graph and side (two walks at most when the first
    # size guess was short), one walk per s = 1 query (two at most)
    assert st["walks"] <= 2 * (len(keys) + ones)


def test_warm_start_then_stream(pool):
    # warm() builds every base list before the queries arrive; afterwards the
    # memory in flight is back to zero and every s >= 2 query is a filter
    from paper_2010_11448_gb300.serve import Server
    hs, dhs = pool
    srv = Server(dhs, slots=3, keep_results=True, reuse=True, base_s=2, memory_budget=1 << 30)
    assert srv.warm() > 0
    assert srv.in_flight == 0 and len(srv.cached) == 2 * len(dhs)
    reqs = [(g, s, d) for g in range(len(dhs)) for s in (1, 2, 7) for d in (False, True)]
    qs = [srv.submit(*r) for r in reqs]
    for q in qs:
        assert q.wait(300)
    srv.close()
    assert srv.in_flight == 0
    for (gid, s, dual), q in zip(reqs, qs):
        assert q.error is None and q.reused == (s >= 2)
        assert np.array_equal(as_np(q.result), as_np(slg.build(dhs[gid], s, dual=dual)))
