"""The sparse bin (rows of 1,025 to 16,384 wedges with s >= 2, above the CTA
bins only when their far ends are sparse in their id span): a first pass
marks far ends seen twice in a Bloom filter and claims them as candidates
in a shared table, a second pass counts the candidates' wedges exactly.
Rows above 8,192 wedges run in the kernel instance with the larger table,
the others in the one with the smaller table; a row whose candidates or
survivors do not fit its table is handed to the giant bin.  Every case is
compared with the CPU oracle element by element."""
import numpy as np
import pytest

import hypergen as hg
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
slg = pytest.importorskip("paper_2010_11448_gb300")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_11448_gb300 import build_lib
    build_lib.build()
    slg.load()


def as_np(t):
    i, j, w = t
    cols = [i.cpu().numpy(), j.cpu().numpy()]
    cols.append(w.cpu().numpy() if w is not None else np.zeros_like(cols[0]))
    return np.stack(cols, 1).astype(np.int64) if cols[0].shape[0] else np.zeros((0, 3), np.int64)


def many_repeats(m=100_000, n=20_000, k=3, shared=3000, seed=4):
    """Hyperedge 0 holds vertices 0..k-1; hyperedges 10000 .. 10000+shared-1
    hold all of them too (plus a few random vertices), so row 0 has k x
    shared wedges and `shared` distinct far ends that each repeat k times:
    more repeated far ends than one window of the sparse bin's table holds.
    The rest are small random hyperedges over the other vertices."""
    rng = np.random.default_rng(seed)
    rows = []
    for e in range(m):
        if e == 0:
            rows.append(np.arange(k))
        elif 10_000 <= e < 10_000 + shared:
            extra = rng.choice(np.arange(k, n), 3, replace=False)
            rows.append(np.concatenate([np.arange(k), np.sort(extra)]))
        else:
            rows.append(np.sort(rng.choice(np.arange(k, n), int(rng.integers(1, 6)),
                                           replace=False)))
    return hg.from_rows(rows, n)


@pytest.mark.parametrize("k", [2, 3])
def test_window_overflow_split(k):
    h = many_repeats(k=k)
    dh = slg.to_device(h)
    for s in (2, k):
        got = as_np(slg.build(dh, s))
        st = slg.last_stats()
        assert st["rows_bin"][4] >= 1, "row 0 did not take the sparse bin"
        assert np.array_equal(got, oracle.canonical(*oracle.line_graph_of(h, s, threads=8)))
        # the short-circuit gives the same pairs
        i, j, w = slg.build(dh, s, unweighted=True)
        assert w is None
        assert np.array_equal(np.stack([i.cpu().numpy(), j.cpu().numpy()], 1), got[:, :2])
        assert slg.count(dh, s) == got.shape[0]


def test_rows_across_two_windows():
    # The dual of a Chung-Lu hypergraph with 1.5M vertices: long rows whose
    # far ends spread over an id span of up to 1.5M (a Bloom filter of at
    # most 2^17 bits per row), on both sides of the 8,192-wedge split.
    h = hg.chung_lu(200_000, 1_500_000, seed=33, size_cap=10_000)
    dh = slg.to_device(h)
    m, n, off, idx = oracle.side(h, True)
    deg = np.diff(off)
    heavy = np.argsort(-deg, kind="stable")[:2000]
    rows = np.unique(np.concatenate([heavy, np.arange(0, m, 211)])).astype(np.int32)
    want2 = oracle.canonical(*oracle.line_graph(m, n, off, idx, 2, rows=rows, threads=16))
    rows_t = torch.from_numpy(rows).cuda()
    for s in (2, 3, 5):
        i, j, w = slg.build(dh, s, dual=True)
        st = slg.last_stats()
        assert st["rows_bin"][4] > 100
        sel = torch.isin(i, rows_t)
        got = np.stack([i[sel].cpu().numpy(), j[sel].cpu().numpy(), w[sel].cpu().numpy()],
                       1).astype(np.int64)
        assert np.array_equal(got, want2[want2[:, 2] >= s]), s
        key = i.long() * m + j.long()
        assert bool(torch.all(key[1:] > key[:-1])) and bool(torch.all(w >= s))
        assert i.shape[0] == slg.count(dh, s, dual=True)


def split_rows(m=200_000, n=400_000, seed=8):
    """Small random hyperedges (1 to 4 of vertices 1000 .. n-1) plus hubs:
    row 0 holds hubs 0..19, each also in 640 random hyperedges (about
    12,800 wedges at s = 2, 9,900 at s = 3: the larger-table instance); row
    1 holds hubs 20..29, each in 500 (about 5,000: the smaller-table
    instance); row 2 holds hubs 30 and 31, both in the same 3,000 random
    hyperedges, so that row 2 has 3,000 far ends of two wedges each, more
    distinct candidates than a 2,048-slot table holds, and every one of
    those 3,000 rows meets the others in two vertices.  All far ends spread
    over ids up to m: the rows are sparse in their span."""
    rng = np.random.default_rng(seed)
    size = rng.integers(1, 5, m)
    r = [np.repeat(np.arange(m), size), np.zeros(20, np.int64), np.ones(10, np.int64),
         np.full(2, 2)]
    c = [rng.integers(1000, n, int(size.sum())), np.arange(20), np.arange(20, 30),
         np.array([30, 31])]
    for hub in range(30):
        f = rng.choice(np.arange(3, m), 640 if hub < 20 else 500, replace=False)
        r.append(f)
        c.append(np.full(f.shape[0], hub))
    f = rng.choice(np.arange(3, m), 3000, replace=False)
    r += [f, f]
    c += [np.full(3000, 30), np.full(3000, 31)]
    return hg.from_pairs(np.concatenate(r), np.concatenate(c), m, n)


@pytest.mark.parametrize("s", [2, 3])
def test_two_instances_and_hand_off(s):
    from test_shard_cpu import row_work_by_definition
    h = split_rows()
    work = row_work_by_definition(h, s, False)
    assert work[0] > 8192 and 1024 < work[1] <= 8192 and 1024 < work[2] <= 8192
    dh = slg.to_device(h)
    want = oracle.canonical(*oracle.line_graph_of(h, s, threads=8))
    got = as_np(slg.build(dh, s))
    st = slg.last_stats()
    assert st["rows_bin"][4] >= 3, "rows 0, 1 and 2 take the sparse bin"
    # row 2's 3,000 candidates cannot fit the smaller table: handed over
    assert st["rows_bin"][3] >= 1, "no sparse row was handed to the giant bin"
    assert np.array_equal(got, want)
    i, j, w = slg.build(dh, s, unweighted=True)
    assert w is None
    assert np.array_equal(np.stack([i.cpu().numpy(), j.cpu().numpy()], 1), want[:, :2])
    assert slg.count(dh, s) == want.shape[0]
