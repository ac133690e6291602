"""The sparse bin (large rows whose far ends are sparse in their id span,
s >= 2): a seen-bit per id of a window of the span, repeats counted in a
small shared table, windows redone at half the width when the table would
overflow.  Every case is compared with the CPU oracle element by element."""
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
    # The dual of a Chung-Lu hypergraph with 1.5M vertices: the rows of the
    # first ~450K vertices span more than one window of 2^20 ids.  Large
    # sparse rows at or below 8192 wedges keep their far ends in shared
    # memory; the larger ones walk again for the second window.
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
