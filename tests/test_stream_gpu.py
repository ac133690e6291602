"""Streaming an edge list too large for memory: slg_row_offsets gives each
row's start in the canonical list, and row ranges of bounded size built with
slg_build_rows concatenate to the whole list (checked against the oracle, and
at full size against the closed form sum of weights of L_1 =
sum over vertices of C(d(v), 2))."""
import ctypes

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


@pytest.fixture(scope="module")
def medium():
    h = hg.chung_lu(30_000, 60_000, seed=21, size_cap=3000)
    return h, slg.to_device(h)


@pytest.mark.parametrize("dual", [False, True])
def test_offsets_and_chunks(medium, dual):
    h, dh = medium
    want = oracle.canonical(*oracle.line_graph_of(h, 2, dual=dual, threads=8))
    R = h.n if dual else h.m
    ptr = slg.row_offsets(dh, 2, dual).cpu().numpy()
    counts = np.bincount(want[:, 0], minlength=R)
    assert ptr[0] == 0 and np.array_equal(np.diff(ptr), counts)
    parts, sizes = [], []
    for a, b, i, j, w in slg.build_stream(dh, 2, 5000, dual=dual):
        assert i.shape[0] == ptr[b] - ptr[a]
        assert i.shape[0] <= 5000 or b == a + 1
        sizes.append(i.shape[0])
        parts.append(np.stack([i.cpu().numpy(), j.cpu().numpy(), w.cpu().numpy()], 1))
    got = np.concatenate(parts).astype(np.int64)
    assert len(sizes) > 3 and np.array_equal(got, want)


def test_unsupported(medium):
    h, dh = medium
    lib = slg.load()
    ptr = torch.empty(h.m + 1, dtype=torch.int64, device="cuda")
    for flags in (slg.SLG_RELABEL_ASC, slg.SLG_ALGO_PLAIN, slg.SLG_ALGO_SPGEMM):
        assert lib.slg_row_offsets(ctypes.byref(dh.struct), 2, flags, ptr.data_ptr(), None) == 6


def test_l1_full_size_streamed():
    # L_1 of the 1M x 2M Chung-Lu workload has 1.7e9 (H) and 7.8e9 (H*) pairs;
    # streamed in chunks of at most 4e8 pairs: every 997th row of every chunk
    # equals the oracle's element by element, the weights add up to the
    # closed form and the pair count matches slg_count
    c = dict(hg.CONFIGS["chung_lu_1m"])
    c.pop("kind")
    h = hg.chung_lu(name="chung_lu_1m", **c)
    dh = slg.to_device(h)
    for dual in (False, True):
        m, n, off, idx = oracle.side(h, dual)
        d = np.bincount(idx, minlength=n).astype(np.int64)
        closed = int((d * (d - 1) // 2).sum())
        rows = np.arange(0, m, 997, dtype=np.int32)
        want = oracle.canonical(*oracle.line_graph(m, n, off, idx, 1, rows=rows, threads=16))
        rows_t = torch.from_numpy(rows).cuda()
        total_w = 0
        total_p = 0
        chunks = 0
        got = []
        for a, b, i, j, w in slg.build_stream(dh, 1, 400_000_000, dual=dual):
            chunks += 1
            total_p += int(i.shape[0])
            total_w += int(w.sum(dtype=torch.int64))
            sel = torch.isin(i, rows_t)
            got.append(np.stack([i[sel].cpu().numpy(), j[sel].cpu().numpy(),
                                 w[sel].cpu().numpy()], 1).astype(np.int64))
        assert chunks >= 4
        assert np.array_equal(np.concatenate(got), want)
        assert total_w == closed
        assert total_p == slg.count(dh, 1, dual)
