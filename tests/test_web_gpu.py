"""The dense-core tile path at full size: the web-shaped workload (4M
hyperedges over 10M vertices, lognormal sizes capped at 10^5, a planted core
of 4,096 hyperedges x 8,192 vertices at density 0.3) built with
SLG_TENSOR_CORE at s = 2, 8, 32 on H and H*, in the launch configuration of
the dense-core benchmark.  Every 97th row, every row of the planted core and
the 64 largest rows are compared with the CPU oracle element by element
(§III definition of L_s; §IV-D's B·Bᵀ view, which the tile path computes
exactly); order, threshold and size-filter properties are checked on all
pairs on the device.

The oracle runs once per side at s = 2 on the sampled rows; L_s for s = 8
and 32 are its pairs with w >= s (L_s is the part of L_2 with w >= s, with
the same weights: §III)."""
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
    slg.set_core_params()  # the library defaults the benchmark uses


@pytest.fixture(scope="module")
def web_4m():
    h = hg.config("web_4m")
    assert h.core_edges is not None and h.core_edges.shape[0] == 4096
    return h, slg.to_device(h)


@pytest.mark.parametrize("dual", [False, True])
def test_web_4m_tile_path_sampled_rows(web_4m, dual):
    h, dh = web_4m
    m, n, off, idx = oracle.side(h, dual)
    sizes_np = np.diff(off)
    core = h.core_vertices if dual else h.core_edges
    heavy = np.argsort(sizes_np, kind="stable")[-64:]
    rows = np.unique(np.concatenate([np.arange(0, m, 97), core, heavy])).astype(np.int32)
    want2 = oracle.canonical(*oracle.line_graph(m, n, off, idx, 2, rows=rows, threads=16))
    rows_t = torch.from_numpy(rows).cuda()
    sizes = torch.from_numpy(sizes_np.astype(np.int32)).cuda()
    for s in (2, 8, 32):
        i, j, w = slg.build(dh, s, dual=dual, tensor=True)
        st = slg.last_stats()
        assert st["core_rows"] >= 1024, "tile path not taken"
        sel = torch.isin(i, rows_t)
        got = np.stack([i[sel].cpu().numpy(), j[sel].cpu().numpy(), w[sel].cpu().numpy()],
                       1).astype(np.int64)
        want = want2[want2[:, 2] >= s]
        assert np.array_equal(got, want), (dual, s)
        # properties of every pair, on the device
        assert bool(torch.all(i < j)) and bool(torch.all(w >= s))
        key = i.long() * m + j.long()
        assert bool(torch.all(key[1:] > key[:-1]))
        assert bool(torch.all(sizes[i.long()] >= s)) and bool(torch.all(sizes[j.long()] >= s))
        assert i.shape[0] == slg.count(dh, s, dual, tensor=True)
        del i, j, w, sel, key
