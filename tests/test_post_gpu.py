"""After the edge list: ID squeezing (Section IV-E), the line graph's
adjacency and its connected components, each equal to the oracle's plain
definition element by element."""
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


def np_(t):
    return t.cpu().numpy()


@pytest.mark.parametrize("dual", [False, True])
@pytest.mark.parametrize("s", [2, 8, 40])
def test_squeeze_adjacency_components(medium, dual, s):
    h, dh = medium
    R = h.n if dual else h.m
    i, j, w = slg.build(dh, s, dual=dual)
    ri, rj, rw = np_(i), np_(j), np_(w)
    si, sj, old = slg.squeeze(i, j, R)
    wi, wj, wold = oracle.squeeze(ri, rj, R)
    assert np.array_equal(np_(si), wi) and np.array_equal(np_(sj), wj)
    assert np.array_equal(np_(old), wold)
    V = int(old.shape[0])
    off, adj, adj_w = slg.adjacency(si, sj, w, V)
    woff, wadj, wadjw = oracle.adjacency(wi, wj, rw, V)
    assert np.array_equal(np_(off), woff)
    assert np.array_equal(np_(adj), wadj) and np.array_equal(np_(adj_w), wadjw)
    lab, k = slg.components(i, j, R)
    wlab, wk = oracle.components(ri, rj, R)
    assert np.array_equal(np_(lab), wlab) and k == wk


def test_larger_components():
    h = hg.chung_lu(200_000, 400_000, seed=33, size_cap=5000)
    dh = slg.to_device(h)
    for dual in (False, True):
        R = h.n if dual else h.m
        i, j, _ = slg.build(dh, 3, dual=dual)
        lab, k = slg.components(i, j, R)
        wlab, wk = oracle.components(np_(i), np_(j), R)
        assert np.array_equal(np_(lab), wlab) and k == wk


def test_empty_and_invalid():
    e = torch.zeros(0, dtype=torch.int32, device="cuda")
    si, sj, old = slg.squeeze(e, e, 5)
    assert si.numel() == 0 and old.numel() == 0
    off, adj, _ = slg.adjacency(e, e, e, 5)
    assert np.array_equal(np_(off), np.zeros(6, np.int64)) and adj.numel() == 0
    lab, k = slg.components(e, e, 5)
    assert np.array_equal(np_(lab), np.arange(5)) and k == 0
    lib = slg.load()
    t = lambda a: torch.tensor(a, dtype=torch.int32, device="cuda")
    k64 = ctypes.c_int64(0)
    lab = torch.empty(8, dtype=torch.int32, device="cuda")
    # i >= j, id out of range
    for a, b in (([3], [3]), ([4], [2]), ([0], [8]), ([-1], [2])):
        assert lib.slg_components(t(a).data_ptr(), t(b).data_ptr(), 1, 8, lab.data_ptr(),
                                  ctypes.byref(k64), None) == 1
    # the adjacency wants a canonical list
    off = torch.empty(9, dtype=torch.int64, device="cuda")
    adj = torch.empty(4, dtype=torch.int32, device="cuda")
    a, b = t([1, 0]), t([2, 3])
    assert lib.slg_adjacency(a.data_ptr(), b.data_ptr(), None, 2, 8, off.data_ptr(),
                             adj.data_ptr(), None, None) == 1
    a, b = t([0, 1]), t([3, 2])
    assert lib.slg_adjacency(a.data_ptr(), b.data_ptr(), None, 2, 8, off.data_ptr(),
                             adj.data_ptr(), None, None) == 0
    assert np.array_equal(np_(adj), [3, 2, 1, 0])
