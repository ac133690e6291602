"""Degree-ordered relabelling (Section IV-F) changes only which row carries
each pair's work: with SLG_RELABEL_ASC / SLG_RELABEL_DESC the canonical
edge list must equal the oracle's bit for bit, for every algorithm, both
sides, weighted and unweighted, and together with the tensor-core path."""
import ctypes

import numpy as np
import pytest

import hypergen as hg
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
slg = pytest.importorskip("paper_2010_11448_gb300")

ORDERS = ["asc", "desc"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_11448_gb300 import build_lib
    build_lib.build()
    slg.load()


def gpu(dh, s, dual, **kw):
    i, j, w = slg.build(dh, s, dual=dual, **kw)
    if i.shape[0] == 0:
        return np.zeros((0, 3), np.int64)
    w = w.cpu().numpy() if w is not None else np.zeros(i.shape[0], np.int64)
    return np.stack([i.cpu().numpy(), j.cpu().numpy(), w], 1).astype(np.int64)


def want(h, s, dual, unweighted=False):
    got = oracle.canonical(*oracle.line_graph_of(h, s, dual=dual, threads=8))
    if unweighted:
        got[:, 2] = 0
    return got


@pytest.mark.parametrize("relabel", ORDERS)
def test_small_cases(relabel):
    # empty rows, singletons, duplicated rows (ties in size), isolated vertices
    for seed in range(30):
        h = hg.random_small(seed)
        dh = slg.to_device(h)
        for dual in (False, True):
            for s in (1, 2, 3):
                assert np.array_equal(gpu(dh, s, dual, relabel=relabel),
                                      want(h, s, dual)), (seed, dual, s)


@pytest.mark.parametrize("relabel", ORDERS)
@pytest.mark.parametrize("dual", [False, True])
def test_uniform_2k(relabel, dual):
    h = hg.config("uniform_2k")
    dh = slg.to_device(h)
    for s in (1, 2, 3):
        assert np.array_equal(gpu(dh, s, dual, relabel=relabel), want(h, s, dual))
        assert slg.count(dh, s, dual, relabel=relabel) == want(h, s, dual).shape[0]


def test_equal_sizes_keep_order():
    # every row has the same size: the stable relabelling is the identity
    h = hg.uniform(3000, 900, 6, 6, seed=5)
    dh = slg.to_device(h)
    for relabel in ORDERS:
        for dual in (False, True):
            assert np.array_equal(gpu(dh, 2, dual, relabel=relabel), want(h, 2, dual))


def test_tiny_sides():
    for rows in ([], [[0]], [[0, 1]], [[0, 1], [1]], [[0, 1, 2], [0, 1, 2]]):
        h = hg.from_rows(rows, n=3)
        dh = slg.to_device(h)
        for relabel in ORDERS:
            for dual in (False, True):
                for s in (1, 2):
                    assert np.array_equal(gpu(dh, s, dual, relabel=relabel, capacity=16),
                                          want(h, s, dual)), (rows, relabel, dual, s)


@pytest.fixture(scope="module")
def medium():
    h = hg.chung_lu(30_000, 60_000, seed=21, size_cap=3000)
    return h, slg.to_device(h)


@pytest.mark.parametrize("relabel", ORDERS)
@pytest.mark.parametrize("dual", [False, True])
@pytest.mark.parametrize("s", [1, 2, 8])
def test_medium(medium, relabel, dual, s):
    h, dh = medium
    assert np.array_equal(gpu(dh, s, dual, relabel=relabel), want(h, s, dual))


@pytest.mark.parametrize("relabel", ORDERS)
def test_medium_unweighted(medium, relabel):
    h, dh = medium
    for dual in (False, True):
        got = gpu(dh, 3, dual, relabel=relabel, unweighted=True)
        assert np.array_equal(got, want(h, 3, dual, unweighted=True))


@pytest.mark.parametrize("algo", ["plain", "spgemm"])
def test_other_algorithms(medium, algo):
    h, dh = medium
    for relabel in ORDERS:
        for dual in (False, True):
            assert np.array_equal(gpu(dh, 4, dual, relabel=relabel, algo=algo),
                                  want(h, 4, dual)), (relabel, dual)


def test_with_tensor_core():
    h = hg.lognormal_web(20_000, 40_000, seed=7, cap=2000, core_edges=256,
                         core_vertices=512, core_density=0.3)
    dh = slg.to_device(h)
    for relabel in ORDERS:
        for dual in (False, True):
            for s in (2, 8):
                got = gpu(dh, s, dual, relabel=relabel, tensor=True)
                assert np.array_equal(got, want(h, s, dual)), (relabel, dual, s)


def test_stats_and_work(medium):
    # the wedge total is a property of the graph; its split over rows is not
    h, dh = medium
    m, n, off, idx = oracle.side(h, True)
    W = oracle.wedges(m, n, off, idx, 2)
    slg.set_profiling(True)
    try:
        for relabel in (None, "asc", "desc"):
            slg.build(dh, 2, dual=True, relabel=relabel)
            st = slg.last_stats()
            assert st["wedges"] == W
            if relabel:
                assert st["ms_relabel"] > 0 and st["ms_order"] > 0
            else:
                assert st["ms_relabel"] == 0 and st["ms_order"] == 0
    finally:
        slg.set_profiling(False)


def test_flag_errors(medium):
    h, dh = medium
    lib = slg.load()
    n = ctypes.c_int64(0)
    both = slg.SLG_RELABEL_ASC | slg.SLG_RELABEL_DESC
    assert lib.slg_count(ctypes.byref(dh.struct), 2, both, ctypes.byref(n), None) == 1
    oi, oj, ow = slg.alloc_outputs(16)
    rc = lib.slg_build_rows(ctypes.byref(dh.struct), 2, slg.SLG_RELABEL_ASC, 0, 10,
                            oi.data_ptr(), oj.data_ptr(), ow.data_ptr(), 16,
                            ctypes.byref(n), None)
    assert rc == 6
    # capacity errors report the count, as without relabelling
    P = slg.count(dh, 2, relabel="asc")
    rc = lib.slg_build(ctypes.byref(dh.struct), 2, slg.SLG_RELABEL_ASC, oi.data_ptr(),
                       oj.data_ptr(), ow.data_ptr(), 16, ctypes.byref(n), None)
    assert rc == 2 and n.value == P
