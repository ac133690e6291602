"""The comparison paths (plain per-hyperedge kernel, filtered SpGEMM) give
the same canonical edge list as the oracle, bit for bit."""
import numpy as np
import pytest

import hypergen as hg
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
slg = pytest.importorskip("paper_2010_11448_gb300")

ALGOS = ["plain", "spgemm"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_11448_gb300 import build_lib
    build_lib.build()
    slg.load()


def gpu(dh, s, dual, algo, **kw):
    i, j, w = slg.build(dh, s, dual=dual, algo=algo, **kw)
    if i.shape[0] == 0:
        return np.zeros((0, 3), np.int64)
    w = w.cpu().numpy() if w is not None else np.zeros(i.shape[0], np.int64)
    return np.stack([i.cpu().numpy(), j.cpu().numpy(), w], 1).astype(np.int64)


def want(h, s, dual):
    return oracle.canonical(*oracle.line_graph_of(h, s, dual=dual, threads=8))


@pytest.mark.parametrize("algo", ALGOS)
def test_small_cases(algo):
    for seed in range(20):
        h = hg.random_small(seed)
        dh = slg.to_device(h)
        for dual in (False, True):
            for s in (1, 2, 3):
                assert np.array_equal(gpu(dh, s, dual, algo), want(h, s, dual)), (seed, dual, s)


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("dual", [False, True])
def test_uniform_2k(algo, dual):
    h = hg.config("uniform_2k")
    dh = slg.to_device(h)
    for s in (1, 2, 3):
        assert np.array_equal(gpu(dh, s, dual, algo), want(h, s, dual))


@pytest.fixture(scope="module")
def medium():
    h = hg.chung_lu(30_000, 60_000, seed=21, size_cap=3000)
    return h, slg.to_device(h)


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("dual", [False, True])
@pytest.mark.parametrize("s", [2, 8])
def test_medium(medium, algo, dual, s):
    h, dh = medium
    assert np.array_equal(gpu(dh, s, dual, algo), want(h, s, dual))


def test_plain_counts_wedges(medium):
    h, dh = medium
    for dual in (False, True):
        m, n, off, idx = oracle.side(h, dual)
        for s in (2, 5):
            slg.count(dh, s, dual, algo="plain")
            assert slg.last_stats()["wedges"] == oracle.wedges(m, n, off, idx, s)


def test_spgemm_work_is_full_product(medium):
    # Gustavson's multiply count: sum over rows of the column lengths of the
    # row's vertices = sum over vertices of d(v)^2 (both triangles + diagonal)
    h, dh = medium
    for dual in (False, True):
        m, n, off, idx = oracle.side(h, dual)
        d = np.bincount(idx, minlength=n).astype(np.int64)
        assert slg.wedges(dh, 3, dual) != int((d * d).sum())   # binned: W_s only
        lib = slg.load()
        import ctypes
        out = ctypes.c_int64(0)
        rc = lib.slg_wedges(ctypes.byref(dh.struct), 3, 0x200 | (1 if dual else 0),
                            ctypes.byref(out), None)
        assert rc == 0 and out.value == int((d * d).sum())
