"""s-sweeps (L_s ⊆ L_s' for s >= s', Section III): slg_filter keeps the
triples of a canonical list with w >= s, and slg_build_sweep answers several
thresholds with one walk.  Every list must equal the oracle's L_s bit for
bit."""
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


def as_np(t):
    i, j, w = t
    if i.shape[0] == 0:
        return np.zeros((0, 3), np.int64)
    w = w.cpu().numpy() if w is not None else np.zeros(i.shape[0], np.int64)
    return np.stack([i.cpu().numpy(), j.cpu().numpy(), w], 1).astype(np.int64)


def want(h, s, dual):
    return oracle.canonical(*oracle.line_graph_of(h, s, dual=dual, threads=8))


@pytest.fixture(scope="module")
def medium():
    h = hg.chung_lu(30_000, 60_000, seed=21, size_cap=3000)
    return h, slg.to_device(h)


@pytest.mark.parametrize("dual", [False, True])
def test_sweep_medium(medium, dual):
    h, dh = medium
    S = [8, 2, 3, 5, 2, 16]  # any order, repeats allowed
    got = slg.build_sweep(dh, S, dual=dual)
    for s, t in zip(S, got):
        assert np.array_equal(as_np(t), want(h, s, dual)), s


def test_sweep_small_cases():
    for seed in range(20):
        h = hg.random_small(seed)
        dh = slg.to_device(h)
        for dual in (False, True):
            got = slg.build_sweep(dh, [1, 2, 3], dual=dual)
            for s, t in zip([1, 2, 3], got):
                assert np.array_equal(as_np(t), want(h, s, dual)), (seed, dual, s)


def test_filter_from_l1(medium):
    h, dh = medium
    for dual in (False, True):
        base = slg.build(dh, 1, dual=dual)
        for s in (1, 2, 4, 7, 50, 10_000):
            got = slg.filter_pairs(*base, s)
            assert np.array_equal(as_np(got), want(h, s, dual)), (dual, s)
        # without weights in the output
        i, j, w = slg.filter_pairs(*base, 3, weights=False)
        ref = want(h, 3, dual)
        assert w is None and np.array_equal(i.cpu().numpy(), ref[:, 0])
        assert np.array_equal(j.cpu().numpy(), ref[:, 1])


def test_filter_edges():
    lib = slg.load()
    n = ctypes.c_int64(-5)
    e = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert lib.slg_filter(None, None, None, 0, 2, None, None, None, 0, ctypes.byref(n), None) == 0
    assert n.value == 0
    assert lib.slg_filter(e.data_ptr(), e.data_ptr(), e.data_ptr(), 1, 0, None, None, None, 0,
                          ctypes.byref(n), None) == 1  # s < 1
    # capacity error reports the kept count; tail of a tile and several tiles
    for size in (1, 8191, 8192, 8193, 50_000):
        w = torch.arange(size, dtype=torch.int32, device="cuda") % 7
        i = torch.arange(size, dtype=torch.int32, device="cuda")
        j = i + 1
        keep = (w >= 3).cpu().numpy()
        rc = lib.slg_filter(i.data_ptr(), j.data_ptr(), w.data_ptr(), size, 3, None, None, None,
                            0, ctypes.byref(n), None)
        assert n.value == int(keep.sum()) and rc == (2 if keep.any() else 0)
        oi, oj, ow = slg.filter_pairs(i, j, w, 3)
        idx = np.nonzero(keep)[0]
        assert np.array_equal(oi.cpu().numpy(), idx)
        assert np.array_equal(oj.cpu().numpy(), idx + 1)
        assert np.array_equal(ow.cpu().numpy(), (np.arange(size) % 7)[idx])


def test_sweep_errors(medium):
    h, dh = medium
    lib = slg.load()
    S = [2, 5]
    n2 = slg.count(dh, 2)
    n5 = slg.count(dh, 5)
    outs = [slg.alloc_outputs(n2), slg.alloc_outputs(3)]  # the second list is too small
    k = 2
    arr = lambda vals, t: (t * k)(*vals)
    ptrs = lambda q: arr([o[q].data_ptr() for o in outs], ctypes.c_void_p)
    cnt = (ctypes.c_int64 * k)()
    rc = lib.slg_build_sweep(ctypes.byref(dh.struct), arr(S, ctypes.c_int32), k, 0, ptrs(0),
                             ptrs(1), ptrs(2), arr([n2, 3], ctypes.c_int64), cnt, None)
    assert rc == 2 and list(cnt) == [n2, n5]
    # the base list itself too small: only its count is known
    rc = lib.slg_build_sweep(ctypes.byref(dh.struct), arr(S, ctypes.c_int32), k, 0, ptrs(0),
                             ptrs(1), ptrs(2), arr([5, n5], ctypes.c_int64), cnt, None)
    assert rc == 2 and list(cnt) == [n2, -1]
    # unweighted sweeps are not provided (the weights decide membership)
    rc = lib.slg_build_sweep(ctypes.byref(dh.struct), arr(S, ctypes.c_int32), k,
                             slg.SLG_UNWEIGHTED, ptrs(0), ptrs(1), ptrs(2),
                             arr([n2, n5], ctypes.c_int64), cnt, None)
    assert rc == 6
    # other lists may skip their weights
    outs2 = [slg.alloc_outputs(n2), slg.alloc_outputs(n5, unweighted=True)]
    ow = arr([outs2[0][2].data_ptr(), None], ctypes.c_void_p)
    rc = lib.slg_build_sweep(ctypes.byref(dh.struct), arr(S, ctypes.c_int32), k, 0,
                             arr([o[0].data_ptr() for o in outs2], ctypes.c_void_p),
                             arr([o[1].data_ptr() for o in outs2], ctypes.c_void_p), ow,
                             arr([n2, n5], ctypes.c_int64), cnt, None)
    assert rc == 0
    ref = want(h, 5, False)
    assert np.array_equal(outs2[1][0][:n5].cpu().numpy(), ref[:, 0])


def test_sweep_with_relabel_and_tensor():
    h = hg.lognormal_web(20_000, 40_000, seed=7, cap=2000, core_edges=256,
                         core_vertices=512, core_density=0.3)
    dh = slg.to_device(h)
    for dual in (False, True):
        for kw in ({"relabel": "asc"}, {"tensor": True}):
            got = slg.build_sweep(dh, [2, 8, 32], dual=dual, **kw)
            for s, t in zip([2, 8, 32], got):
                assert np.array_equal(as_np(t), want(h, s, dual)), (dual, kw, s)
