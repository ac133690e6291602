"""GPU analogues of the heuristic ablation of Section V (Table 3: f0 all
heuristics, f1 degree-based pruning only, f2 skipping visited hyperedges
only, f3 short-circuit only, f4 none).  Every switch changes the work, never
the result: all variants must equal the oracle's L_s."""
import ctypes

import numpy as np
import pytest

import hypergen as hg
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
slg = pytest.importorskip("paper_2010_11448_gb300")

# (name, build keyword arguments); counting per far end visits each pair
# once per row, which is the GPU form of skipping visited hyperedges.
VARIANTS = [
    ("f0", dict(unweighted=True)),
    ("f1", dict()),
    ("f2", dict(prune=False)),
    ("f3", dict(prune=False, unweighted=True)),
    ("f4", dict(algo="spgemm")),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_11448_gb300 import build_lib
    build_lib.build()
    slg.load()


def as_np(t, weighted):
    i, j, w = t
    if i.shape[0] == 0:
        return np.zeros((0, 3 if weighted else 2), np.int64)
    cols = [i.cpu().numpy(), j.cpu().numpy()] + ([w.cpu().numpy()] if weighted else [])
    return np.stack(cols, 1).astype(np.int64)


@pytest.fixture(scope="module")
def medium():
    h = hg.chung_lu(30_000, 60_000, seed=21, size_cap=3000)
    return h, slg.to_device(h)


@pytest.mark.parametrize("dual", [False, True])
@pytest.mark.parametrize("s", [1, 2, 4, 8])
def test_variants_equal_oracle(medium, dual, s):
    h, dh = medium
    ref = oracle.canonical(*oracle.line_graph_of(h, s, dual=dual, threads=8))
    for name, kw in VARIANTS:
        weighted = not kw.get("unweighted", False)
        got = as_np(slg.build(dh, s, dual=dual, **kw), weighted)
        assert np.array_equal(got, ref if weighted else ref[:, :2]), name


def test_no_prune_work(medium):
    # without pruning the walk visits every upper-triangle wedge:
    # sum over vertices of C(d(v), 2), whatever s is
    h, dh = medium
    for dual in (False, True):
        m, n, off, idx = oracle.side(h, dual)
        full = oracle.wedges(m, n, off, idx, 1)
        for s in (2, 8):
            slg.build(dh, s, dual=dual, prune=False)
            assert slg.last_stats()["wedges"] == full
            slg.build(dh, s, dual=dual)
            assert slg.last_stats()["wedges"] == oracle.wedges(m, n, off, idx, s)


def test_no_prune_small_and_core():
    for seed in range(20):
        h = hg.random_small(seed)
        dh = slg.to_device(h)
        for dual in (False, True):
            for s in (1, 2, 3):
                ref = oracle.canonical(*oracle.line_graph_of(h, s, dual=dual))
                got = as_np(slg.build(dh, s, dual=dual, prune=False), True)
                assert np.array_equal(got, ref), (seed, dual, s)
    h = hg.lognormal_web(20_000, 40_000, seed=7, cap=2000, core_edges=256,
                         core_vertices=512, core_density=0.3)
    dh = slg.to_device(h)
    for dual in (False, True):
        ref = oracle.canonical(*oracle.line_graph_of(h, 8, dual=dual, threads=8))
        got = as_np(slg.build(dh, 8, dual=dual, prune=False, tensor=True), True)
        assert np.array_equal(got, ref), dual


def test_no_prune_other_algorithms_rejected(medium):
    h, dh = medium
    lib = slg.load()
    n = ctypes.c_int64(0)
    for algo in (slg.SLG_ALGO_PLAIN, slg.SLG_ALGO_SPGEMM):
        assert lib.slg_count(ctypes.byref(dh.struct), 2, algo | slg.SLG_NO_PRUNE,
                             ctypes.byref(n), None) == 6
