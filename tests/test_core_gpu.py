"""The dense-core tile path (SLG_TENSOR_CORE): a planted dense block counted
on the tensor cores plus the walk over the rest gives exactly the oracle's
L_s, and the same result as the walk alone (tensor path on/off equal)."""
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
    slg.set_core_params(64, 32, 0.02)


def gpu(dh, s, dual, tensor):
    i, j, w = slg.build(dh, s, dual=dual, tensor=tensor)
    if i.shape[0] == 0:
        return np.zeros((0, 3), np.int64), slg.last_stats()
    st = slg.last_stats()
    return np.stack([i.cpu().numpy(), j.cpu().numpy(), w.cpu().numpy()], 1).astype(np.int64), st


@pytest.fixture(scope="module")
def planted():
    h = hg.lognormal_web(20_000, 40_000, seed=7, cap=2000, core_edges=256,
                         core_vertices=512, core_density=0.3)
    return h, slg.to_device(h)


@pytest.mark.parametrize("dual", [False, True])
@pytest.mark.parametrize("s", [1, 2, 8, 32])
def test_planted_core_matches_oracle(planted, dual, s):
    h, dh = planted
    got, st = gpu(dh, s, dual, True)
    assert st["core_rows"] >= 128, "tile path not taken"
    want = oracle.canonical(*oracle.line_graph_of(h, s, dual=dual, threads=8))
    assert np.array_equal(got, want)
    off, _ = gpu(dh, s, dual, False)
    assert np.array_equal(off, got)


def test_larger_core_and_unweighted(planted):
    h = hg.lognormal_web(60_000, 120_000, seed=8, cap=5000, core_edges=1024,
                         core_vertices=2048, core_density=0.3)
    dh = slg.to_device(h)
    for dual in (False, True):
        got, st = gpu(dh, 16, dual, True)
        assert st["core_rows"] >= 1000
        off, _ = gpu(dh, 16, dual, False)
        assert np.array_equal(got, off)
        i, j, _w = slg.build(dh, 16, dual=dual, tensor=True, unweighted=True)
        assert np.array_equal(np.stack([i.cpu().numpy(), j.cpu().numpy()], 1), got[:, :2])


def test_no_core_leaves_walk_alone():
    h = hg.uniform(5000, 8000, 1, 20, seed=4)
    dh = slg.to_device(h)
    got, st = gpu(dh, 2, False, True)
    assert st["core_rows"] == 0
    want = oracle.canonical(*oracle.line_graph_of(h, 2))
    assert np.array_equal(got, want)
