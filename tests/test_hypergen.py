"""The seeded generators produce well-formed, reproducible incidences."""
import numpy as np
import pytest

import hypergen as hg


def well_formed(h):
    for off, idx, rows, cols in ((h.e_off, h.e_idx, h.m, h.n),
                                 (h.v_off, h.v_idx, h.n, h.m)):
        assert off.dtype == np.int32 and idx.dtype == np.int32
        assert off.shape == (rows + 1,) and off[0] == 0 and off[-1] == idx.shape[0]
        assert np.all(np.diff(off) >= 0)
        if idx.shape[0]:
            assert idx.min() >= 0 and idx.max() < cols
            owner = np.repeat(np.arange(rows), np.diff(off))
            same = owner[1:] == owner[:-1]
            assert np.all(idx[1:][same] > idx[:-1][same])   # strictly ascending
    # CSC is the transpose of the CSR
    owner = np.repeat(np.arange(h.m), np.diff(h.e_off))
    a = np.lexsort((owner, h.e_idx))
    assert np.array_equal(owner[a], h.v_idx)


@pytest.mark.parametrize("make", [
    lambda: hg.uniform(300, 500, 1, 20, seed=5),
    lambda: hg.chung_lu(3000, 6000, seed=5, size_cap=500),
    lambda: hg.lognormal_web(4000, 9000, seed=5, cap=2000, core_edges=64,
                             core_vertices=128, core_density=0.3),
    lambda: hg.random_small(9),
    lambda: hg.config("uniform_2k"),
])
def test_well_formed_and_reproducible(make):
    a, b = make(), make()
    well_formed(a)
    assert np.array_equal(a.e_idx, b.e_idx) and np.array_equal(a.e_off, b.e_off)


def test_uniform_2k_shape():
    h = hg.config("uniform_2k")
    sizes = np.diff(h.e_off)
    assert h.m == 2000 and h.n == 4000
    assert sizes.min() >= 1 and sizes.max() <= 20
    assert abs(sizes.mean() - 10.5) < 0.5


def test_chung_lu_heavy_tail():
    h = hg.chung_lu(20_000, 40_000, seed=1)
    sizes = np.diff(h.e_off)
    deg = np.diff(h.v_off)
    assert 15 < sizes.mean() < 25            # mean near 20
    assert sizes.max() > 20 * sizes.mean()    # heavy tail
    assert deg.max() > 10 * deg.mean()


def test_planted_core_density():
    h = hg.lognormal_web(6000, 12000, seed=4, cap=1000, core_edges=200,
                         core_vertices=400, core_density=0.3)
    deg = np.diff(h.v_off)
    assert np.sum(deg > 40) >= 380            # core vertices stand out
