"""slg_row_work and the row-range split on the GPU: the per-row wedge work
equals its definition, and ranges cut by balanced work (as every rank of a
multi-GPU build would cut them), built with slg_build_rows, concatenate to
the oracle's list; build_sharded on a single rank is the whole build."""
import numpy as np
import pytest

import hypergen as hg
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
slg = pytest.importorskip("paper_2010_11448_gb300")
from paper_2010_11448_gb300 import shard  # noqa: E402
from test_shard_cpu import row_work_by_definition  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_11448_gb300 import build_lib
    build_lib.build()
    slg.load()


def as_np(i, j, w):
    return np.stack([i.cpu().numpy(), j.cpu().numpy(), w.cpu().numpy()], 1).astype(np.int64)


@pytest.mark.parametrize("dual", [False, True])
def test_row_work_and_balanced_ranges(dual):
    h = hg.chung_lu(6000, 12000, seed=17, size_cap=1500)
    dh = slg.to_device(h)
    for s in (2, 4):
        work = slg.row_work(dh, s, dual).cpu().numpy()
        assert np.array_equal(work, row_work_by_definition(h, s, dual))
        want = oracle.canonical(*oracle.line_graph_of(h, s, dual=dual, threads=8))
        for parts in (3, 5):
            b = shard.balanced_ranges(work, parts)
            got = [as_np(*slg.build_rows(dh, s, b[k], b[k + 1], dual=dual,
                                         capacity=want.shape[0] + 1)) for k in range(parts)]
            assert np.array_equal(np.concatenate(got), want)
        off, rng, i, j, w, total = shard.build_sharded(dh, s, 0, 1, dual=dual)
        assert off == 0 and rng == (0, h.n if dual else h.m) and total == want.shape[0]
        assert np.array_equal(as_np(i, j, w), want)
