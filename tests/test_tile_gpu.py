"""The tensor-core tile path (tcgen05, FP8 0/1 operands, FP32 accumulate)
against an exact integer product, on and above the diagonal tiles."""
import numpy as np
import pytest

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


def run(bits):
    A = torch.from_numpy(np.where(bits, 0x38, 0).astype(np.uint8)).cuda()
    return slg.tile_overlap(A).cpu().numpy()


@pytest.mark.parametrize("rows,cols,p,seed", [(128, 128, 0.5, 0), (256, 384, 0.3, 1),
                                              (384, 1024, 0.1, 2), (512, 8192, 0.3, 3)])
def test_matches_integer_product(rows, cols, p, seed):
    rng = np.random.default_rng(seed)
    bits = rng.random((rows, cols)) < p
    got = run(bits)
    want = bits.astype(np.int64) @ bits.T.astype(np.int64)
    nt = rows // 128
    for bi in range(nt):
        for bj in range(nt):
            blk = (slice(bi * 128, bi * 128 + 128), slice(bj * 128, bj * 128 + 128))
            if bj >= bi:
                assert np.array_equal(got[blk], want[blk]), (bi, bj)
            else:
                assert not got[blk].any()


def test_ragged_block_zero_padding():
    # a 300 x 500 block padded to 384 x 512 with zeros: counts are unchanged
    rng = np.random.default_rng(9)
    bits = np.zeros((384, 512), dtype=bool)
    bits[:300, :500] = rng.random((300, 500)) < 0.25
    got = run(bits)
    want = bits.astype(np.int64) @ bits.T.astype(np.int64)
    iu = np.triu_indices(384)
    assert np.array_equal(got[iu][want[iu] >= 0], want[iu])


def test_bad_shapes_rejected():
    A = torch.zeros((100, 128), dtype=torch.uint8, device="cuda")
    with pytest.raises(slg.SlgError) as ei:
        slg.tile_overlap(A)
    assert ei.value.status == 1
