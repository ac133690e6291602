"""slg_count_noalloc, the entry point for callers that cannot allocate.

Some callers must not allocate device memory during a call: a process whose
device memory is already reserved by another allocator (a framework caching
allocator that holds nearly all of the GPU), or a latency-bound loop where a
cudaMalloc could stall behind the device.  slg_count_noalloc serves them:
its working memory is a fixed array inside the library.  This file checks,
through the C ABI, that it returns exactly the oracle's pair count and what
slg_count returns, on calls in a row (the array keeps the previous call's
contents, so later calls also show that a call starts from a clean state,
including after a call that was refused for a malformed input), weighted and
with the short-circuit, at the documented row limit, that a CSR and CSC that
disagree are refused as slg_count refuses them, and that an input beyond the
array's capacity is refused with its own status.

It is collected last (test_zz_*) so that a run that stops at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import hypergen as hg
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
slg = pytest.importorskip("paper_2010_11448_gb300")

SLG_ERR_INVALID = 1
SLG_ERR_TOO_LARGE = 7
SLG_DUAL, SLG_UNWEIGHTED = 1, 2
MAX_ROWS = 2_094_080  # the largest computed side the fixed array serves


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_11448_gb300 import build_lib
    build_lib.build()
    L = slg.load()
    f = L.slg_count_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32,
                  ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p]
    return L


def noalloc(L, dh, s, flags):
    n = ctypes.c_int64(-1)
    rc = L.slg_count_noalloc(ctypes.byref(dh.struct), s, flags, ctypes.byref(n),
                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, n.value


def with_alloc(L, dh, s, flags):
    n = ctypes.c_int64(-1)
    rc = L.slg_count(ctypes.byref(dh.struct), s, flags, ctypes.byref(n),
                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, n.value


def oracle_count(h, s, flags):
    return oracle.canonical(*oracle.line_graph_of(h, s, dual=bool(flags & SLG_DUAL),
                                                  threads=8)).shape[0]


def test_matches_oracle_and_slg_count_on_calls_in_a_row(lib):
    ha = hg.chung_lu(20_000, 40_000, seed=5, size_cap=2000)
    hb = hg.config("uniform_2k")
    a, b = slg.to_device(ha), slg.to_device(hb)
    # the same inputs twice, then another graph, the dual and the
    # short-circuit: every call matches the oracle and the allocating entry
    # point exactly (integer counts)
    cases = ((ha, a, 2, 0), (ha, a, 2, 0), (hb, b, 3, SLG_DUAL), (ha, a, 4, SLG_DUAL),
             (ha, a, 2, SLG_UNWEIGHTED), (hb, b, 3, SLG_DUAL | SLG_UNWEIGHTED))
    for h, dh, s, flags in cases:
        rc1, n1 = noalloc(lib, dh, s, flags)
        rc2, n2 = with_alloc(lib, dh, s, flags)
        assert rc1 == 0 and rc2 == 0
        assert n1 == n2 == oracle_count(h, s, flags), (s, flags)


def _bad(h, what):
    e_off, e_idx = h.e_off.copy(), h.e_idx.copy()
    v_off, v_idx = h.v_off.copy(), h.v_idx.copy()
    if what == "id_out_of_range":
        e_idx[0] = h.n + 5
    elif what == "csc_mismatch":
        # column 0 names a different hyperedge (still sorted, same nnz)
        v_idx[0] = (v_idx[0] + 1) % h.m
        v_idx[: v_off[1]] = np.sort(v_idx[: v_off[1]])
    return hg.Hypergraph(h.m, h.n, e_off, e_idx, v_off, v_idx)


@pytest.mark.parametrize("what", ["id_out_of_range", "csc_mismatch"])
def test_malformed_input_refused_and_next_call_clean(lib, what):
    h = hg.uniform(3000, 5000, 3, 15, seed=2)
    good = slg.to_device(h)
    bad = slg.to_device(_bad(h, what))
    for flags in (0, SLG_DUAL):
        assert noalloc(lib, bad, 2, flags)[0] == SLG_ERR_INVALID
        assert with_alloc(lib, bad, 2, flags)[0] == SLG_ERR_INVALID
        # the call after a refused one starts clean
        rc, n = noalloc(lib, good, 2, flags)
        assert rc == 0 and n == oracle_count(h, 2, flags) == with_alloc(lib, good, 2, flags)[1]


def test_at_the_row_limit(lib):
    # the dual of 40K hyperedges over exactly MAX_ROWS vertices: the largest
    # computed side the fixed array serves
    h = hg.uniform(40_000, MAX_ROWS, 2, 30, seed=11)
    dh = slg.to_device(h)
    for s, flags in ((3, SLG_DUAL), (3, SLG_DUAL | SLG_UNWEIGHTED)):
        rc, n = noalloc(lib, dh, s, flags)
        assert rc == 0
        assert n == oracle_count(h, s, flags) == with_alloc(lib, dh, s, flags)[1]


def test_rejects_inputs_beyond_its_fixed_memory(lib):
    # 3M isolated vertices on the dual side: more rows than the array serves
    n = 3_000_000
    h = hg.Hypergraph(1, n, np.array([0, 0], np.int32), np.zeros(0, np.int32),
                      np.zeros(n + 1, np.int32), np.zeros(0, np.int32))
    dh = slg.to_device(h)
    rc, _ = noalloc(lib, dh, 2, SLG_DUAL)
    assert rc == SLG_ERR_TOO_LARGE
    assert lib.slg_strerror(rc).decode().startswith("input too large")
    # one row more than the limit is refused too
    h = hg.Hypergraph(1, MAX_ROWS + 1, np.array([0, 0], np.int32), np.zeros(0, np.int32),
                      np.zeros(MAX_ROWS + 2, np.int32), np.zeros(0, np.int32))
    assert noalloc(lib, slg.to_device(h), 2, SLG_DUAL)[0] == SLG_ERR_TOO_LARGE
