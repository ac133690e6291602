"""slg_count_noalloc, the entry point for callers that cannot allocate.

Some callers must not allocate device memory during a call: a process whose
device memory is already reserved by another allocator (a framework caching
allocator that holds nearly all of the GPU), or a latency-bound loop where a
cudaMalloc could stall behind the device.  slg_count_noalloc serves them:
its working memory is a fixed array inside the library.  This file checks,
through the C ABI, that it returns exactly what slg_count returns, on two
calls in a row (the array keeps the previous call's contents, so the second
call also shows that the call clears what must start at zero), and that an
input beyond the array's capacity is refused with its own status.

It is collected last (test_zz_*) so that a run that stops at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import hypergen as hg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
slg = pytest.importorskip("paper_2010_11448_gb300")

SLG_ERR_TOO_LARGE = 7


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


def test_matches_slg_count_on_two_calls_in_a_row(lib):
    a = slg.to_device(hg.chung_lu(20_000, 40_000, seed=5, size_cap=2000))
    b = slg.to_device(hg.config("uniform_2k"))
    # the same inputs twice, then another graph and the dual: every call
    # must match the allocating entry point exactly (integer counts)
    for dh, s, flags in ((a, 2, 0), (a, 2, 0), (b, 3, 1), (a, 4, 1)):
        rc1, n1 = noalloc(lib, dh, s, flags)
        rc2, n2 = with_alloc(lib, dh, s, flags)
        assert rc1 == 0 and rc2 == 0
        assert n1 == n2


def test_rejects_inputs_beyond_its_fixed_memory(lib):
    # 3M isolated vertices on the dual side: more rows than the array serves
    n = 3_000_000
    h = hg.Hypergraph(1, n, np.array([0, 0], np.int32), np.zeros(0, np.int32),
                      np.zeros(n + 1, np.int32), np.zeros(0, np.int32))
    dh = slg.to_device(h)
    rc, _ = noalloc(lib, dh, 2, 1)
    assert rc == SLG_ERR_TOO_LARGE
    assert lib.slg_strerror(rc).decode().startswith("input too large")
