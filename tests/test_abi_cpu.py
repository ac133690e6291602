"""The C-ABI library builds, loads and exports every declared entry point
(no device calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:int|const char|void)\s*\**\s*(slg_\w+)\s*\(",
                                text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2010_11448_gb300 import build_lib
    path = build_lib.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("slg_count", "slg_build", "slg_build_rows", "slg_build_host",
                 "slg_wedges", "slg_strerror"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    import paper_2010_11448_gb300 as slg
    assert set(declared_functions()) == set(slg.ABI_FUNCTIONS)


def test_binding_constants_match_header():
    import paper_2010_11448_gb300 as slg
    text = open(os.path.join(ROOT, "include", "slg.h")).read()
    defs = dict(re.findall(r"^#define (SLG_\w+) (0x[0-9A-Fa-f]+|-?\d+)u?\b", text, flags=re.M))
    defs.update(re.findall(r"^\s+(SLG_\w+) = (\d+),?", text, flags=re.M))  # slg_status
    assert "SLG_ASYNC" in defs and "SLG_ERR_CAPACITY" in defs
    for name, val in defs.items():
        if hasattr(slg, name):
            assert getattr(slg, name) == int(val, 0), name


def test_host_only_calls(lib):
    import paper_2010_11448_gb300 as slg
    L = slg.load()
    assert L.slg_abi_version() == 8
    assert L.slg_strerror(2).decode().startswith("output capacity")
    # argument checks run on the host before any device work
    n = ctypes.c_int64(0)
    assert L.slg_count(None, 2, 0, ctypes.byref(n), None) == 1


def test_async_flag_only_for_host_builds(lib):
    # flag checks run on the host before any device work: SLG_ASYNC is
    # accepted by slg_build_host alone (the others reject it as invalid)
    import paper_2010_11448_gb300 as slg
    L = slg.load()
    dummy = ctypes.c_void_p(16)  # never dereferenced: the calls stop at the flag check
    h = slg._Hypergraph(3, 4, 5, dummy, dummy, dummy, dummy)
    n = ctypes.c_int64(0)
    assert L.slg_count(ctypes.byref(h), 2, slg.SLG_ASYNC, ctypes.byref(n), None) == 1
    assert L.slg_build(ctypes.byref(h), 2, slg.SLG_ASYNC, None, None, None, 0,
                       ctypes.byref(n), None) == 1
    # with SLG_ASYNC the host entry point still checks its own arguments
    assert L.slg_build_host(ctypes.byref(h), 0, slg.SLG_ASYNC, None, None, None, 0,
                            ctypes.byref(n), None) == 1  # s < 1
    assert L.slg_build_host(ctypes.byref(h), 2, slg.SLG_ASYNC | 0x80, None, None, None, 0,
                            ctypes.byref(n), None) == 1  # unknown flag


def test_missing_library_fails_loudly(tmp_path):
    import paper_2010_11448_gb300 as slg
    with pytest.raises(RuntimeError):
        slg.load(str(tmp_path / "nope.so"))
