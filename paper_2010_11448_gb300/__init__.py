"""slg: s-line graphs of hypergraphs on one GB300 (sm_103a).

Thin Python binding over the C ABI of ``include/slg.h`` (``libslg.so``).
It only marshals arguments: every step of the computation runs in the CUDA
kernels of the library.  There is no CPU fallback; if the compiled library
is missing the functions raise ``RuntimeError``.

PyTorch supplies device memory and streams.  A hypergraph lives on the
device as four int32 tensors (CSR e_off/e_idx and CSC v_off/v_idx, see
``DeviceHypergraph``); results come back as three int32 tensors (i, j, w)
forming the canonical edge list of L_s (i < j, w >= s, ascending (i, j)).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

__all__ = [
    "DeviceHypergraph", "to_device", "count", "build", "build_rows",
    "build_host", "wedges", "last_stats", "set_profiling", "tile_overlap",
    "filter_pairs", "build_sweep", "squeeze", "adjacency", "components", "row_offsets",
    "build_stream",
    "set_core_params", "SLG_TENSOR_CORE", "SLG_RELABEL_ASC", "SLG_RELABEL_DESC",
    "SLG_NO_PRUNE",
    "Plan", "Graph", "alloc_outputs",
    "library_path", "load",
    "SLG_DUAL", "SLG_UNWEIGHTED", "SLG_ALGO_BINNED", "SLG_ALGO_PLAIN",
    "SLG_ALGO_SPGEMM", "SlgError", "ABI_FUNCTIONS",
]

SLG_DUAL = 0x1
SLG_UNWEIGHTED = 0x2
SLG_TENSOR_CORE = 0x4
SLG_RELABEL_ASC = 0x8
SLG_RELABEL_DESC = 0x10
SLG_NO_PRUNE = 0x20
SLG_ASYNC = 0x40
SLG_W16 = 0x80
SLG_ALGO_BINNED = 0x000
SLG_ALGO_PLAIN = 0x100
SLG_ALGO_SPGEMM = 0x200
_ALGOS = {"binned": SLG_ALGO_BINNED, "plain": SLG_ALGO_PLAIN,
          "spgemm": SLG_ALGO_SPGEMM}
_RELABEL = {None: 0, "asc": SLG_RELABEL_ASC, "desc": SLG_RELABEL_DESC}

SLG_ERR_CAPACITY = 2

_HERE = os.path.dirname(os.path.abspath(__file__))


def library_path() -> str:
    return os.path.join(_HERE, "_build", "libslg.so")


class SlgError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        self.where = _last_where() if status == 1 else 0
        at = f", device check {self.where}" if self.where else ""
        super().__init__(f"{what}: {_strerror(status)} (status {status}{at})")


class _Hypergraph(ctypes.Structure):
    _fields_ = [("n_edges", ctypes.c_int32), ("n_vertices", ctypes.c_int32),
                ("nnz", ctypes.c_int64), ("e_off", ctypes.c_void_p),
                ("e_idx", ctypes.c_void_p), ("v_off", ctypes.c_void_p),
                ("v_idx", ctypes.c_void_p)]


class _Stats(ctypes.Structure):
    _fields_ = [("wedges", ctypes.c_int64), ("pairs", ctypes.c_int64),
                ("rows_active", ctypes.c_int64),
                ("rows_bin", ctypes.c_int64 * 5),
                ("wedges_bin", ctypes.c_int64 * 5),
                ("incid_bin", ctypes.c_int64 * 5),
                ("pairs_bin", ctypes.c_int64 * 5),
                ("kernel_launches", ctypes.c_int32),
                ("profiled", ctypes.c_int32),
                ("ms_plan", ctypes.c_float),
                ("ms_walk", ctypes.c_float * 5),
                ("ms_scan", ctypes.c_float),
                ("ms_gather", ctypes.c_float),
                ("core_rows", ctypes.c_int64),
                ("core_cols", ctypes.c_int64),
                ("core_nnz", ctypes.c_int64),
                ("giant_cycles", ctypes.c_int64 * 4),
                ("max_row_work", ctypes.c_int64),
                ("ms_relabel", ctypes.c_float),
                ("ms_order", ctypes.c_float),
                ("sparse_cycles", ctypes.c_int64 * 5),
                ("ms_tile", ctypes.c_float)]


class _Query(ctypes.Structure):
    _fields_ = [("s", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("row_ptr", ctypes.c_void_p), ("out_i", ctypes.c_void_p),
                ("out_j", ctypes.c_void_p), ("out_w", ctypes.c_void_p),
                ("capacity", ctypes.c_int64), ("n_pairs", ctypes.c_int64),
                ("status", ctypes.c_int32)]


_I64P = ctypes.POINTER(ctypes.c_int64)
_VP = ctypes.c_void_p
_HP = ctypes.POINTER(_Hypergraph)

# name -> (restype, argtypes); every symbol include/slg.h declares.
ABI_FUNCTIONS = {
    "slg_count": (ctypes.c_int, [_HP, ctypes.c_int32, ctypes.c_uint32, _I64P, _VP]),
    "slg_count_noalloc": (ctypes.c_int, [_HP, ctypes.c_int32, ctypes.c_uint32, _I64P, _VP]),
    "slg_build": (ctypes.c_int, [_HP, ctypes.c_int32, ctypes.c_uint32, _VP, _VP, _VP,
                                 ctypes.c_int64, _I64P, _VP]),
    "slg_build_rows": (ctypes.c_int, [_HP, ctypes.c_int32, ctypes.c_uint32,
                                      ctypes.c_int32, ctypes.c_int32, _VP, _VP, _VP,
                                      ctypes.c_int64, _I64P, _VP]),
    "slg_build_host": (ctypes.c_int, [_HP, ctypes.c_int32, ctypes.c_uint32, _VP, _VP,
                                      _VP, ctypes.c_int64, _I64P, _VP]),
    "slg_build_csr": (ctypes.c_int, [_HP, ctypes.c_int32, ctypes.c_uint32, _VP, _VP, _VP,
                                     ctypes.c_int64, _I64P, _VP]),
    "slg_build_host_csr": (ctypes.c_int, [_HP, ctypes.c_int32, ctypes.c_uint32, _VP, _VP,
                                          _VP, ctypes.c_int64, _I64P, _VP]),
    "slg_build_host_many": (ctypes.c_int, [_HP, ctypes.POINTER(_Query), ctypes.c_int32,
                                           _VP]),
    "slg_row_work": (ctypes.c_int, [_HP, ctypes.c_int32, ctypes.c_uint32, _VP, _I64P, _VP]),
    "slg_wedges": (ctypes.c_int, [_HP, ctypes.c_int32, ctypes.c_uint32, _I64P, _VP]),
    "slg_row_offsets": (ctypes.c_int, [_HP, ctypes.c_int32, ctypes.c_uint32, _VP, _VP]),
    "slg_last_stats": (ctypes.c_int, [ctypes.POINTER(_Stats)]),
    "slg_set_profiling": (ctypes.c_int, [ctypes.c_int]),
    "slg_release_memory": (ctypes.c_int, []),
    "slg_set_core_params": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_float]),
    "slg_tile_overlap": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32, _VP, _VP]),
    "slg_filter": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64, ctypes.c_int32, _VP, _VP,
                                  _VP, ctypes.c_int64, _I64P, _VP]),
    "slg_build_sweep": (ctypes.c_int, [_HP, _VP, ctypes.c_int32, ctypes.c_uint32, _VP, _VP,
                                       _VP, _VP, _VP, _VP]),
    "slg_squeeze": (ctypes.c_int, [_VP, _VP, ctypes.c_int64, ctypes.c_int32, _VP, _VP, _VP,
                                   ctypes.POINTER(ctypes.c_int32), _VP]),
    "slg_adjacency": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64, ctypes.c_int32, _VP, _VP,
                                     _VP, _VP]),
    "slg_components": (ctypes.c_int, [_VP, _VP, ctypes.c_int64, ctypes.c_int32, _VP, _I64P,
                                      _VP]),
    "slg_plan_create": (ctypes.c_int, [_VP, _VP, ctypes.c_int32, ctypes.c_uint32,
                                       ctypes.POINTER(ctypes.c_void_p), _VP]),
    "slg_plan_execute": (ctypes.c_int, [_VP, _VP]),
    "slg_plan_result": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_void_p),
                                       ctypes.POINTER(ctypes.c_void_p),
                                       ctypes.POINTER(ctypes.c_void_p), _I64P, _VP]),
    "slg_plan_info": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(ctypes.c_float),
                                     ctypes.POINTER(ctypes.c_int32)]),
    "slg_plan_destroy": (ctypes.c_int, [_VP]),
    "slg_graph_create": (ctypes.c_int, [_HP, ctypes.POINTER(ctypes.c_void_p), _VP]),
    "slg_graph_count": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_uint32, _I64P, _VP]),
    "slg_graph_build": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_uint32, _VP, _VP, _VP,
                                       ctypes.c_int64, _I64P, _VP]),
    "slg_graph_destroy": (ctypes.c_int, [_VP]),
    "slg_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "slg_abi_version": (ctypes.c_int, []),
    "slg_last_error_where": (ctypes.c_int, []),
}

_lib = None
_lock = threading.Lock()


def load(path: str | None = None):
    """Load libslg.so (raises RuntimeError if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or library_path()
        if not os.path.exists(p):
            raise RuntimeError(
                f"slg CUDA library not found at {p}; build it with "
                "paper_2010_11448_gb300.build_lib.build() (no CPU fallback exists)")
        lib = ctypes.CDLL(p)
        for name, (res, args) in ABI_FUNCTIONS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        if path is None:
            _lib = lib
        return lib


def _last_where() -> int:
    try:
        return int(load().slg_last_error_where())
    except Exception:  # pragma: no cover - library missing
        return 0


def _strerror(status: int) -> str:
    try:
        return load().slg_strerror(status).decode()
    except Exception:  # pragma: no cover - library missing
        return "unknown"


class DeviceHypergraph:
    """CSR + CSC of H as int32 CUDA tensors (caller-owned device memory)."""

    def __init__(self, m, n, e_off, e_idx, v_off, v_idx):
        self.m, self.n = int(m), int(n)
        self.e_off, self.e_idx, self.v_off, self.v_idx = e_off, e_idx, v_off, v_idx
        self.nnz = int(e_idx.shape[0])
        self._s = _Hypergraph(self.m, self.n, self.nnz, e_off.data_ptr(),
                              e_idx.data_ptr() if self.nnz else 0, v_off.data_ptr(),
                              v_idx.data_ptr() if self.nnz else 0)

    @property
    def struct(self):
        return self._s

    def rows(self, dual: bool) -> int:
        return self.n if dual else self.m


def to_device(h, device="cuda") -> DeviceHypergraph:
    """Copy a host hypergraph (any object with m, n, e_off, e_idx, v_off,
    v_idx numpy arrays) to the device."""
    import torch

    def t(a):
        a = np.ascontiguousarray(a, dtype=np.int32)
        if a.shape[0] == 0:
            return torch.zeros(1, dtype=torch.int32, device=device)[:0]
        return torch.from_numpy(a).to(device)

    return DeviceHypergraph(h.m, h.n, t(h.e_off), t(h.e_idx), t(h.v_off), t(h.v_idx))


def _flags(dual, unweighted, algo, tensor=False, relabel=None, prune=True):
    f = _ALGOS[algo] | _RELABEL[relabel] | (0 if prune else SLG_NO_PRUNE)
    if tensor:
        f |= SLG_TENSOR_CORE
    if dual:
        f |= SLG_DUAL
    if unweighted:
        f |= SLG_UNWEIGHTED
    return f


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def count(h: DeviceHypergraph, s: int, dual=False, unweighted=False,
          algo="binned", stream=None, tensor=False, relabel=None, prune=True) -> int:
    """|L_s(H)| (or of H* with dual=True)."""
    n = ctypes.c_int64(0)
    rc = load().slg_count(ctypes.byref(h.struct), int(s),
                          _flags(dual, unweighted, algo, tensor, relabel, prune),
                          ctypes.byref(n), _stream(stream))
    if rc != 0:
        raise SlgError(rc, "slg_count")
    return int(n.value)


def alloc_outputs(capacity, unweighted=False, device="cuda"):
    """Three int32 device tensors of `capacity` entries for build(out=...)."""
    return _outputs(capacity, unweighted, device)


def _outputs(capacity, unweighted, device):
    import torch
    cap = max(int(capacity), 1)
    oi = torch.empty(cap, dtype=torch.int32, device=device)
    oj = torch.empty(cap, dtype=torch.int32, device=device)
    ow = None if unweighted else torch.empty(cap, dtype=torch.int32, device=device)
    return oi, oj, ow


def build(h: DeviceHypergraph, s: int, dual=False, unweighted=False,
          algo="binned", capacity=None, out=None, stream=None, tensor=False,
          relabel=None, prune=True):
    """The canonical edge list of L_s as int32 tensors (i, j, w); w is None
    with unweighted=True.  Without ``capacity``/``out`` the pair count is
    taken first with ``count`` (an extra walk).  tensor=True counts a dense
    core block on the tensor cores; relabel="asc"/"desc" renumbers the rows
    by size for the walk; prune=False switches off the degree-based pruning
    (all give the same result)."""
    flags = _flags(dual, unweighted, algo, tensor, relabel, prune)
    if out is None:
        if capacity is None:
            capacity = count(h, s, dual, unweighted, algo, stream, tensor)
        out = _outputs(capacity, unweighted, h.e_off.device)
    oi, oj, ow = out
    cap = int(oi.shape[0])
    n = ctypes.c_int64(0)
    rc = load().slg_build(ctypes.byref(h.struct), int(s), flags, oi.data_ptr(),
                          oj.data_ptr(), ow.data_ptr() if ow is not None else None,
                          cap, ctypes.byref(n), _stream(stream))
    if rc != 0:
        err = SlgError(rc, "slg_build")
        err.needed = int(n.value)  # |L_s| when the capacity was too small
        raise err
    p = int(n.value)
    return oi[:p], oj[:p], (ow[:p] if ow is not None else None)


def build_rows(h: DeviceHypergraph, s: int, row_begin: int, row_end: int,
               dual=False, unweighted=False, algo="binned", capacity=0,
               out=None, stream=None):
    """Rows [row_begin, row_end) of the edge list.  Returns (i, j, w) or
    raises SlgError with status 2 (capacity) carrying the needed count in
    ``.needed``."""
    flags = _flags(dual, unweighted, algo)
    if out is None:
        out = _outputs(capacity, unweighted, h.e_off.device)
    oi, oj, ow = out
    n = ctypes.c_int64(0)
    rc = load().slg_build_rows(ctypes.byref(h.struct), int(s), flags, int(row_begin),
                               int(row_end), oi.data_ptr(), oj.data_ptr(),
                               ow.data_ptr() if ow is not None else None,
                               int(oi.shape[0]) if capacity else 0, ctypes.byref(n),
                               _stream(stream))
    if rc != 0:
        err = SlgError(rc, "slg_build_rows")
        err.needed = int(n.value)
        raise err
    p = int(n.value)
    return oi[:p], oj[:p], (ow[:p] if ow is not None else None)


def build_host(h, s: int, dual=False, unweighted=False, algo="binned",
               capacity: int = 0, out=None, stream=None, relabel=None, wait=True):
    """End-to-end from host arrays: ``h`` holds numpy (ideally pinned torch
    CPU) int32 arrays; the library copies them in, builds, copies back.
    ``out`` = three host int32 arrays of the same capacity.  wait=False
    (SLG_ASYNC) returns once the copies back are enqueued on ``stream``: the
    arrays are filled when that stream's work completes."""
    def ptr(a):
        if hasattr(a, "data_ptr"):
            return a.data_ptr()
        return a.ctypes.data
    st = _Hypergraph(int(h.m), int(h.n), int(h.e_idx.shape[0]), ptr(h.e_off),
                     ptr(h.e_idx), ptr(h.v_off), ptr(h.v_idx))
    if out is None:
        cap = max(int(capacity), 1)
        out = (np.empty(cap, np.int32), np.empty(cap, np.int32),
               None if unweighted else np.empty(cap, np.int32))
    oi, oj, ow = out
    n = ctypes.c_int64(0)
    flags = _flags(dual, unweighted, algo, relabel=relabel) | (0 if wait else SLG_ASYNC)
    rc = load().slg_build_host(ctypes.byref(st), int(s), flags,
                               ptr(oi), ptr(oj), ptr(ow) if ow is not None else None,
                               int(oi.shape[0]), ctypes.byref(n), _stream(stream))
    if rc != 0:
        err = SlgError(rc, "slg_build_host")
        err.needed = int(n.value)
        raise err
    p = int(n.value)
    return oi[:p], oj[:p], (ow[:p] if ow is not None else None)


def build_csr(h: DeviceHypergraph, s: int, dual=False, unweighted=False, algo="binned",
              capacity=None, out=None, stream=None, tensor=False, prune=True):
    """L_s in compressed row form: (row_ptr int64 [R + 1], j, w) device
    tensors; row i's pairs are j[row_ptr[i]:row_ptr[i + 1]] (w None with
    unweighted=True)."""
    import torch
    flags = _flags(dual, unweighted, algo, tensor, None, prune)
    R = h.rows(dual)
    if out is None:
        if capacity is None:
            capacity = count(h, s, dual, unweighted, algo, stream, tensor)
        _, oj, ow = _outputs(capacity, unweighted, h.e_off.device)
        ptr = torch.empty(R + 1, dtype=torch.int64, device=h.e_off.device)
    else:
        ptr, oj, ow = out
    n = ctypes.c_int64(0)
    rc = load().slg_build_csr(ctypes.byref(h.struct), int(s), flags, ptr.data_ptr(),
                              oj.data_ptr(), ow.data_ptr() if ow is not None else None,
                              int(oj.shape[0]), ctypes.byref(n), _stream(stream))
    if rc != 0:
        err = SlgError(rc, "slg_build_csr")
        err.needed = int(n.value)
        raise err
    p = int(n.value)
    return ptr, oj[:p], (ow[:p] if ow is not None else None)


def _host_struct(h):
    def ptr(a):
        if hasattr(a, "data_ptr"):
            return a.data_ptr()
        return a.ctypes.data
    return _Hypergraph(int(h.m), int(h.n), int(h.e_idx.shape[0]), ptr(h.e_off),
                       ptr(h.e_idx), ptr(h.v_off), ptr(h.v_idx))


def _hptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def build_host_many(h, queries, stream=None):
    """Several builds of one host hypergraph (slg_build_host_many): the
    incidence is copied to the device once and each result is copied back
    while the next is built.  ``queries``: dicts with keys s, dual,
    unweighted (optional), algo (optional), w16 (optional: out_w is a
    16-bit host array and receives the weights as uint16), capacity, and
    host arrays row_ptr (int64[R + 1]; compressed row form) or out_i, plus
    out_j, out_w.  Returns a list of (status, n_pairs)."""
    qs = (_Query * len(queries))()
    for k, q in enumerate(queries):
        qs[k].s = int(q["s"])
        qs[k].flags = _flags(q.get("dual", False), q.get("unweighted", False),
                             q.get("algo", "binned")) | (SLG_W16 if q.get("w16") else 0)
        qs[k].row_ptr = _hptr(q.get("row_ptr"))
        qs[k].out_i = _hptr(q.get("out_i"))
        qs[k].out_j = _hptr(q.get("out_j"))
        qs[k].out_w = _hptr(q.get("out_w"))
        qs[k].capacity = int(q["capacity"])
    st = _host_struct(h)
    load().slg_build_host_many(ctypes.byref(st), qs, len(queries), _stream(stream))
    return [(int(q.status), int(q.n_pairs)) for q in qs]


def row_offsets(h: DeviceHypergraph, s: int, dual=False, unweighted=False, stream=None,
                tensor=False, prune=True):
    """int64 CUDA tensor [R + 1]: where each row's pairs start in the
    canonical edge list (slg_row_offsets)."""
    import torch
    R = h.rows(dual)
    ptr = torch.empty(R + 1, dtype=torch.int64, device=h.e_off.device)
    rc = load().slg_row_offsets(ctypes.byref(h.struct), int(s),
                                _flags(dual, unweighted, "binned", tensor, None, prune),
                                ptr.data_ptr(), _stream(stream))
    if rc != 0:
        raise SlgError(rc, "slg_row_offsets")
    return ptr


def build_stream(h: DeviceHypergraph, s: int, max_pairs: int, dual=False, unweighted=False,
                 stream=None, tensor=False):
    """The canonical edge list in consecutive row ranges of at most
    ``max_pairs`` pairs each (a single larger row forms its own range).
    Yields (row_begin, row_end, i, j, w); the tensors are views of one
    output buffer that the next chunk overwrites."""
    import numpy as np
    ptr = row_offsets(h, s, dual, unweighted, stream, tensor).cpu().numpy()
    R = len(ptr) - 1
    biggest = int(np.diff(ptr).max()) if R else 0
    out = _outputs(max(int(max_pairs), biggest), unweighted, h.e_off.device)
    flags = _flags(dual, unweighted, "binned", tensor)
    a = 0
    while a < R:
        b = int(np.searchsorted(ptr, ptr[a] + max_pairs, side="right")) - 1
        b = min(max(b, a + 1), R)
        n = ctypes.c_int64(0)
        rc = load().slg_build_rows(ctypes.byref(h.struct), int(s), flags, a, b,
                                   out[0].data_ptr(), out[1].data_ptr(),
                                   out[2].data_ptr() if out[2] is not None else None,
                                   int(out[0].shape[0]), ctypes.byref(n), _stream(stream))
        if rc != 0:
            raise SlgError(rc, "slg_build_rows")
        p = int(n.value)
        yield a, b, out[0][:p], out[1][:p], (out[2][:p] if out[2] is not None else None)
        a = b


def row_work(h: DeviceHypergraph, s: int, dual=False, stream=None, prune=True):
    """int32 CUDA tensor [R]: the wedge work of every row (slg_row_work)."""
    import torch
    R = h.rows(dual)
    work = torch.empty(max(R, 1), dtype=torch.int32, device=h.e_off.device)
    n = ctypes.c_int64(0)
    rc = load().slg_row_work(ctypes.byref(h.struct), int(s),
                             _flags(dual, False, "binned", False, None, prune),
                             work.data_ptr(), ctypes.byref(n), _stream(stream))
    if rc != 0:
        raise SlgError(rc, "slg_row_work")
    return work[:R]


def wedges(h: DeviceHypergraph, s: int, dual=False, stream=None) -> int:
    """W_s: the upper-triangle wedges the walk visits after the size filter."""
    n = ctypes.c_int64(0)
    rc = load().slg_wedges(ctypes.byref(h.struct), int(s), _flags(dual, False, "binned"),
                           ctypes.byref(n), _stream(stream))
    if rc != 0:
        raise SlgError(rc, "slg_wedges")
    return int(n.value)


def filter_pairs(i, j, w, s: int, out=None, stream=None, weights=True):
    """L_s from a canonical weighted edge list (i, j, w) of any L_s' with
    s' <= s: the triples with w >= s, in order (slg_filter)."""
    n = int(i.shape[0])
    if out is None:
        cnt = ctypes.c_int64(0)
        rc = load().slg_filter(i.data_ptr(), j.data_ptr(), w.data_ptr(), n, int(s), None, None,
                               None, 0, ctypes.byref(cnt), _stream(stream))
        if rc not in (0, SLG_ERR_CAPACITY):
            raise SlgError(rc, "slg_filter")
        out = _outputs(cnt.value, not weights, i.device)
    oi, oj, ow = out
    cnt = ctypes.c_int64(0)
    rc = load().slg_filter(i.data_ptr(), j.data_ptr(), w.data_ptr(), n, int(s), oi.data_ptr(),
                           oj.data_ptr(), ow.data_ptr() if ow is not None else None,
                           int(oi.shape[0]), ctypes.byref(cnt), _stream(stream))
    if rc != 0:
        err = SlgError(rc, "slg_filter")
        err.needed = int(cnt.value)
        raise err
    p = int(cnt.value)
    return oi[:p], oj[:p], (ow[:p] if ow is not None else None)


def build_sweep(h: DeviceHypergraph, s_list, dual=False, algo="binned", outs=None,
                stream=None, tensor=False, relabel=None):
    """L_s for every s in s_list from one walk at min(s_list) (slg_build_sweep).
    ``outs``: one (i, j, w) tensor triple per threshold; without it the lists
    are sized by slg_count at each threshold.  Returns a list of triples."""
    s_list = [int(x) for x in s_list]
    k = len(s_list)
    if outs is None:
        outs = [_outputs(count(h, x, dual, False, algo, stream, tensor), False, h.e_off.device)
                for x in s_list]
    arr = lambda vals, t: (t * k)(*vals)
    oi = arr([o[0].data_ptr() for o in outs], ctypes.c_void_p)
    oj = arr([o[1].data_ptr() for o in outs], ctypes.c_void_p)
    ow = arr([o[2].data_ptr() if o[2] is not None else None for o in outs], ctypes.c_void_p)
    cap = arr([int(o[0].shape[0]) for o in outs], ctypes.c_int64)
    np_ = (ctypes.c_int64 * k)()
    sv = arr(s_list, ctypes.c_int32)
    rc = load().slg_build_sweep(ctypes.byref(h.struct), sv, k,
                                _flags(dual, False, algo, tensor, relabel), oi, oj, ow, cap,
                                np_, _stream(stream))
    if rc != 0:
        err = SlgError(rc, "slg_build_sweep")
        err.needed = list(np_)
        raise err
    res = []
    for (a, b, c), p in zip(outs, list(np_)):
        res.append((a[:p], b[:p], c[:p] if c is not None else None))
    return res


def _ptr(t):
    return t.data_ptr() if t is not None and t.numel() else None


def squeeze(i, j, R: int, stream=None):
    """ID squeezing: (i', j', old_of_new) with the ids of the list renumbered
    0 .. n_ids-1 in ascending order of their original id."""
    import torch
    n = int(i.shape[0])
    oi = torch.empty(max(n, 1), dtype=torch.int32, device=i.device)
    oj = torch.empty(max(n, 1), dtype=torch.int32, device=i.device)
    old = torch.empty(max(int(R), 1), dtype=torch.int32, device=i.device)
    k = ctypes.c_int32(0)
    rc = load().slg_squeeze(_ptr(i), _ptr(j), n, int(R), oi.data_ptr(), oj.data_ptr(),
                            old.data_ptr(), ctypes.byref(k), _stream(stream))
    if rc != 0:
        raise SlgError(rc, "slg_squeeze")
    return oi[:n], oj[:n], old[:k.value]


def adjacency(i, j, w, V: int, weights=True, stream=None):
    """Symmetric CSR (off int64 [V+1], adj int32 [2n], adj_w or None) of the
    line graph from a canonical list over V vertices."""
    import torch
    n = int(i.shape[0])
    off = torch.empty(int(V) + 1, dtype=torch.int64, device=i.device)
    adj = torch.empty(max(2 * n, 1), dtype=torch.int32, device=i.device)
    adj_w = torch.empty(max(2 * n, 1), dtype=torch.int32, device=i.device) if weights else None
    rc = load().slg_adjacency(_ptr(i), _ptr(j), _ptr(w) if weights else None, n, int(V),
                              off.data_ptr(), adj.data_ptr(),
                              adj_w.data_ptr() if weights else None, _stream(stream))
    if rc != 0:
        raise SlgError(rc, "slg_adjacency")
    return off, adj[:2 * n], (adj_w[:2 * n] if weights else None)


def components(i, j, R: int, stream=None):
    """(labels [R], n_components): the smallest id of each id's component in
    L_s, and the number of components among the ids of the list."""
    import torch
    n = int(i.shape[0])
    labels = torch.empty(max(int(R), 1), dtype=torch.int32, device=i.device)
    k = ctypes.c_int64(0)
    rc = load().slg_components(_ptr(i), _ptr(j), n, int(R), labels.data_ptr(),
                               ctypes.byref(k), _stream(stream))
    if rc != 0:
        raise SlgError(rc, "slg_components")
    return labels[:int(R)], int(k.value)


def last_stats() -> dict:
    st = _Stats()
    load().slg_last_stats(ctypes.byref(st))
    return {"wedges": st.wedges, "pairs": st.pairs, "rows_active": st.rows_active,
            "rows_bin": list(st.rows_bin), "wedges_bin": list(st.wedges_bin),
            "incid_bin": list(st.incid_bin), "pairs_bin": list(st.pairs_bin),
            "kernel_launches": st.kernel_launches, "profiled": bool(st.profiled),
            "ms_plan": st.ms_plan, "ms_walk": list(st.ms_walk), "ms_scan": st.ms_scan,
            "ms_gather": st.ms_gather, "core_rows": st.core_rows, "core_cols": st.core_cols,
            "core_nnz": st.core_nnz, "giant_cycles": list(st.giant_cycles),
            "max_row_work": st.max_row_work, "ms_relabel": st.ms_relabel,
            "ms_order": st.ms_order, "sparse_cycles": list(st.sparse_cycles),
            "ms_tile": st.ms_tile}


def set_core_params(tau_c: int = 64, tau_r: int = 32, min_density: float = 0.02) -> None:
    """Dense-core selection used by tensor=True on this thread."""
    rc = load().slg_set_core_params(int(tau_c), int(tau_r), float(min_density))
    if rc != 0:
        raise SlgError(rc, "slg_set_core_params")


def tile_overlap(A, stream=None):
    """C = A·Aᵀ on the tensor cores for a dense 0/1 block.  ``A`` is a CUDA
    uint8 tensor [rows_pad, cols_pad] (0x38 = 1, 0 = 0), both dimensions
    multiples of 128; returns the int32 [rows_pad, rows_pad] tensor whose
    tiles on and above the diagonal hold the overlap counts (others 0)."""
    import torch
    rows, cols = int(A.shape[0]), int(A.shape[1])
    C = torch.zeros((rows, rows), dtype=torch.int32, device=A.device)
    rc = load().slg_tile_overlap(A.data_ptr(), rows, cols, C.data_ptr(), _stream(stream))
    if rc != 0:
        raise SlgError(rc, "slg_tile_overlap")
    return C


class _DeviceInt32:
    """A device int32 array owned by the library, seen through the CUDA
    array interface (no copy until .clone())."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<i4",
                                         "data": (ptr, False), "version": 3}


class Graph:
    """A device hypergraph prepared for several calls (slg_graph_*): the
    input is validated and both sides' CSR->CSC maps are made once, in
    ``Graph(h)``; ``count`` and ``build`` then take the same arguments as the
    module-level functions (binned or plain algorithm, either side) and skip
    that work.  ``close()`` (or the context manager) releases it; ``h`` must
    stay alive and unchanged meanwhile."""

    def __init__(self, h: DeviceHypergraph, stream=None):
        self.h = h
        self._g = ctypes.c_void_p()
        rc = load().slg_graph_create(ctypes.byref(h.struct), ctypes.byref(self._g),
                                     _stream(stream))
        if rc != 0:
            raise SlgError(rc, "slg_graph_create")

    def count(self, s: int, dual=False, unweighted=False, algo="binned", stream=None,
              tensor=False, prune=True) -> int:
        n = ctypes.c_int64(0)
        rc = load().slg_graph_count(self._g, int(s),
                                    _flags(dual, unweighted, algo, tensor, None, prune),
                                    ctypes.byref(n), _stream(stream))
        if rc != 0:
            raise SlgError(rc, "slg_graph_count")
        return int(n.value)

    def build(self, s: int, dual=False, unweighted=False, algo="binned", capacity=None,
              out=None, stream=None, tensor=False, prune=True):
        flags = _flags(dual, unweighted, algo, tensor, None, prune)
        if out is None:
            if capacity is None:
                capacity = self.count(s, dual, unweighted, algo, stream, tensor, prune)
            out = _outputs(capacity, unweighted, self.h.e_off.device)
        oi, oj, ow = out
        n = ctypes.c_int64(0)
        rc = load().slg_graph_build(self._g, int(s), flags, oi.data_ptr(), oj.data_ptr(),
                                    ow.data_ptr() if ow is not None else None,
                                    int(oi.shape[0]), ctypes.byref(n), _stream(stream))
        if rc != 0:
            err = SlgError(rc, "slg_graph_build")
            err.needed = int(n.value)
            raise err
        p = int(n.value)
        return oi[:p], oj[:p], (ow[:p] if ow is not None else None)

    def close(self):
        if self._g:
            load().slg_graph_destroy(self._g)
            self._g = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """A batch of hypergraphs (each with its own s) built by one captured
    pipeline: ``Plan(graphs, s)``, then ``execute()`` (one CUDA-graph launch)
    and ``results()`` -> list of (i, j, w) tensors per member (member ids)."""

    def __init__(self, graphs, s, dual=False, unweighted=False, stream=None):
        import torch
        self._graphs = list(graphs)          # keep device arrays alive
        self.count = len(self._graphs)
        arr = (_Hypergraph * self.count)(*[g.struct for g in self._graphs])
        sv = (ctypes.c_int32 * self.count)(*[int(x) for x in s])
        self._h = ctypes.c_void_p()
        self.flags = _flags(dual, unweighted, "binned")
        self.unweighted = unweighted
        rc = load().slg_plan_create(ctypes.cast(arr, ctypes.c_void_p),
                                    ctypes.cast(sv, ctypes.c_void_p), self.count, self.flags,
                                    ctypes.byref(self._h), _stream(stream))
        if rc != 0:
            raise SlgError(rc, "slg_plan_create")
        self.device = self._graphs[0].e_off.device
        del torch

    def execute(self, stream=None):
        rc = load().slg_plan_execute(self._h, _stream(stream))
        if rc != 0:
            raise SlgError(rc, "slg_plan_execute")

    def info(self):
        b = (ctypes.c_int32 * 6)()
        ms = ctypes.c_float(0)
        n = ctypes.c_int32(0)
        load().slg_plan_info(self._h, ctypes.cast(b, ctypes.c_void_p), ctypes.byref(ms),
                             ctypes.byref(n))
        return {"bins": list(b), "tuned_ms": ms.value, "launches": n.value}

    def results(self):
        """Per-member (i, j, w) as int32 CUDA tensors (copies)."""
        import torch
        pi, pj, pw = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        n = ctypes.c_int64(0)
        offs = (ctypes.c_int64 * (self.count + 1))()
        torch.cuda.synchronize(self.device)
        rc = load().slg_plan_result(self._h, ctypes.byref(pi), ctypes.byref(pj),
                                    ctypes.byref(pw), ctypes.byref(n),
                                    ctypes.cast(offs, ctypes.c_void_p))
        if rc != 0:
            raise SlgError(rc, "slg_plan_result")
        total = int(n.value)

        def view(ptr):
            if total == 0 or not ptr.value:
                return None
            return torch.as_tensor(_DeviceInt32(ptr.value, total), device=self.device).clone()
        I, J, W = view(pi), view(pj), None if self.unweighted else view(pw)
        out = []
        for g in range(self.count):
            a, b = int(offs[g]), int(offs[g + 1])
            if I is None:
                z = torch.zeros(0, dtype=torch.int32, device=self.device)
                out.append((z, z, None if self.unweighted else z))
            else:
                out.append((I[a:b], J[a:b], None if W is None else W[a:b]))
        return out

    def close(self):
        if self._h:
            load().slg_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def release_memory() -> None:
    """Give the library's cached device memory back (slg_release_memory)."""
    rc = load().slg_release_memory()
    if rc != 0:
        raise SlgError(rc, "slg_release_memory")


def set_profiling(enable: bool) -> None:
    """Per-phase CUDA-event timing of later calls on this thread."""
    load().slg_set_profiling(1 if enable else 0)
