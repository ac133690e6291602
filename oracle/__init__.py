"""CPU oracle for s-overlaps and s-line graphs L_s(H).

TEST INFRASTRUCTURE ONLY.  Only the tests, the harness smoke check and the
benchmark's CPU-baseline leg import this package; the CUDA library never
does, and the two share no code (the seeded input generators in ``hypergen``
are the only common module, and they hold none of the method's arithmetic).

Definition followed (Section III): the s-line graph L_s(H) has one node per
hyperedge and an edge {e_i, e_j}, i != j, of weight w_ij = |e_i ∩ e_j|
whenever w_ij >= s.  Canonical form used everywhere: triples (i, j, w) with
i < j, sorted by (i, j).  The dual H* (Section III) swaps the roles of
vertices and hyperedges; ``transpose`` builds its incidence here.

Three independent ways to compute the same set:

* ``line_graph``   -- Mode A, wedge counting in plain C (Algorithm 2 with
                      the strict upper triangle of Algorithm 3, no pruning);
* ``brute_force``  -- Mode B, every pair i < j intersected as Python sets
                      (the naive all-pairs method of Section IV-A);
* ``spgemm_scipy`` -- Mode C, the linear-algebra form of Section IV-D: the
                      off-diagonal upper triangle of B·Bᵀ, B the m x n
                      hyperedge-by-vertex 0/1 matrix, kept where >= s.

``wedges`` gives the exact work of the s-filtered walk in closed form,
sum over vertices of C(d_s(v), 2) with d_s(v) the number of hyperedges of
size >= s containing v.

After the edge list, by their plain definitions:

* ``squeeze``     -- ID squeezing (Section IV-E): the ids occurring in the
                     list, renumbered in ascending order;
* ``adjacency``   -- the symmetric CSR of L_s, rows ascending;
* ``components``  -- connected components of L_s (s-connected components,
                     Section I), each id labelled by the smallest id of its
                     component; scipy's graph search is the library step.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "slg_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libslg_oracle.so")
_lock = threading.Lock()
_lib = None

I32P = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (host code only, portable flags)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or \
            os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                               "-pthread", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load(path: str | None = None):
    global _lib
    with _lock:
        if path is not None:
            lib = ctypes.CDLL(path)
        elif _lib is not None:
            return _lib
        else:
            lib = ctypes.CDLL(build())
        f = lib.slg_oracle_line_graph
        f.restype = ctypes.c_int64
        f.argtypes = [ctypes.c_int32, ctypes.c_int32, I32P, I32P,
                      ctypes.c_int32, I32P, ctypes.c_int64, ctypes.c_int32,
                      ctypes.POINTER(I32P), ctypes.POINTER(I32P),
                      ctypes.POINTER(I32P), ctypes.POINTER(ctypes.c_int64)]
        lib.slg_oracle_free.argtypes = [ctypes.c_void_p]
        lib.slg_oracle_free.restype = None
        if path is None:
            _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(I32P)


def line_graph(m: int, n: int, e_off: np.ndarray, e_idx: np.ndarray, s: int,
               rows: np.ndarray | None = None, threads: int = 1,
               lib_path: str | None = None, return_wedges: bool = False):
    """Mode A (C): L_s of the hypergraph given by its CSR, as int32 arrays
    (i, j, w) sorted by (i, j).  ``rows`` restricts the report to an
    ascending list of hyperedges (their full rows of L_s)."""
    lib = _load(lib_path)
    e_off = np.ascontiguousarray(e_off, dtype=np.int32)
    e_idx = np.ascontiguousarray(e_idx, dtype=np.int32)
    if e_idx.shape[0] == 0:
        e_idx = np.zeros(1, dtype=np.int32)
    rp = None
    nr = 0
    if rows is not None:
        rows = np.ascontiguousarray(rows, dtype=np.int32)
        if rows.shape[0] > 1 and np.any(np.diff(rows) <= 0):
            raise ValueError("rows must be strictly ascending")
        rp, nr = _ptr(rows) if rows.shape[0] else _ptr(np.zeros(1, np.int32)), rows.shape[0]
    oi, oj, ow = I32P(), I32P(), I32P()
    wd = ctypes.c_int64(0)
    cnt = lib.slg_oracle_line_graph(m, n, _ptr(e_off), _ptr(e_idx), int(s),
                                    rp, nr, int(threads), ctypes.byref(oi),
                                    ctypes.byref(oj), ctypes.byref(ow),
                                    ctypes.byref(wd))
    if cnt < 0:
        raise MemoryError("oracle failed (allocation or invalid arguments)")
    out = []
    for p in (oi, oj, ow):
        a = np.ctypeslib.as_array(p, shape=(max(cnt, 1),))[:cnt].copy()
        lib.slg_oracle_free(ctypes.cast(p, ctypes.c_void_p))
        out.append(a)
    if return_wedges:
        return out[0], out[1], out[2], int(wd.value)
    return out[0], out[1], out[2]


def transpose(m: int, n: int, e_off: np.ndarray, e_idx: np.ndarray):
    """CSR of the dual H*: row v lists the hyperedges containing v,
    ascending.  Written here (not taken from the input generator) so that
    the dual side of the oracle does not trust the caller's CSC."""
    e_off = np.asarray(e_off, dtype=np.int64)
    e_idx = np.asarray(e_idx, dtype=np.int64)
    owner = np.repeat(np.arange(m, dtype=np.int64), np.diff(e_off))
    order = np.lexsort((owner, e_idx))          # by vertex, then hyperedge
    d_idx = owner[order].astype(np.int32)
    deg = np.bincount(e_idx, minlength=n)
    d_off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=d_off[1:])
    return d_off.astype(np.int32), d_idx


def side(h, dual: bool):
    """(m, n, e_off, e_idx) of H or of H* (the latter by ``transpose``)."""
    if not dual:
        return h.m, h.n, h.e_off, h.e_idx
    d_off, d_idx = transpose(h.m, h.n, h.e_off, h.e_idx)
    return h.n, h.m, d_off, d_idx


def line_graph_of(h, s: int, dual: bool = False, **kw):
    """Mode A on H or on its dual."""
    m, n, off, idx = side(h, dual)
    return line_graph(m, n, off, idx, s, **kw)


def brute_force(rows, s: int):
    """Mode B: all pairs i < j, w = |e_i ∩ e_j| from Python sets, w >= s.
    Tiny inputs only (quadratic in the number of hyperedges)."""
    sets = [set(int(v) for v in r) for r in rows]
    out = []
    for i in range(len(sets)):
        for j in range(i + 1, len(sets)):
            w = len(sets[i] & sets[j])
            if w >= s:
                out.append((i, j, w))
    if not out:
        z = np.zeros(0, dtype=np.int32)
        return z, z.copy(), z.copy()
    a = np.asarray(out, dtype=np.int32)
    return a[:, 0].copy(), a[:, 1].copy(), a[:, 2].copy()


def spgemm_scipy(m: int, n: int, e_off: np.ndarray, e_idx: np.ndarray, s: int):
    """Mode C (Section IV-D read as: off-diagonal of B·Bᵀ with B the m x n
    hyperedge-by-vertex incidence; the diagonal is dropped explicitly)."""
    import scipy.sparse as sp
    e_off = np.asarray(e_off, dtype=np.int64)
    data = np.ones(int(e_off[-1]), dtype=np.int64)
    B = sp.csr_matrix((data, np.asarray(e_idx, dtype=np.int64), e_off),
                      shape=(m, n))
    C = sp.triu(B @ B.T, k=1).tocoo()
    keep = C.data >= s
    i, j, w = C.row[keep], C.col[keep], C.data[keep]
    order = np.lexsort((j, i))
    return (i[order].astype(np.int32), j[order].astype(np.int32),
            w[order].astype(np.int32))


def wedges(m: int, n: int, e_off: np.ndarray, e_idx: np.ndarray, s: int) -> int:
    """Closed form of the walk's work after the size filter:
    sum over v of C(d_s(v), 2), d_s(v) = #{e ∋ v : |e| >= s}."""
    sizes = np.diff(np.asarray(e_off, dtype=np.int64))
    keep_row = sizes >= s
    owner_keep = np.repeat(keep_row, sizes)
    d = np.bincount(np.asarray(e_idx)[owner_keep], minlength=n).astype(np.int64)
    return int((d * (d - 1) // 2).sum())


def canonical(i, j, w):
    """Stack triples into one int64 array of shape (P, 3) for comparisons."""
    return np.stack([np.asarray(i, np.int64), np.asarray(j, np.int64),
                     np.asarray(w, np.int64)], axis=1)


def squeeze(i, j, R: int):
    """(i', j', old_of_new): the ids of the list renumbered 0 .. k-1 in
    ascending order of their original id (Section IV-E)."""
    i = np.asarray(i, np.int64)
    j = np.asarray(j, np.int64)
    ids = np.unique(np.concatenate([i, j]))
    return (np.searchsorted(ids, i).astype(np.int32), np.searchsorted(ids, j).astype(np.int32),
            ids.astype(np.int32))


def adjacency(i, j, w, V: int):
    """Symmetric CSR of the line graph: (off [V+1] int64, adj, adj_w), every
    pair listed in the rows of both its ends, each row ascending."""
    i = np.asarray(i, np.int64)
    j = np.asarray(j, np.int64)
    w = np.asarray(w, np.int64)
    rows = np.concatenate([i, j])
    cols = np.concatenate([j, i])
    ws = np.concatenate([w, w])
    order = np.lexsort((cols, rows))
    off = np.zeros(V + 1, np.int64)
    off[1:] = np.cumsum(np.bincount(rows, minlength=V))
    return off, cols[order].astype(np.int32), ws[order].astype(np.int32)


def components(i, j, R: int):
    """(labels [R], count): for every id the smallest id of its connected
    component in the graph with edges (i, j) (its own id when isolated), and
    the number of components among the ids that occur in an edge."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    i = np.asarray(i, np.int64)
    j = np.asarray(j, np.int64)
    g = coo_matrix((np.ones(len(i), np.int8), (i, j)), shape=(R, R))
    _, lab = connected_components(g, directed=False)
    smallest = np.full(lab.max() + 1 if R else 0, R, np.int64)
    np.minimum.at(smallest, lab, np.arange(R))
    labels = smallest[lab].astype(np.int32)
    used = np.zeros(R, bool)
    used[i] = True
    used[j] = True
    return labels, int(np.unique(labels[used]).size)
