"""Pins for the CPU oracle: facts fixed by the paper and by mathematics.

Each ``pin_*`` function runs the oracle (optionally a specific build of it,
``lib_path``) and returns a list of failure messages (empty = pinned).  The
same suite checks the real oracle (test_oracle_pins.py) and deliberately
broken copies of it (test_oracle_mutants.py), which shows that a plausible
mistake anywhere in the oracle fails at least one pin.
"""
from __future__ import annotations

import os
from itertools import combinations

import numpy as np

import hypergen as hg
import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _lg(h, s, lib_path=None, dual=False, rows=None):
    m, n, off, idx = oracle.side(h, dual)
    return oracle.canonical(*oracle.line_graph(m, n, off, idx, s, rows=rows,
                                               lib_path=lib_path))


def _as_dict(t):
    return {(int(a), int(b)): int(c) for a, b, c in t}


def load_fig1():
    """Parse tests/golden/fig1.txt -> (names, rows, facts)."""
    names, rows, facts = [], [], []
    with open(os.path.join(GOLDEN, "fig1.txt")) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "edge":
                names.append(tok[1])
                rows.append([int(x) - 1 for x in tok[2:]])   # 1-based labels
            else:
                facts.append(tok)
    return names, rows, facts


def pin_fig1(lib_path=None):
    """Every number the paper prints about Fig. 1 (Section I)."""
    fails = []
    names, rows, facts = load_fig1()
    h = hg.from_rows(rows, 12)
    idx = {nm: k for k, nm in enumerate(names)}
    l1 = _as_dict(_lg(h, 1, lib_path))
    for f in facts:
        if f[0] == "size":
            if len(rows[idx[f[1]]]) != int(f[2]):
                fails.append(f"fig1 size {f}")
        elif f[0] == "overlap":
            a, b = sorted((idx[f[1]], idx[f[2]]))
            if l1.get((a, b), 0) != int(f[3]):
                fails.append(f"fig1 overlap {f}: got {l1.get((a, b), 0)}")
        elif f[0] in ("inline", "absent"):
            ls = _as_dict(_lg(h, int(f[1]), lib_path))
            a, b = sorted((idx[f[2]], idx[f[3]]))
            if ((a, b) in ls) != (f[0] == "inline"):
                fails.append(f"fig1 {f}")
    # In the dual H*, hyperedges 9 and 10 both contain B and C (they lie in
    # B ∩ C), neither contains A (A ∩ B = {3, 4}), and D holds at most one
    # of them (|B ∩ D| = 1), so w(9, 10) = 2 follows from the printed facts.
    d2 = _as_dict(_lg(h, 2, lib_path, dual=True))
    if d2.get((8, 9)) != 2:
        fails.append(f"fig1 dual w(9,10) != 2: {d2.get((8, 9))}")
    return fails


def _brute_side(h, dual):
    if not dual:
        return [list(r) for r in h.rows()]
    sets = [[] for _ in range(h.n)]
    for e, r in enumerate(h.rows()):
        for v in r:
            sets[int(v)].append(e)
    return sets


def pin_brute_force(lib_path=None, seeds=range(60)):
    """Mode A equals the naive all-pairs intersection (Section IV-A) on tiny
    random hypergraphs with empty rows, singletons and duplicated rows."""
    fails = []
    for seed in seeds:
        h = hg.random_small(seed)
        for dual in (False, True):
            for s in (1, 2, 3):
                a = _lg(h, s, lib_path, dual=dual)
                b = oracle.canonical(*oracle.brute_force(_brute_side(h, dual), s))
                if not np.array_equal(a, b):
                    fails.append(f"brute seed={seed} dual={dual} s={s}")
                    return fails
    return fails


def pin_closed_forms(lib_path=None):
    """Sum of L_1 weights = sum_v C(d(v), 2); with sizes >= s on both ends
    it equals sum_v C(d_s(v), 2); row sums of both triangles equal
    sum_{v in e} (d(v) - 1) (row sums of B·Bᵀ minus the diagonal |e|)."""
    fails = []
    for seed, (m, n) in enumerate([(300, 500), (200, 60), (50, 2000)]):
        h = hg.uniform(m, n, 0, 25, seed=100 + seed)
        for dual in (False, True):
            mm, nn, off, idx = oracle.side(h, dual)
            t = _lg(h, 1, lib_path, dual=dual)
            sizes = np.diff(off.astype(np.int64))
            deg = np.bincount(idx, minlength=nn).astype(np.int64)
            if int(t[:, 2].sum()) != int((deg * (deg - 1) // 2).sum()):
                fails.append(f"closed form L1 sum seed={seed} dual={dual}")
            for s in (2, 3, 5):
                both = (sizes[t[:, 0]] >= s) & (sizes[t[:, 1]] >= s)
                if int(t[both, 2].sum()) != oracle.wedges(mm, nn, off, idx, s):
                    fails.append(f"closed form W_s seed={seed} dual={dual} s={s}")
            rs = np.bincount(t[:, 0], weights=t[:, 2], minlength=mm) + \
                np.bincount(t[:, 1], weights=t[:, 2], minlength=mm)
            owner = np.repeat(np.arange(mm), sizes)
            want = np.bincount(owner, weights=deg[idx] - 1, minlength=mm)
            if not np.array_equal(rs.astype(np.int64), want.astype(np.int64)):
                fails.append(f"row sums seed={seed} dual={dual}")
    return fails


def pin_special_cases(lib_path=None):
    """Graphs (2-uniform hypergraphs, Section III), duplicates, complete
    k-uniform hypergraphs and sunflowers, whose line graphs are known."""
    fails = []
    rng = np.random.default_rng(7)
    nv = 40
    pairs = set()
    while len(pairs) < 120:
        a, b = sorted(rng.choice(nv, size=2, replace=False).tolist())
        pairs.add((a, b))
    edges = sorted(pairs)
    g = hg.graph(nv, edges)
    l1 = _lg(g, 1, lib_path)
    # classical line graph: edges sharing an endpoint, weight 1
    want = [(i, j, 1) for i, j in combinations(range(len(edges)), 2)
            if set(edges[i]) & set(edges[j])]
    if l1.tolist() != [list(x) for x in want]:
        fails.append("graph: L_1 is not the classical line graph")
    if _lg(g, 2, lib_path).shape[0] != 0:
        fails.append("graph: L_2 not empty")
    # the dual of a simple graph joins the two endpoints of each edge, w = 1
    d1 = _lg(g, 1, lib_path, dual=True)
    if d1.tolist() != [[a, b, 1] for a, b in edges]:
        fails.append("graph: L_1(H*) is not the graph's own edge list")
    # duplicated hyperedges (an indexed family allows copies): w = |e|
    r = [[1, 4, 6, 9], [0, 2], [1, 4, 6, 9], [3]]
    if _as_dict(_lg(hg.from_rows(r, 10), 4, lib_path)) != {(0, 2): 4}:
        fails.append("duplicates: w != |e|")
    # complete k-uniform hypergraph on k+1 vertices: all pairs share k-1
    for k in (2, 3, 5, 8):
        rows = [sorted(set(range(k + 1)) - {x}) for x in range(k + 1)]
        t = _lg(hg.from_rows(rows, k + 1), 1, lib_path)
        if t.shape[0] != (k + 1) * k // 2 or not np.all(t[:, 2] == k - 1):
            fails.append(f"complete {k}-uniform")
    # sunflower: a common core of c vertices plus disjoint petals
    c, petals = 3, 6
    rows = [list(range(c)) + list(range(c + 4 * p, c + 4 * p + 4))
            for p in range(petals)]
    t = _lg(hg.from_rows(rows, c + 4 * petals), 1, lib_path)
    if t.shape[0] != petals * (petals - 1) // 2 or not np.all(t[:, 2] == c):
        fails.append("sunflower")
    if _lg(hg.from_rows(rows, c + 4 * petals), c + 1, lib_path).shape[0]:
        fails.append("sunflower above core size")
    # empty hyperedges, isolated vertices: nothing
    if _lg(hg.from_rows([[], [], [3]], 8), 1, lib_path).shape[0]:
        fails.append("empty / singleton rows produced pairs")
    return fails


def pin_invariants(lib_path=None):
    """Structural invariants of L_s (Section III): canonical order, i < j,
    no endpoint with |e| < s, L_s ⊆ L_{s-1} with the same weights."""
    fails = []
    h = hg.uniform(400, 600, 1, 20, seed=3)
    for dual in (False, True):
        m, n, off, idx = oracle.side(h, dual)
        sizes = np.diff(off.astype(np.int64))
        prev = None
        for s in (1, 2, 3, 4):
            t = _lg(h, s, lib_path, dual=dual)
            if t.shape[0]:
                if not np.all(t[:, 0] < t[:, 1]):
                    fails.append(f"i<j dual={dual} s={s}")
                key = t[:, 0] * m + t[:, 1]
                if not np.all(np.diff(key) > 0):
                    fails.append(f"order dual={dual} s={s}")
                if not np.all(t[:, 2] >= s):
                    fails.append(f"w>=s dual={dual} s={s}")
                if np.any(sizes[t[:, 0]] < s) or np.any(sizes[t[:, 1]] < s):
                    fails.append(f"size filter dual={dual} s={s}")
            if prev is not None:
                pd = _as_dict(prev)
                for a, b, w in t:
                    if pd.get((int(a), int(b))) != int(w):
                        fails.append(f"nesting dual={dual} s={s}")
                        break
            prev = t
    return fails


def pin_scipy(lib_path=None):
    """Mode A equals the library product B·Bᵀ (Section IV-D) thresholded."""
    fails = []
    h = hg.config("uniform_2k")
    for dual in (False, True):
        m, n, off, idx = oracle.side(h, dual)
        for s in (1, 2, 3):
            a = _lg(h, s, lib_path, dual=dual)
            b = oracle.canonical(*oracle.spgemm_scipy(m, n, off, idx, s))
            if not np.array_equal(a, b):
                fails.append(f"scipy dual={dual} s={s}")
    return fails


def pin_rows_subset(lib_path=None):
    """Reporting a subset of rows gives exactly those rows of the full
    result (used for sampled checks at full size)."""
    fails = []
    h = hg.uniform(500, 300, 1, 15, seed=11)
    full = _lg(h, 2, lib_path)
    rows = np.arange(3, 500, 7, dtype=np.int32)
    sub = _lg(h, 2, lib_path, rows=rows)
    want = full[np.isin(full[:, 0], rows)]
    if not np.array_equal(sub, want):
        fails.append("row subset")
    return fails


def _bfs_labels(R, pairs):
    """Smallest id of each id's component by breadth-first search."""
    nb = {v: [] for v in range(R)}
    for a, b in pairs:
        nb[a].append(b)
        nb[b].append(a)
    lab = [-1] * R
    for v in range(R):
        if lab[v] < 0:
            comp, todo = [v], [v]
            lab[v] = v
            while todo:
                x = todo.pop()
                for y in nb[x]:
                    if lab[y] < 0:
                        lab[y] = v
                        comp.append(y)
                        todo.append(y)
    return lab  # v is the smallest id of its component when first reached


def pin_post(lib_path=None):
    """Squeezing, adjacency and components of L_s against their definitions:
    Fig. 1 (L_1(H) = {AB, BC, BD, CD} is one component; L_2(H) = {AB, BC}
    leaves D out; L_3(H) = {BC}), a path, and breadth-first search / dict
    construction on random small lists."""
    fails = []
    names, rows, _ = load_fig1()
    h = hg.from_rows(rows, n=max(max(r) for r in rows) + 1)
    want = {1: ([0] * 4, 1), 2: ([0, 0, 0, 3], 1), 3: ([0, 1, 1, 3], 1)}
    for s, (lab, k) in want.items():
        t = _lg(h, s, lib_path)
        got, cnt = oracle.components(t[:, 0], t[:, 1], 4)
        if list(got) != lab or cnt != k:
            fails.append(f"Fig. 1 components at s={s}: {list(got)} / {cnt}")
    # a path 0-1-...-9 plus an isolated id 10 and an edge 11-12
    i = np.array(list(range(9)) + [11])
    j = np.array(list(range(1, 10)) + [12])
    got, cnt = oracle.components(i, j, 13)
    if list(got) != [0] * 10 + [10, 11, 11] or cnt != 2:
        fails.append(f"path components {list(got)} / {cnt}")
    rng = np.random.default_rng(5)
    for trial in range(40):
        R = int(rng.integers(1, 40))
        k = int(rng.integers(0, 60))
        pairs = sorted({tuple(sorted(rng.choice(R, 2, replace=False))) for _ in range(k)}
                       if R > 1 else set())
        i = np.array([p[0] for p in pairs], np.int64)
        j = np.array([p[1] for p in pairs], np.int64)
        w = rng.integers(1, 9, len(pairs))
        lab, cnt = oracle.components(i, j, R)
        ref = _bfs_labels(R, pairs)
        used = sorted({x for p in pairs for x in p})
        if list(lab) != ref or cnt != len({ref[v] for v in used}):
            fails.append(f"components trial {trial}")
        si, sj, old = oracle.squeeze(i, j, R)
        if list(old) != used or any(old[si[q]] != i[q] or old[sj[q]] != j[q]
                                    for q in range(len(pairs))):
            fails.append(f"squeeze trial {trial}")
        off, adj, aw = oracle.adjacency(i, j, w, R)
        for v in range(R):
            want_row = sorted([(b, int(c)) for (a, b), c in zip(pairs, w) if a == v] +
                              [(a, int(c)) for (a, b), c in zip(pairs, w) if b == v])
            row = list(zip(adj[off[v]:off[v + 1]].tolist(), aw[off[v]:off[v + 1]].tolist()))
            if row != want_row:
                fails.append(f"adjacency trial {trial} row {v}")
                break
    return fails


ALL_PINS = [pin_fig1, pin_brute_force, pin_closed_forms, pin_special_cases,
            pin_invariants, pin_scipy, pin_rows_subset, pin_post]


def run_all(lib_path=None):
    fails = []
    for p in ALL_PINS:
        try:
            fails += p(lib_path)
        except Exception as exc:  # a crashing oracle fails the pin too
            fails.append(f"{p.__name__} raised {type(exc).__name__}: {exc}")
    return fails
