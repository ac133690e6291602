"""Seeded synthetic hypergraphs: input data only.

This module is shared by the CPU oracle tests and by the CUDA path (tests and
benchmark).  It draws incidence structures and stores them as CSR + CSC int32
arrays; it contains none of the s-overlap arithmetic (no intersections, no
wedge counting, no thresholds).

A hypergraph H = (V, E) is an indexed family of vertex sets (Section III).
Rows are hyperedges, columns are vertices; every CSR row is sorted ascending
and holds distinct vertex ids, every CSC row (a vertex's hyperedge list) is
sorted ascending.  Swapping the two arrays gives the dual H* (Section III).

Workload recipes (the paper's datasets are not available; these stand in for
their shapes, Table 2: power-law / heavy-tailed hyperedge sizes with a maximum
size far above the mean):

* ``uniform``      -- |e| ~ U{kmin..kmax}, vertices uniform without replacement.
* ``chung_lu``     -- |e| discrete power law (exponent 2.1, capped), vertex
                      weights power law (exponent 2.3); each hyperedge draws
                      |e| distinct vertices with probability proportional to
                      the vertex weight.
* ``lognormal_web``-- |e| = round(lognormal(mu, sigma)) clipped, uniform
                      vertices, plus a planted dense core (a random set of
                      hyperedges x a random set of vertices, Bernoulli(p)).
* ``batch``        -- many ``chung_lu`` hypergraphs of log-uniform size.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

__all__ = [
    "Hypergraph", "from_rows", "from_pairs", "csr_to_csc", "uniform",
    "chung_lu", "lognormal_web", "batch", "random_small", "graph",
    "config", "CONFIGS",
]


@dataclass
class Hypergraph:
    """CSR (hyperedge -> vertices) and CSC (vertex -> hyperedges) of H."""

    m: int                 # number of hyperedges |E|
    n: int                 # number of vertices |V|
    e_off: np.ndarray      # int32[m+1]
    e_idx: np.ndarray      # int32[nnz], rows ascending, unique
    v_off: np.ndarray      # int32[n+1]
    v_idx: np.ndarray      # int32[nnz], rows ascending
    name: str = ""
    # planted dense core (lognormal_web): its hyperedge and vertex ids, else None
    core_edges: np.ndarray | None = None
    core_vertices: np.ndarray | None = None

    @property
    def nnz(self) -> int:
        return int(self.e_idx.shape[0])

    def dual(self) -> "Hypergraph":
        """H*: vertices become hyperedges and vice versa (arrays swapped)."""
        return Hypergraph(self.n, self.m, self.v_off, self.v_idx,
                          self.e_off, self.e_idx, self.name + "*",
                          self.core_vertices, self.core_edges)

    def side(self, dual: bool) -> "Hypergraph":
        return self.dual() if dual else self

    def rows(self):
        """List of per-hyperedge vertex arrays (small inputs only)."""
        return [self.e_idx[self.e_off[i]:self.e_off[i + 1]]
                for i in range(self.m)]


def _unique_sorted(x: np.ndarray) -> np.ndarray:
    """Sorted distinct values (sort-based; numpy's hash-based unique is slow
    on tens of millions of int64 keys)."""
    x = np.sort(x)
    if x.shape[0] == 0:
        return x
    keep = np.empty(x.shape[0], dtype=bool)
    keep[0] = True
    np.not_equal(x[1:], x[:-1], out=keep[1:])
    return x[keep]


def csr_to_csc(e_off: np.ndarray, e_idx: np.ndarray, n: int):
    """Stable counting transpose: vertex -> ascending hyperedge ids."""
    m = e_off.shape[0] - 1
    rows = np.repeat(np.arange(m, dtype=np.int64),
                     np.diff(e_off.astype(np.int64)))
    order = np.argsort(e_idx, kind="stable")
    v_idx = rows[order].astype(np.int32)
    deg = np.bincount(e_idx, minlength=n).astype(np.int64)
    v_off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=v_off[1:])
    return v_off.astype(np.int32), v_idx


def from_pairs(row: np.ndarray, col: np.ndarray, m: int, n: int,
               name: str = "") -> Hypergraph:
    """Build H from incidence pairs; duplicates are merged."""
    key = _unique_sorted(row.astype(np.int64) * n + col.astype(np.int64))
    r = (key // n).astype(np.int64)
    c = (key % n).astype(np.int32)
    sizes = np.bincount(r, minlength=m).astype(np.int64)
    if int(sizes.sum()) >= 2**31:
        raise ValueError("nnz must stay below 2^31 for int32 offsets")
    e_off = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(sizes, out=e_off[1:])
    e_off = e_off.astype(np.int32)
    v_off, v_idx = csr_to_csc(e_off, c, n)
    return Hypergraph(m, n, e_off, c, v_off, v_idx, name)


def from_rows(rows, n: int, name: str = "") -> Hypergraph:
    """Build H from a list of vertex collections (duplicates within a row are
    merged; empty rows allowed)."""
    m = len(rows)
    r = np.concatenate([np.full(len(x), i, dtype=np.int64)
                        for i, x in enumerate(rows)] or [np.zeros(0, np.int64)])
    c = np.concatenate([np.asarray(x, dtype=np.int64)
                        for x in rows] or [np.zeros(0, np.int64)])
    return from_pairs(r, c, m, n, name)


def _draw_distinct(sizes: np.ndarray, n: int, rng: np.random.Generator,
                   cdf: np.ndarray | None) -> tuple[np.ndarray, np.ndarray]:
    """For each row i draw sizes[i] distinct columns in [0, n).

    Uniform columns when ``cdf`` is None, else columns with probability given
    by the cumulative weights ``cdf`` (inverse-CDF draws).  Rows are filled by
    drawing with replacement, merging duplicates and topping up the rows that
    came out short until every row has its target size.
    """
    sizes = np.minimum(sizes.astype(np.int64), n)
    m = sizes.shape[0]

    def draw(k: int) -> np.ndarray:
        if cdf is None:
            return rng.integers(0, n, size=k, dtype=np.int64)
        u = rng.random(k) * cdf[-1]
        return np.minimum(np.searchsorted(cdf, u, side="right"), n - 1)

    rows = np.repeat(np.arange(m, dtype=np.int64), sizes)
    key = _unique_sorted(rows * n + draw(rows.shape[0]))
    short = sizes - np.bincount(key // n, minlength=m)
    # Rows that came out short (duplicates merged) are topped up on their own,
    # so each round only re-sorts the keys of those rows.
    pending = short > 0
    sel = pending[key // n]
    done, work = key[~sel], key[sel]
    for _ in range(50):
        need = np.nonzero(short > 0)[0]
        if need.shape[0] == 0:
            break
        add_rows = np.repeat(need, short[need])
        work = _unique_sorted(np.concatenate(
            [work, add_rows * n + draw(add_rows.shape[0])]))
        have = np.bincount(work // n, minlength=m)
        short = np.where(pending, sizes - have, 0)
    # Rows still short (targets close to n under skewed weights: rare, tiny
    # graphs) take their missing vertices from their complement, uniformly
    # without replacement.
    need = np.nonzero(short > 0)[0]
    if need.shape[0]:
        extra = []
        r_all = work // n
        for row in need:
            present = work[r_all == row] % n
            comp = np.setdiff1d(np.arange(n, dtype=np.int64), present)
            pick = rng.choice(comp, size=int(short[row]), replace=False)
            extra.append(row * n + pick)
        work = _unique_sorted(np.concatenate([work] + extra))
    key = np.sort(np.concatenate([done, work]))
    return key // n, key % n


def uniform(m: int, n: int, kmin: int, kmax: int, seed: int,
            name: str = "uniform") -> Hypergraph:
    """|e| ~ U{kmin..kmax}; vertices uniform without replacement."""
    rng = np.random.default_rng(seed)
    sizes = rng.integers(kmin, kmax + 1, size=m)
    r, c = _draw_distinct(sizes, n, rng, None)
    return from_pairs(r, c, m, n, name)


def _power_law_sizes(m: int, exponent: float, cap: int, mean: float,
                     rng: np.random.Generator) -> np.ndarray:
    """Discrete power law P(k) ~ k^-exponent on [kmin, cap], with kmin the
    integer whose distribution mean is closest to ``mean``."""
    ks = np.arange(1, cap + 1, dtype=np.float64)
    best = None
    for kmin in range(1, min(cap, 200) + 1):
        p = ks[kmin - 1:] ** (-exponent)
        mu = float((ks[kmin - 1:] * p).sum() / p.sum())
        if best is None or abs(mu - mean) < best[0]:
            best = (abs(mu - mean), kmin)
    kmin = best[1]
    p = ks[kmin - 1:] ** (-exponent)
    cdf = np.cumsum(p)
    u = rng.random(m) * cdf[-1]
    return (np.searchsorted(cdf, u, side="right") + kmin).astype(np.int64)


def chung_lu(m: int, n: int, seed: int, size_exp: float = 2.1,
             size_cap: int = 10_000, mean_size: float = 20.0,
             deg_exp: float = 2.3, name: str = "chung_lu") -> Hypergraph:
    """Power-law Chung-Lu bipartite hypergraph.

    Hyperedge sizes follow a discrete power law with exponent ``size_exp``
    capped at ``size_cap`` and lower cut-off chosen so the mean is about
    ``mean_size``.  Vertex weights follow a continuous power law with exponent
    ``deg_exp`` (Pareto), scaled to mean nnz/n and capped at nnz/size_cap so
    that the Chung-Lu inclusion probabilities stay at most one.
    """
    rng = np.random.default_rng(seed)
    sizes = np.minimum(_power_law_sizes(m, size_exp, size_cap, mean_size, rng), n)
    nnz = int(sizes.sum())
    w = rng.pareto(deg_exp - 1.0, size=n) + 1.0
    w *= (nnz / n) / w.mean()
    cap = max(nnz / max(int(sizes.max()), 1), 1.0)
    w = np.minimum(w, cap)
    cdf = np.cumsum(w)
    r, c = _draw_distinct(sizes, n, rng, cdf)
    return from_pairs(r, c, m, n, name)


def lognormal_web(m: int, n: int, seed: int, mu: float = 2.0,
                  sigma: float = 1.5, cap: int = 100_000,
                  core_edges: int = 4096, core_vertices: int = 8192,
                  core_density: float = 0.3,
                  name: str = "lognormal_web") -> Hypergraph:
    """Heavy-tailed web-shaped hypergraph with a planted dense core.

    Sizes round(lognormal(mu, sigma)) clipped to [1, cap]; vertices uniform.
    The core is a seeded random set of ``core_edges`` hyperedges times a
    random set of ``core_vertices`` vertices, each incidence present with
    probability ``core_density``; it is merged with the sparse part.
    """
    rng = np.random.default_rng(seed)
    sizes = np.clip(np.rint(rng.lognormal(mu, sigma, size=m)), 1, cap)
    sizes = np.minimum(sizes.astype(np.int64), n)
    r, c = _draw_distinct(sizes, n, rng, None)
    ce = cv = None
    if core_edges > 0 and core_vertices > 0 and core_density > 0:
        ce = rng.choice(m, size=min(core_edges, m), replace=False)
        cv = rng.choice(n, size=min(core_vertices, n), replace=False)
        hit = rng.random((ce.shape[0], cv.shape[0])) < core_density
        ri, ci = np.nonzero(hit)
        r = np.concatenate([r, ce[ri].astype(np.int64)])
        c = np.concatenate([c, cv[ci].astype(np.int64)])
    h = from_pairs(r, c, m, n, name)
    if ce is not None:
        h.core_edges = np.sort(ce).astype(np.int32)
        h.core_vertices = np.sort(cv).astype(np.int32)
    return h


def _batch_member(args):
    mk, seed, k = args
    return chung_lu(mk, 2 * mk, seed, name=f"batch{k}")


def batch(count: int, seed: int, m_lo: int = 1_000, m_hi: int = 200_000,
          s_lo: int = 2, s_hi: int = 32, workers: int = 1):
    """``count`` Chung-Lu hypergraphs with m log-uniform in [m_lo, m_hi],
    n = 2m, mean size 20, each with its own s ~ U{s_lo..s_hi}.  Graph k uses
    seed ``seed + k``, so the result does not depend on ``workers`` (spawned
    processes generating members in parallel).  Returns a list of
    (Hypergraph, s)."""
    rng = np.random.default_rng(seed)
    ms = np.exp(rng.uniform(np.log(m_lo), np.log(m_hi), size=count))
    ss = rng.integers(s_lo, s_hi + 1, size=count)
    jobs = [(int(ms[k]), seed + k, k) for k in range(count)]
    if workers > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as pool:
            hs = pool.map(_batch_member, jobs, chunksize=1)
    else:
        hs = [_batch_member(j) for j in jobs]
    return [(h, int(ss[k])) for k, h in enumerate(hs)]


def random_small(seed: int, m_max: int = 24, n_max: int = 24,
                 k_max: int = 10) -> Hypergraph:
    """Tiny random hypergraph with empty rows, singletons, duplicated rows
    and isolated vertices mixed in (the cases an indexed family allows)."""
    rng = np.random.default_rng(seed)
    m = int(rng.integers(1, m_max + 1))
    n = int(rng.integers(1, n_max + 1))
    rows = []
    for i in range(m):
        if rows and rng.random() < 0.15:           # a duplicated hyperedge
            rows.append(rows[int(rng.integers(0, len(rows)))].copy())
            continue
        k = int(rng.integers(0, min(k_max, n) + 1))
        rows.append(rng.choice(n, size=k, replace=False))
    return from_rows(rows, n, f"small{seed}")


def graph(n: int, edges, name: str = "graph") -> Hypergraph:
    """A simple graph as a 2-uniform hypergraph (one hyperedge per edge)."""
    return from_rows([list(e) for e in edges], n, name)


# Named workloads: sizes as stated in each recipe.
CONFIGS = {
    "uniform_2k": dict(kind="uniform", m=2_000, n=4_000, kmin=1, kmax=20, seed=0),
    "chung_lu_1m": dict(kind="chung_lu", m=1_000_000, n=2_000_000, seed=1),
    "web_4m": dict(kind="lognormal_web", m=4_000_000, n=10_000_000, seed=2),
}


def config(name: str, scale: float = 1.0) -> Hypergraph:
    """Generate a named workload, optionally scaled down in m and n."""
    c = dict(CONFIGS[name])
    kind = c.pop("kind")
    if scale != 1.0:
        c["m"] = max(1, int(c["m"] * scale))
        c["n"] = max(1, int(c["n"] * scale))
    fn = {"uniform": uniform, "chung_lu": chung_lu,
          "lognormal_web": lognormal_web}[kind]
    return fn(name=name, **c)
