"""Serving form: s-line-graph queries against device-resident hypergraphs,
with continuous batching.

A query is (hypergraph id, s, side).  The hypergraphs stay in device memory.
Each of ``slots`` worker threads owns a CUDA stream.  A free worker takes the
oldest waiting query whose memory estimate fits the budget that the queries
in flight leave.  That query then runs on the worker's stream while the
others run on theirs, so their kernels overlap on the GPU.  A query that
arrives while others are on the GPU is admitted as soon as a slot and the
memory are free.  Latency is measured from submission to completion.

One walk per query: the output is sized from what the server already knows
(the query's own pair count from an earlier identical query, else the count
of the same graph and side at the nearest smaller threshold -- L_s is the
part of L_s' with w >= s for s' <= s (Section III), so that count bounds it
-- else a first guess), and a build whose list does not fit returns its
exact size and is run once more at that size.

Reuse across thresholds (``reuse=True``): per hypergraph and side the server
keeps one base list L_{base_s} (within ``cache_bytes``), built by the first
query with s >= base_s on that graph and side, and answers every query with
s >= base_s by filtering it (slg_filter) instead of walking again.
``base_s=None`` keeps instead the list of the smallest threshold queried so
far.

All computation runs in the library's CUDA kernels (slg_build / slg_filter
through the binding); this module only schedules.
"""
from __future__ import annotations

import bisect
import collections
import threading
import time

import numpy as np

from . import (DeviceHypergraph, SlgError, alloc_outputs, build, count, filter_pairs,
               last_stats, release_memory, wedges)

_FIRST_GUESS = 1 << 24  # pairs, when nothing bounds a query's list yet
_GUESS_DIV = 16         # ... or W_s / 16: a pair of L_s takes >= s >= 2 of its wedges,
                        # and on these workloads about 1 wedge in 20 ends in a pair


class Query:
    """One request and its outcome."""

    __slots__ = ("gid", "s", "dual", "t_submit", "t_start", "t_done", "pairs", "result",
                 "error", "est_bytes", "admitted", "reused", "walks", "_done")

    def __init__(self, gid: int, s: int, dual: bool):
        self.gid, self.s, self.dual = gid, s, dual
        self.t_submit = self.t_start = self.t_done = 0.0
        self.pairs = -1
        self.result = None
        self.error = None
        self.est_bytes = 0
        self.admitted = False   # counted in the server's memory in flight
        self.reused = False
        self.walks = 0
        self._done = threading.Event()

    def wait(self, timeout=None) -> bool:
        return self._done.wait(timeout)

    @property
    def latency_ms(self) -> float:
        return (self.t_done - self.t_submit) * 1e3


class ResultTooLarge(RuntimeError):
    """The query's list is larger than the server's per-query limit."""


class Server:
    """Continuous-batching scheduler over a resident pool of hypergraphs.

    With ``max_result_bytes`` set, a query whose list would take more than
    that (20 bytes a pair: the (i, j, w) output and the build's staging) is
    refused with ResultTooLarge; for s = 1, whose lists can be far larger
    than any other threshold's, the size is counted (one walk, no output)
    before the build.
    """

    def __init__(self, graphs: list[DeviceHypergraph], slots: int = 4,
                 memory_budget: int = 64 << 30, keep_results: bool = False,
                 reuse: bool = False, cache_bytes: int = 32 << 30, base_s: int | None = 2,
                 max_result_bytes: int | None = None):
        import torch
        self.graphs = graphs
        self.keep = keep_results
        self.reuse = reuse
        self.base_s = base_s
        self.cache_bytes = int(cache_bytes)
        self.cached = {}     # (gid, dual) -> (s, (i, j, w), bytes)
        self.building = {}   # (gid, dual) -> threading.Event while its base list is built
        self.cache_used = 0
        self.budget = int(memory_budget)
        self.max_result = int(max_result_bytes) if max_result_bytes is not None else 1 << 62
        self.in_flight = 0     # estimated bytes of the admitted queries
        self.n_in_flight = 0   # admitted queries not yet done
        self.pending = collections.deque()
        self.cv = threading.Condition()
        self.closed = False
        self.counts: dict = {}  # (gid, dual) -> sorted [(s, |L_s|)]
        self.done: list[Query] = []
        # per graph and side: incidences, rows, columns, largest row work at
        # s = 1 (an upper bound for every s), for the memory estimate
        self.shape = {}
        for gid, g in enumerate(graphs):
            for dual in (False, True):
                wedges(g, 1, dual)
                self.shape[(gid, dual)] = (g.nnz, g.rows(dual), g.rows(not dual),
                                           last_stats()["max_row_work"])
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self.workers = [threading.Thread(target=self._worker, args=(k,), daemon=True)
                        for k in range(slots)]
        for t in self.workers:
            t.start()

    # ------------------------------------------------------ counts, bounds --
    def _known(self, gid: int, dual: bool, s: int, n: int):
        with self.cv:
            lst = self.counts.setdefault((gid, dual), [])
            k = bisect.bisect_left(lst, (s, -1))
            if k < len(lst) and lst[k][0] == s:
                return
            lst.insert(k, (s, n))

    def _bound(self, gid: int, dual: bool, s: int):
        """|L_s| if known, else |L_s'| for the largest known s' < s (an upper
        bound), else None."""
        with self.cv:
            lst = self.counts.get((gid, dual), [])
            k = bisect.bisect_right(lst, (s, 1 << 62))
            return lst[k - 1][1] if k else None

    # ----------------------------------------------------------- estimates --
    def _estimate(self, q: Query) -> int:
        base = self._cached_for(q)
        if base is not None:                                # a filter of a kept list
            return 2 * base[2] + 8 * (base[1][0].shape[0] // 8192 + 2)
        nnz, rows, cols, maxw = self.shape[(q.gid, q.dual)]
        work = 4 * (7 * nnz + 12 * rows + cols)            # planning arrays
        giant = 304 * 16 * maxw                             # giant-bin scratch bound
        s = self._base_for(q) or q.s
        pairs = self._bound(q.gid, q.dual, s)
        out = 20 * (pairs if pairs is not None else _FIRST_GUESS)
        return work + giant + out

    def _base_for(self, q: Query):
        """The base threshold this query's answer comes from, or None."""
        if self.reuse and self.base_s is not None and q.s >= self.base_s:
            return self.base_s
        return None

    def _cached_for(self, q: Query):
        if not self.reuse:
            return None
        e = self.cached.get((q.gid, q.dual))
        return e if e is not None and e[0] <= q.s else None

    def _keep_list(self, gid: int, dual: bool, s: int, res) -> bool:
        """Keep `res` = L_s as the list of its graph and side if it has the
        smallest threshold so far and fits the cache."""
        nbytes = 12 * int(res[0].shape[0])
        with self.cv:
            key = (gid, dual)
            old = self.cached.get(key)
            if old is not None and old[0] <= s:
                return False
            free = self.cache_bytes - self.cache_used + (old[2] if old else 0)
            if nbytes > free:
                return False
            self.cached[key] = (s, res, nbytes)
            self.cache_used += nbytes - (old[2] if old else 0)
            return True

    # ----------------------------------------------------------------- API --
    def warm(self) -> float:
        """Builds and keeps the base list of every graph and side now (reuse
        with base_s set), so that queries with s >= base_s are answered by
        filters from their first arrival.  Returns the seconds it took."""
        import torch
        if not self.reuse or self.base_s is None:
            return 0.0
        t0 = time.perf_counter()
        st = self.streams[0]
        for gid in range(len(self.graphs)):
            for dual in (False, True):
                q = Query(gid, self.base_s, dual)
                try:
                    with torch.cuda.stream(st):
                        self._base_list(q, st)
                except (SlgError, ResultTooLarge, torch.cuda.OutOfMemoryError):
                    pass  # not kept: such queries walk
        st.synchronize()
        return time.perf_counter() - t0

    def submit(self, gid: int, s: int, dual: bool = False) -> Query:
        q = Query(gid, s, dual)
        q.t_submit = time.perf_counter()
        with self.cv:
            self.pending.append(q)
            self.cv.notify()
        return q

    def close(self):
        with self.cv:
            self.closed = True
            self.cv.notify_all()
        for t in self.workers:
            t.join()

    # -------------------------------------------------------------- worker --
    def _take(self) -> Query | None:
        with self.cv:
            while True:
                for k, q in enumerate(self.pending):
                    est = self._estimate(q)
                    # the oldest query that fits; a lone query is always admitted
                    if self.n_in_flight == 0 or self.in_flight + est <= self.budget:
                        del self.pending[k]
                        q.est_bytes = est
                        q.admitted = True
                        self.in_flight += est
                        self.n_in_flight += 1
                        return q
                if self.closed and not self.pending:
                    return None
                self.cv.wait(0.05)

    def _walk(self, q: Query, s: int, st):
        """L_s of the query's graph and side in one walk (two when the first
        guess of its size was too small)."""
        g = self.graphs[q.gid]
        n = self._bound(q.gid, q.dual, s)
        if n is None and s == 1:
            q.walks += 1
            n = count(g, s, q.dual, stream=st)
            self._known(q.gid, q.dual, s, n)
            self._resize(q, n)
        if n is not None and s == 1 and 20 * n > self.max_result:
            raise ResultTooLarge(f"L_1 of graph {q.gid}{'*' if q.dual else ''} has {n} pairs")
        if n is None:  # first guess: from W_s (slg_wedges: planning only, no walk)
            guess = wedges(g, s, q.dual, stream=st) // _GUESS_DIV
            n = min(max(guess, 1 << 16), self.max_result // 20)
        cap = n
        for attempt in (0, 1):
            out = alloc_outputs(max(cap, 1), False, g.e_off.device)
            q.walks += 1
            try:
                res = build(g, s, dual=q.dual, out=out, stream=st)
                self._known(q.gid, q.dual, s, int(res[0].shape[0]))
                return res
            except SlgError as exc:
                if exc.status != 2 or attempt:
                    raise
                cap = exc.needed            # the exact size, counted by the walk
                self._known(q.gid, q.dual, s, cap)
                del out
                self._resize(q, cap)
                if 20 * cap > self.max_result:
                    raise ResultTooLarge(f"L_{s} of graph {q.gid}{'*' if q.dual else ''} has "
                                         f"{cap} pairs") from None

    def _resize(self, q: Query, pairs: int):
        """The query's list turned out to have `pairs` pairs: its share of
        the memory budget follows (new queries see it at admission)."""
        if not q.admitted:  # a warm-up build outside the admission count
            return
        nnz, rows, cols, maxw = self.shape[(q.gid, q.dual)]
        est = 4 * (7 * nnz + 12 * rows + cols) + 304 * 16 * maxw + 20 * pairs
        with self.cv:
            self.in_flight += est - q.est_bytes
            q.est_bytes = est

    def _base_list(self, q: Query, st):
        """The kept base list of the query's graph and side, built now if it
        is missing (other queries on the same graph and side wait for it)."""
        key = (q.gid, q.dual)
        while True:
            with self.cv:
                e = self.cached.get(key)
                if e is not None and e[0] <= q.s:
                    return e[1]
                ev = self.building.get(key)
                if ev is None:
                    ev = threading.Event()
                    self.building[key] = ev
                    mine = True
                else:
                    mine = False
            if not mine:
                ev.wait()
                with self.cv:
                    e = self.cached.get(key)
                if e is None or e[0] > q.s:
                    return None          # not kept (cache full): walk instead
                return e[1]
            try:
                res = self._walk(q, self.base_s, st)
                st.synchronize()
                kept = self._keep_list(q.gid, q.dual, self.base_s, res)
                return res
            finally:
                with self.cv:
                    del self.building[key]
                ev.set()

    def _answer(self, q: Query, st):
        import torch
        with torch.cuda.stream(st):
            if self.reuse:
                base = None
                if self._base_for(q) is not None:
                    base = self._base_list(q, st)
                else:
                    e = self._cached_for(q)
                    base = e[1] if e is not None else None
                if base is not None:
                    q.reused = True
                    return filter_pairs(*base, q.s, stream=st)
            res = self._walk(q, q.s, st)
            if self.reuse and self.base_s is None:
                st.synchronize()
                self._keep_list(q.gid, q.dual, q.s, res)
            return res

    def _worker(self, k: int):
        import torch
        st = self.streams[k]
        while True:
            q = self._take()
            if q is None:
                return
            q.t_start = time.perf_counter()
            try:
                for attempt in (0, 1):
                    try:
                        i, j, w = self._answer(q, st)
                        st.synchronize()
                        break
                    except (SlgError, torch.cuda.OutOfMemoryError) as exc:
                        # out of device memory: give the kept lists and both
                        # allocators' cached memory back, retry once
                        if attempt or getattr(exc, "status", 3) != 3:
                            raise
                        if self.reuse:
                            with self.cv:
                                self.cached.clear()
                                self.cache_used = 0
                        torch.cuda.empty_cache()
                        release_memory()
                q.pairs = int(i.shape[0])
                if self.keep:
                    q.result = (i, j, w)
            except Exception as exc:  # reported on the query
                q.error = exc
            q.t_done = time.perf_counter()
            with self.cv:
                self.in_flight -= q.est_bytes
                self.n_in_flight -= 1
                q.admitted = False
                self.done.append(q)
                self.cv.notify_all()
            q._done.set()

    # --------------------------------------------------------------- stats --
    @staticmethod
    def summary(queries: list[Query], wall_s: float) -> dict:
        lat = np.array([q.latency_ms for q in queries if q.error is None])
        errs = [q for q in queries if q.error is not None]
        return {"queries": len(queries), "errors": len(errs),
                "first_error": (f"{errs[0].gid}/{errs[0].s}/{errs[0].dual}: {errs[0].error!r}"
                                if errs else None),
                "too_large": sum(isinstance(q.error, ResultTooLarge) for q in queries),
                "answered_by_filter": sum(q.reused for q in queries),
                "walks": sum(q.walks for q in queries),
                "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
                "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
                "mean_ms": float(lat.mean()) if lat.size else None,
                "queries_per_s": len(queries) / wall_s if wall_s > 0 else None}
