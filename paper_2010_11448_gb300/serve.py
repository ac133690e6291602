"""Serving form: s-line-graph queries against device-resident hypergraphs,
with continuous batching.

A query is (hypergraph id, s, side).  The hypergraphs stay in device memory.
Each of ``slots`` worker threads owns a CUDA stream.  A free worker takes the
oldest waiting query whose memory estimate fits the budget that the queries
in flight leave.  That query then runs on the worker's stream while the
others run on theirs, so their kernels overlap on the GPU.  A query that
arrives while others are on the GPU is admitted as soon as a slot and the
memory are free.  Latency is measured from submission to completion.

Reuse across thresholds (``reuse=True``): L_s is the sub-list of any L_s'
with s' <= s and w >= s (Section III), so per hypergraph and side the
server keeps the list of the smallest threshold built so far (within
``cache_bytes``) and answers any larger threshold by filtering it
(slg_filter) instead of walking again.

All computation runs in the library's CUDA kernels (slg_count / slg_build
through the binding); this module only schedules.
"""
from __future__ import annotations

import collections
import threading
import time

import numpy as np

from . import (DeviceHypergraph, SlgError, alloc_outputs, build, count, filter_pairs,
               last_stats, wedges)


class Query:
    """One request and its outcome."""

    __slots__ = ("gid", "s", "dual", "t_submit", "t_start", "t_done", "pairs", "result",
                 "error", "est_bytes", "reused", "_done")

    def __init__(self, gid: int, s: int, dual: bool):
        self.gid, self.s, self.dual = gid, s, dual
        self.t_submit = self.t_start = self.t_done = 0.0
        self.pairs = -1
        self.result = None
        self.error = None
        self.est_bytes = 0
        self.reused = False
        self._done = threading.Event()

    def wait(self, timeout=None) -> bool:
        return self._done.wait(timeout)

    @property
    def latency_ms(self) -> float:
        return (self.t_done - self.t_submit) * 1e3


class Server:
    """Continuous-batching scheduler over a resident pool of hypergraphs."""

    def __init__(self, graphs: list[DeviceHypergraph], slots: int = 4,
                 memory_budget: int = 64 << 30, keep_results: bool = False,
                 reuse: bool = False, cache_bytes: int = 32 << 30):
        import torch
        self.graphs = graphs
        self.keep = keep_results
        self.reuse = reuse
        self.cache_bytes = int(cache_bytes)
        self.cached = {}     # (gid, dual) -> (s, (i, j, w), bytes)
        self.cache_used = 0
        self.budget = int(memory_budget)
        self.in_flight = 0
        self.pending = collections.deque()
        self.cv = threading.Condition()
        self.closed = False
        self.pair_cache: dict = {}
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

    # ----------------------------------------------------------- estimates --
    def _estimate(self, q: Query) -> int:
        base = self._cached_for(q)
        if base is not None:                                # a filter of a kept list
            return 2 * base[2] + 8 * (base[1][0].shape[0] // 8192 + 2)
        nnz, rows, cols, maxw = self.shape[(q.gid, q.dual)]
        work = 4 * (7 * nnz + 12 * rows + cols)            # planning arrays
        giant = 152 * 16 * maxw                             # giant-bin scratch bound
        pairs = self.pair_cache.get((q.gid, q.s, q.dual))
        out = 20 * (pairs if pairs is not None else 2 * nnz)
        return work + giant + out

    def _cached_for(self, q: Query):
        if not self.reuse:
            return None
        e = self.cached.get((q.gid, q.dual))
        return e if e is not None and e[0] <= q.s else None

    def _keep_list(self, q: Query, res):
        """Keep `res` = L_{q.s} if it is the smallest threshold of its graph
        and side so far and fits the cache."""
        nbytes = 12 * int(res[0].shape[0])
        with self.cv:
            key = (q.gid, q.dual)
            old = self.cached.get(key)
            if old is not None and old[0] <= q.s:
                return
            free = self.cache_bytes - self.cache_used + (old[2] if old else 0)
            if nbytes > free:
                return
            self.cached[key] = (q.s, res, nbytes)
            self.cache_used += nbytes - (old[2] if old else 0)

    # ----------------------------------------------------------------- API --
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
                    if self.in_flight == 0 or self.in_flight + est <= self.budget:
                        del self.pending[k]
                        q.est_bytes = est
                        self.in_flight += est
                        return q
                if self.closed and not self.pending:
                    return None
                self.cv.wait(0.05)

    def _worker(self, k: int):
        import torch
        st = self.streams[k]
        while True:
            q = self._take()
            if q is None:
                return
            q.t_start = time.perf_counter()
            try:
                g = self.graphs[q.gid]
                key = (q.gid, q.s, q.dual)
                for attempt in (0, 1):
                    with self.cv:
                        base = self._cached_for(q)
                    try:
                        with torch.cuda.stream(st):
                            if base is not None:
                                i, j, w = filter_pairs(*base[1], q.s, stream=st)
                                q.reused = True
                            else:
                                n = self.pair_cache.get(key)
                                if n is None:
                                    n = count(g, q.s, q.dual, stream=st)
                                    self.pair_cache[key] = n
                                out = alloc_outputs(n, False, g.e_off.device)
                                i, j, w = build(g, q.s, dual=q.dual, out=out, stream=st)
                            st.synchronize()
                        break
                    except (SlgError, torch.cuda.OutOfMemoryError) as exc:
                        # out of device memory: give the kept lists back, retry once
                        if attempt or getattr(exc, "status", 3) != 3 or not self.reuse:
                            raise
                        base = out = None
                        with self.cv:
                            self.cached.clear()
                            self.cache_used = 0
                        torch.cuda.empty_cache()
                if self.reuse and base is None:
                    self._keep_list(q, (i, j, w))
                q.pairs = int(i.shape[0])
                if self.keep:
                    q.result = (i, j, w)
            except Exception as exc:  # reported on the query
                q.error = exc
            q.t_done = time.perf_counter()
            with self.cv:
                self.in_flight -= q.est_bytes
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
                "answered_by_filter": sum(q.reused for q in queries),
                "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
                "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
                "mean_ms": float(lat.mean()) if lat.size else None,
                "queries_per_s": len(queries) / wall_s if wall_s > 0 else None}
