"""Splitting one line-graph build over several GPUs (host logic).

The rows of the computed side are independent: row e's pairs depend only on
its own CSR row and the CSC columns of its vertices (the parallel loop over
hyperedges of Section IV-F).  With the incidence replicated on every rank,
the rows are cut into contiguous ranges of about equal wedge work (prefix
sums of the per-row work from slg_row_work), each rank builds its range with
slg_build_rows, and one all-gather of the per-range pair counts gives every
rank the place of its pairs in the canonical list: the ranges are in row
order, so the concatenation of the ranks' lists is the whole list.  No data
moves between ranks while the pairs are counted.
"""
from __future__ import annotations

import numpy as np

__all__ = ["balanced_ranges", "offsets_of", "build_sharded"]


def balanced_ranges(work, parts: int):
    """Cut rows [0, R) into `parts` contiguous ranges of about equal total
    work: boundary k is the first row at which the prefix sum of the work
    reaches k / parts of the total.  Every range's work is within the
    largest single row's work of total / parts.  Returns parts + 1 row
    boundaries (non-decreasing, first 0, last R)."""
    w = np.asarray(work, dtype=np.int64)
    R = int(w.shape[0])
    if parts < 1:
        raise ValueError("parts must be at least 1")
    pre = np.concatenate([[0], np.cumsum(w)])
    total = int(pre[-1])
    bounds = [0]
    for k in range(1, parts):
        target = (total * k + parts - 1) // parts
        b = int(np.searchsorted(pre, target, side="left"))
        bounds.append(min(max(b, bounds[-1]), R))
    bounds.append(R)
    return bounds


def offsets_of(counts):
    """Exclusive prefix sum of the per-range pair counts: where each range's
    pairs start in the canonical list, and the total as the last entry."""
    c = np.asarray(counts, dtype=np.int64)
    return np.concatenate([[0], np.cumsum(c)]).tolist()


def build_sharded(h, s: int, rank: int, world: int, dual: bool = False, group=None,
                  stream=None):
    """This rank's part of L_s: (offset, row range, i, j, w, total).  `h` is
    the whole incidence on this rank's GPU (a DeviceHypergraph); the row
    ranges are computed identically on every rank from the per-row work, and
    one all-gather of the pair counts (torch.distributed, when world > 1)
    places this rank's pairs in the canonical list."""
    import torch

    from . import SlgError, build_rows, row_work
    work = row_work(h, s, dual, stream=stream).cpu().numpy()
    bounds = balanced_ranges(work, world)
    a, b = bounds[rank], bounds[rank + 1]
    try:
        i, j, w = build_rows(h, s, a, b, dual=dual, capacity=0, stream=stream)
    except SlgError as exc:
        if exc.status != 2:
            raise
        i, j, w = build_rows(h, s, a, b, dual=dual, capacity=max(exc.needed, 1), stream=stream)
    counts = [int(i.shape[0])]
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([counts[0]], dtype=torch.int64)
        if dist.get_backend(group) == "nccl":
            t = t.to(i.device)
        allc = [torch.zeros_like(t) for _ in range(world)]
        dist.all_gather(allc, t, group=group)
        counts = [int(x.item()) for x in allc]
    off = offsets_of(counts)
    return off[rank if world > 1 else 0], (a, b), i, j, w, off[-1]
