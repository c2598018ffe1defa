"""Size-balanced partition of independent problems over ranks (one process per GPU).

A batch of skew matrices, or a stream of requests, is a set of independent
factorizations: with several GPUs each rank takes a share, nothing crosses ranks on
the data path, and only the per-matrix results (log|Pf|, sign, latencies) are gathered
at the end.  A single factorization does not shard (every column step needs a
grid-wide pivot search and a symmetric exchange over the whole trailing matrix), so
one matrix always stays on one GPU.

Shares are balanced by the work of a factorization, n^3/3 flops for order n, with the
longest-processing-time-first rule: matrices in order of decreasing work (ties by
index), each given to the rank with the least work so far (ties to the lower rank).
Its largest share is at most 4/3 - 1/(3 parts) times the optimum (Graham 1969).  The
result depends only on the orders and the number of parts.
"""
from __future__ import annotations

import heapq

import numpy as np


def work_of(orders) -> np.ndarray:
    """n^3 / 3 per order (the flop count of one factorization)."""
    n = np.asarray(orders, dtype=np.float64)
    return n ** 3 / 3.0


def balanced_bins(orders, parts: int) -> list[np.ndarray]:
    """Indices of `orders` split into `parts` shares of near-equal work; each share is
    sorted by index."""
    if parts < 1:
        raise ValueError("parts must be at least 1")
    w = work_of(orders)
    order = sorted(range(len(w)), key=lambda i: (-w[i], i))
    heap = [(0.0, r) for r in range(parts)]
    bins: list[list[int]] = [[] for _ in range(parts)]
    for i in order:
        load, r = heapq.heappop(heap)
        bins[r].append(i)
        heapq.heappush(heap, (load + w[i], r))
    return [np.array(sorted(b), dtype=np.int64) for b in bins]


def imbalance(orders, bins) -> float:
    """Largest share's work over the mean share's work (1.0 = perfect balance)."""
    w = work_of(orders)
    loads = np.array([w[b].sum() for b in bins])
    return float(loads.max() / loads.mean()) if loads.mean() > 0 else 1.0
