"""Splitting independent grids across ranks.

The grids of a batch never exchange data (each sweep reads only its own
grid's cells), so N processes -- one per GPU -- can advance disjoint subsets
with no collective on the data path.  `lpt_split` balances the subsets by
cell count with the longest-processing-time rule (largest grid first, each to
the rank with the least work so far; ties to the lowest rank), which is
deterministic, so every rank computes the same assignment without
communicating.
"""
from __future__ import annotations

import heapq


def lpt_split(costs, nranks: int) -> list[list[int]]:
    """Indices of `costs` assigned to each of `nranks` ranks (LPT)."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0, r) for r in range(nranks)]
    parts = [[] for _ in range(nranks)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(p) for p in parts]


def shard_of(problems, rank: int, world: int) -> list[int]:
    """This rank's grid indices for a list of problems (cost = cells)."""
    return lpt_split([p.U.shape[1] * p.U.shape[2] for p in problems], world)[rank]
