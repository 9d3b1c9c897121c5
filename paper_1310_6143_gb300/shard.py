"""Splitting independent systems across GPUs (statistical parallelism, Appendix C).

Systems of a batch never interact, so N ranks can each advance a subset with no data-path
collective; only the timing (max over ranks) and counts are combined.  Systems are
assigned longest-first to the rank with the fewest spins so far (LPT scheduling), which
keeps the per-rank work within one system of the mean.
"""
from __future__ import annotations

import heapq
from typing import Sequence


def shard_systems(sizes: Sequence[int], world: int) -> list[list[int]]:
    """Indices of the systems of each rank (each list ascending); every system appears once."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda k: (-int(sizes[k]), k))
    heap = [(0, r) for r in range(world)]
    heapq.heapify(heap)
    out: list[list[int]] = [[] for _ in range(world)]
    for k in order:
        load, r = heapq.heappop(heap)
        out[r].append(k)
        heapq.heappush(heap, (load + int(sizes[k]), r))
    return [sorted(v) for v in out]


def rank_systems(sizes: Sequence[int], rank: int, world: int) -> list[int]:
    return shard_systems(sizes, world)[rank]
