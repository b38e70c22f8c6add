"""Sharding of independent surfaces over ranks (one process per GPU).

Surfaces are independent, so ranks need no data exchange: each rank predicts
a disjoint subset. split_by_cost balances ranks by a cost estimate (greedy
longest-processing-time assignment) and is deterministic, so every rank
computes the same partition without communicating.
"""
from typing import List, Sequence


def split_by_cost(costs: Sequence[float], world: int) -> List[List[int]]:
    """Partition indices 0..n-1 into `world` lists with near-equal total cost.
    Heaviest first, each to the currently lightest rank (ties: lowest rank);
    each rank's indices are returned in ascending order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += float(costs[i])
    return [sorted(p) for p in parts]
