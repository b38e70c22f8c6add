"""Sharding over ranks (one process per GPU): independent surfaces, and one
surface's rows.

Surfaces are independent, so ranks need no data exchange: each rank predicts
a disjoint subset. split_by_cost balances ranks by a cost estimate (greedy
longest-processing-time assignment) and is deterministic, so every rank
computes the same partition without communicating.
"""
import math
from typing import Dict, List, Sequence, Tuple


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


# ---------------------------------------------------------------------------
# One surface over several ranks: row bands.
#
# Cells are independent given the (replicated) tool path, so rank r can
# predict rows [k0, k1) of the map alone: the same process with the grid
# origin moved to row k0 and k1 - k0 rows. The band maps are the full map's
# rows (a point exactly on a band's lower edge is a sampling-boundary tie,
# which the parity tests exempt anyway). The roughness of the whole map then
# needs two small all-reduces of the bands' moment partials
# (fsm_moment_partials): the cell count, sum, min and max give the mean; the
# sums of |d|, d^2, d^3, d^4 about that mean give Sa, Sq, Ssk, Sku.
# ---------------------------------------------------------------------------
def row_bands(ny: int, world: int) -> List[Tuple[int, int]]:
    """Split rows 0..ny-1 into `world` contiguous bands [k0, k1), sizes
    differing by at most one row (empty bands when world > ny)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    q, r = divmod(ny, world)
    bands, k = [], 0
    for i in range(world):
        n = q + (1 if i < r else 0)
        bands.append((k, k + n))
        k += n
    return bands


def band_process(proc, k0: int, k1: int):
    """The process of rows [k0, k1) of `proc`'s map (a ProcessSpec)."""
    if not (0 <= k0 < k1 <= proc.ny):
        raise ValueError("band outside the map")
    return proc.replace(y0=proc.y0 + k0 * proc.pitch, ny=k1 - k0)


# the partials of an empty band (a rank with no rows)
EMPTY_PARTIALS = (0.0, 0.0, float("inf"), float("-inf"), 0.0, 0.0, 0.0, 0.0)


def merge_moments(first: Sequence[float], second: Sequence[float], about0: float = 0.0) -> Dict[str, float]:
    """Areal roughness (Section 4.1.2 definitions) from the bands' summed
    partials: `first` about `about0` (cells, sum d, min, max, ...), `second`
    about the map's mean (..., sum |d|, sum d^2, sum d^3, sum d^4)."""
    n = float(first[0])
    mean = about0 + float(first[1]) / n
    zmin, zmax = float(first[2]), float(first[3])
    sa = float(second[4]) / n
    sq = math.sqrt(float(second[5]) / n)
    out = {"n": n, "mean": mean, "zmin": zmin, "zmax": zmax, "Sa": sa, "Sq": sq, "Sp": zmax - mean,
           "Sv": mean - zmin}
    out["Sz"] = out["Sp"] + out["Sv"]
    if sq > 0.0:
        out["Ssk"] = float(second[6]) / n / sq ** 3
        out["Sku"] = float(second[7]) / n / sq ** 4
    else:
        out["Ssk"] = out["Sku"] = float("nan")
    return out


def allreduce_moments(local: Sequence[float], group=None) -> List[float]:
    """Sum the bands' partials over ranks (min / max for entries 2 / 3):
    torch.distributed all-reduces of 8 doubles in all."""
    import torch
    import torch.distributed as dist
    v = torch.tensor([float(x) for x in local], dtype=torch.float64)
    s = v[[0, 1, 4, 5, 6, 7]].clone()
    lo, hi = v[2:3].clone(), v[3:4].clone()
    dist.all_reduce(s, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(lo, op=dist.ReduceOp.MIN, group=group)
    dist.all_reduce(hi, op=dist.ReduceOp.MAX, group=group)
    return [s[0].item(), s[1].item(), lo.item(), hi.item(), s[2].item(), s[3].item(), s[4].item(), s[5].item()]


def distributed_roughness(partials_about, about0: float = 0.0, group=None) -> Dict[str, float]:
    """Whole-map roughness of a map split in row bands over ranks.
    partials_about(about) returns this rank's band partials about `about`
    (e.g. Context.moment_partials of its band map); every rank gets the
    same result."""
    first = allreduce_moments(partials_about(about0), group)
    mean = about0 + first[1] / first[0]
    second = allreduce_moments(partials_about(mean), group)
    return merge_moments(first, second, about0)
