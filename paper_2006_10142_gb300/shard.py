"""Shot-parallel sharding of a batch over ranks (one process per GPU).

A single grid does not shard (every x line and every y column spans the whole
grid), so multi-GPU runs of one grid are replicas.  A batch of independent
shots shards naturally: each rank advances its own shots and no data crosses
ranks during the time loop.  The partition balances the per-step work, which
is proportional to the grid points n_x * n_y of each shot (longest-processing-
time greedy: largest shots first, each to the least loaded rank).
"""
from __future__ import annotations

from typing import List, Sequence, Tuple


def partition(points: Sequence[int], world: int) -> List[List[int]]:
    """Shot indices per rank; deterministic for a given input."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(points)), key=lambda i: (-points[i], i))
    load = [0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += points[i]
    for p in parts:
        p.sort()
    return parts


def local_shots(shapes: Sequence[Tuple[int, int]], rank: int, world: int) -> List[int]:
    """Shots (indices into `shapes` = [(nx, ny), ...]) owned by `rank`."""
    return partition([nx * ny for nx, ny in shapes], world)[rank]


def imbalance(points: Sequence[int], world: int) -> float:
    """max rank load / mean rank load of the partition (1.0 = perfect)."""
    parts = partition(points, world)
    loads = [sum(points[i] for i in p) for p in parts]
    mean = sum(loads) / world
    return max(loads) / mean if mean > 0 else 1.0
