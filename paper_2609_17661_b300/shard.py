"""Placement of independent field lines on the ranks of a job (one process
per GPU).  Lines never exchange anything, so a job shards them with no
collective on the data path; only timing and diagnostics are reduced.

Lines are placed largest first, each on the rank with the least load so far
(ties to the lower rank) -- the longest-processing-time rule -- with a line's
weight its particle count (its push work per step).  Every rank computes the
same placement from the same weights.
"""
from __future__ import annotations


def shard_lines(weights, world: int) -> list[list[int]]:
    """The line indices of every rank (each list ascending)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    w = [float(x) for x in weights]
    if any(x < 0 for x in w):
        raise ValueError("weights must be >= 0")
    order = sorted(range(len(w)), key=lambda k: (-w[k], k))
    load = [0.0] * world
    out: list[list[int]] = [[] for _ in range(world)]
    for k in order:
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(k)
        load[r] += w[k]
    return [sorted(o) for o in out]


def my_lines(weights, rank: int, world: int) -> list[int]:
    """The line indices of one rank."""
    return shard_lines(weights, world)[rank]
