"""The current of one step recomputed by the oracle's integer deposit (test
helper, not collected).

Given the particles before a step and every slot of the device's state after
it (removed slots included), the path of each particle that was alive at the
start runs from its old to its new fixed-point position; a particle that
left through a wall ends at that wall (node 0 or node N), and one removed
for a non-finite momentum carries no current.  Pairs and supply created in
the step are neutral and absent from the "before" state.  The oracle's
``deposit_int`` (the charge-conserving deposit of Sec. 3 in int64) then
gives the current of every cell, the wall cells included.
"""
import numpy as np

import oracle as O
from paper_2609_17661_b300 import workloads as W

DEAD = 255


def step_paths(before: dict, after: dict, n_cells: int):
    """(p0, p1, w, sp) int64/float64/int32 arrays of the particles alive in
    `before`, with p1 their position after the step (walls for losses)."""
    F = W.fbits(n_cells)
    top = n_cells << F
    alive = before["sp"] != DEAD
    bid = before["id"][alive]
    order = np.argsort(after["id"])
    aid = after["id"][order]
    k = np.searchsorted(aid, bid)
    assert np.all(k < aid.size) and np.array_equal(aid[k], bid), "a particle of the step is missing after it"
    j = order[k]
    p0 = before["pos"][alive].astype(np.int64)
    p1 = after["pos"][j].astype(np.int64)
    dead = after["sp"][j] == DEAD
    c0 = p0 >> F
    north = dead & (p1 == 0) & (c0 == 0)
    south = dead & (p1 == top - 1) & (c0 == n_cells - 1)
    p1 = np.where(north, 0, np.where(south, top, p1))
    p1 = np.where(dead & ~north & ~south, p0, p1)          # removed in place: no current
    return p0, p1, before["w"][alive].astype(np.float64), before["sp"][alive].astype(np.int32)


def step_current(before: dict, after: dict, n_cells: int) -> np.ndarray:
    p0, p1, w, sp = step_paths(before, after, n_cells)
    return O.deposit_int(n_cells, W.fbits(n_cells), p0, p1, w, sp)
