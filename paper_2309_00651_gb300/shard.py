"""Pair-list sharding for several processes (one per GPU), in the manner of the paper's CP groups
(Sec. 2.2): every rank holds all orbitals, evaluates a subset of the pairs, and one global sum of
E_x and V_x phi completes the exchange.

The partition is balanced by pair count and deterministic; `reduce_exchange` is the single
exchange step (a sum over ranks).  Only host logic lives here: each rank's evaluation is a normal
hfx_apply on its subset.
"""
from __future__ import annotations

import numpy as np


def partition_pairs(pairs: np.ndarray, world: int, rank: int) -> np.ndarray:
    """Rank `rank`'s share of `pairs` [P, 2]: every world-th pair, starting at `rank`.

    Pairs are first ordered by (i, j) so that the shares interleave across the triangle and carry
    near-equal numbers of diagonal and off-diagonal pairs whatever the input order.
    """
    if world < 1 or not (0 <= rank < world):
        raise ValueError("need world >= 1 and 0 <= rank < world")
    pairs = np.asarray(pairs, dtype=np.int32).reshape(-1, 2)
    order = np.lexsort((pairs[:, 1], pairs[:, 0]))
    return np.ascontiguousarray(pairs[order][rank::world])


def reduce_exchange(E, V, group=None):
    """Sum E_x and V_x phi over the ranks of `group` (torch.distributed), in place."""
    import torch.distributed as dist
    dist.all_reduce(E, op=dist.ReduceOp.SUM, group=group)
    if V is not None:
        dist.all_reduce(V, op=dist.ReduceOp.SUM, group=group)
    return E, V
