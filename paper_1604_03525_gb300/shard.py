"""Splitting one linewidth problem over ranks (host-side logic, one GPU per rank).

Im Sigma_nk of Eq. (linewidthel) is independent for every k, and the BZ
integral is a weighted sum over q, so one problem splits two ways without any
exchange inside the computation:

* ``mode="k"``: rank r evaluates a contiguous slice of the k list against all q;
  the slices are concatenated.
* ``mode="q"``: rank r evaluates all k against a contiguous slice of the q list
  (with the global weights, 1/N_q when none are given); the partial linewidths
  are added in rank order, so the result does not depend on arrival order.

``compute(k, q, wq) -> ndarray [len(k), nw]`` is the per-rank evaluation, e.g.
``Model.linewidth`` with host arrays.  The exchange goes through
``torch.distributed`` (any backend; results are small, Nk x nw doubles).
"""
from __future__ import annotations

import numpy as np


def shard_bounds(n: int, rank: int, world: int):
    """[lo, hi) of the rank-th of `world` near-equal contiguous slices of range(n)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def linewidth_sharded(compute, k, q, wq=None, mode: str = "k", group=None):
    """Full Im Sigma [nk, nw] on every rank, each rank computing one shard."""
    import torch.distributed as dist

    k = np.ascontiguousarray(k, dtype=np.float64).reshape(-1, 3)
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1, 3)
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    wq = np.full(len(q), 1.0 / len(q)) if wq is None else np.ascontiguousarray(wq, dtype=np.float64)
    if mode == "k":
        lo, hi = shard_bounds(len(k), rank, world)
        part = compute(k[lo:hi], q, wq)
    elif mode == "q":
        lo, hi = shard_bounds(len(q), rank, world)
        part = compute(k, q[lo:hi], wq[lo:hi])
    else:
        raise ValueError("mode must be 'k' or 'q'")
    parts = [None] * world
    dist.all_gather_object(parts, np.asarray(part), group=group)
    if mode == "k":
        return np.concatenate(parts, axis=0)
    total = np.zeros_like(parts[0])
    for p in parts:  # fixed rank order
        total = total + p
    return total
