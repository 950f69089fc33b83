"""Splitting one linewidth problem, or its adjoint, over ranks (host-side logic, one GPU per rank).

Im Sigma_nk of Eq. (linewidthel) is independent for every k, and the BZ
integral is a weighted sum over q, so one problem splits two ways without any
exchange inside the computation:

* ``mode="k"``: rank r evaluates a contiguous slice of the k list against all q;
  the slices are concatenated.
* ``mode="q"``: rank r evaluates all k against a contiguous slice of the q list
  (with the global weights, 1/N_q when none are given); the partial linewidths
  are added in rank order with a compensated (Neumaier) FP64 sum, so the result
  does not depend on arrival order and keeps the per-rank sums' accuracy.

The adjoint of L = sum_nk c_nk Im Sigma_nk is a sum over (k, q) pairs in either
split: dL/dg(Re, Rp), dL/dT and dL/dE_F of the shards are added in rank order
with the same compensated sum, the vertex gradient in bounded chunks.

``compute(k, q, wq) -> [len(k), nw]`` is the per-rank evaluation (e.g.
``Model.linewidth``), ``compute_bwd(k, q, cot, wq) -> (dg, dT, dEF)`` the
per-rank adjoint (e.g. ``Model.linewidth_backward``); numpy arrays or torch
tensors (CUDA tensors exchange through NCCL, host ones through gloo).  Results
come back in the kind the callback returned.  The exchange is torch.distributed
all_gather of fixed-size float64 tensors (no pickling).
"""
from __future__ import annotations

import numpy as np

# vertex-gradient elements (float64) exchanged per all_gather round
_CHUNK = 1 << 23


def shard_bounds(n: int, rank: int, world: int):
    """[lo, hi) of the rank-th of `world` near-equal contiguous slices of range(n)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def compensated_sum(parts):
    """sum(parts) in list order, Neumaier-compensated, elementwise (float64 torch tensors or arrays).

    s_i = s_{i-1} + p_i; the rounding error of each addition, (s - t) + p when |s| >= |p| else
    (p - t) + s, is accumulated in c and added once at the end."""
    import torch
    where = torch.where if isinstance(parts[0], torch.Tensor) else np.where
    s = parts[0] * 1.0
    c = s * 0.0
    for p in parts[1:]:
        t = s + p
        c = c + where(abs(s) >= abs(p), (s - t) + p, (p - t) + s)
        s = t
    return s + c


def _as_tensor(x):
    """(float64 torch tensor view of x, restore function back to x's kind)."""
    import torch
    if isinstance(x, torch.Tensor):
        cplx = x.is_complex()
        t = torch.view_as_real(x.contiguous()) if cplx else x.contiguous()
        t = t.to(torch.float64)
        return t, (lambda y: torch.view_as_complex(y.contiguous()) if cplx else y)
    a = np.asarray(x)
    cplx = np.iscomplexobj(a)
    t = torch.from_numpy(np.ascontiguousarray(a.view(np.float64) if cplx else a.astype(np.float64)))
    return t, (lambda y: y.numpy().view(np.complex128) if cplx else y.numpy())


def _gather_rows(t, counts, group):
    """All ranks' row blocks (rows counts[r] on rank r), concatenated in rank order."""
    import torch
    import torch.distributed as dist
    nmax = max(counts)
    pad = torch.zeros((nmax,) + tuple(t.shape[1:]), dtype=t.dtype, device=t.device)
    pad[:t.shape[0]] = t
    parts = [torch.empty_like(pad) for _ in counts]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([p[:n] for p, n in zip(parts, counts)])


def ordered_sum(t, group=None, chunk: int = _CHUNK):
    """Sum of the ranks' float64 tensors t (same shape everywhere) in rank order, compensated;
    exchanged in chunks of at most `chunk` elements (every rank holds world x chunk at a time)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    flat = t.reshape(-1)
    out = torch.empty_like(flat)
    for lo in range(0, flat.numel(), chunk):
        piece = flat[lo:lo + chunk].contiguous()
        parts = [torch.empty_like(piece) for _ in range(world)]
        dist.all_gather(parts, piece, group=group)
        out[lo:lo + chunk] = compensated_sum(parts)
    return out.reshape(t.shape)


def _to_backend(t, group):
    import torch
    import torch.distributed as dist
    if dist.get_backend(group) == "nccl" and not t.is_cuda:
        return t.to(torch.device("cuda", torch.cuda.current_device()))
    if dist.get_backend(group) != "nccl" and t.is_cuda:
        return t.cpu()
    return t


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
    t, back = _as_tensor(part)
    src_dev = t.device
    t = _to_backend(t, group)
    if mode == "k":
        counts = [shard_bounds(len(k), r, world)[1] - shard_bounds(len(k), r, world)[0] for r in range(world)]
        full = _gather_rows(t, counts, group)
    else:
        full = ordered_sum(t, group)
    return back(full.to(src_dev))


def linewidth_backward_sharded(compute_bwd, k, q, cot, wq=None, mode: str = "k", group=None):
    """(dL/dg, dL/dT, dL/dE_F) of L = sum_nk cot_nk Im Sigma_nk on every rank, each rank
    computing the adjoint of one shard; the shards' gradients are added in rank order
    (compensated FP64)."""
    import torch
    import torch.distributed as dist

    k = np.ascontiguousarray(k, dtype=np.float64).reshape(-1, 3)
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1, 3)
    cot = np.ascontiguousarray(cot, dtype=np.float64).reshape(len(k), -1)
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    wq = np.full(len(q), 1.0 / len(q)) if wq is None else np.ascontiguousarray(wq, dtype=np.float64)
    if mode == "k":
        lo, hi = shard_bounds(len(k), rank, world)
        dg, dT, dE = compute_bwd(k[lo:hi], q, cot[lo:hi], wq)
    elif mode == "q":
        lo, hi = shard_bounds(len(q), rank, world)
        dg, dT, dE = compute_bwd(k, q[lo:hi], cot, wq[lo:hi])
    else:
        raise ValueError("mode must be 'k' or 'q'")
    t, back = _as_tensor(dg)
    src_dev = t.device
    t = _to_backend(t, group)
    dg_sum = back(ordered_sum(t, group).to(src_dev))
    sc = _to_backend(torch.tensor([float(dT), float(dE)], dtype=torch.float64), group)
    sc = ordered_sum(sc, group).cpu()
    return dg_sum, float(sc[0]), float(sc[1])
