"""Sharding one graph's count across ranks (host logic).

Every embedding has exactly one root vertex (see gpm_count_roots in
include/gpm.h), so a partition of [0, n) into root ranges partitions the
count: rank r counts the roots in its range on its own GPU and the partial
counts are summed once at the end. This is the paper's task parallelism over
root vertices (Section 4.1 "Search Strategies": one task per vertex) lifted to
one range of tasks per GPU.

The ranges balance an estimate of the per-root cost, d+(u)^2 (d+ the
out-degree in the degree orientation), over contiguous id ranges. The sum is
exact for uint64 counts: each count is split into 32-bit halves before the
all-reduce so no partial sum can round or overflow an int64.
"""
from __future__ import annotations

import numpy as np


def root_costs(rowptr: np.ndarray, col: np.ndarray, key: np.ndarray | None = None) -> np.ndarray:
    """Estimated cost per root: (out-degree in the orientation)^2 + 1.

    key: the order's key per vertex (ties to the larger id), by default the
    degree; for the core value based orientation pass the peel round of each
    vertex (its roots then follow that order)."""
    d = np.diff(rowptr).astype(np.int64)
    n = len(d)
    kv = d if key is None else np.asarray(key, dtype=np.int64)
    src = np.repeat(np.arange(n, dtype=np.int64), d)
    dst = col.astype(np.int64)
    out = (kv[src] < kv[dst]) | ((kv[src] == kv[dst]) & (src < dst))
    od = np.bincount(src[out], minlength=n)
    return od.astype(np.float64) ** 2 + 1.0


def partition(costs: np.ndarray, world: int) -> list:
    """Contiguous root ranges [(lo, hi), ...], one per rank, with near-equal total cost."""
    n = len(costs)
    if world < 1:
        raise ValueError("world must be >= 1")
    pre = np.concatenate([[0.0], np.cumsum(costs, dtype=np.float64)])
    total = pre[-1]
    cuts = [0]
    for r in range(1, world):
        cuts.append(int(np.searchsorted(pre, total * r / world, side="left")))
    cuts.append(n)
    cuts = np.maximum.accumulate(np.clip(cuts, 0, n))
    return [(int(cuts[i]), int(cuts[i + 1])) for i in range(world)]


def split_u64(counts) -> np.ndarray:
    """uint64 counts -> int64 array [lo32..., hi32...] safe to sum across ranks."""
    c = np.asarray([int(x) for x in counts], dtype=object)
    lo = np.array([int(x) & 0xFFFFFFFF for x in c], dtype=np.int64)
    hi = np.array([int(x) >> 32 for x in c], dtype=np.int64)
    return np.concatenate([lo, hi])


def join_u64(parts: np.ndarray, k: int) -> list:
    lo, hi = parts[:k], parts[k:]
    return [(int(h) << 32) + int(l) for l, h in zip(lo, hi)]


def allreduce_counts(counts, group=None) -> list:
    """Sum per-rank uint64 counts over the process group (exact)."""
    import torch
    import torch.distributed as dist
    k = len(counts)
    t = torch.from_numpy(split_u64(counts))
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return join_u64(t.cpu().numpy(), k)


def sharded_count(count_range, n: int, costs: np.ndarray, rank: int, world: int, group=None) -> list:
    """count_range(lo, hi) -> per-pattern counts for roots in [lo, hi); returns the global counts."""
    lo, hi = partition(costs, world)[rank]
    part = count_range(lo, hi)
    if world == 1:
        return [int(x) for x in part]
    return allreduce_counts(part, group)
