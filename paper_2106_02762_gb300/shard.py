"""One graph counted by several processes (one per GPU).

Alg. 1 counts every static triangle on its own, so the triangle list can be
divided: each rank loads the same edges (the load is deterministic, so every
rank holds the same bins), counts its shard with ``Graph.count_shard`` and
the ranks add their counts.  The sum is the only exchange, 64 bytes per
query.

The counts are unsigned 64-bit integers, which torch.distributed cannot add
directly: each is split into 32-bit halves, the halves are summed as int64
(exact for fewer than 2^31 ranks) and recombined, and a total of 2^64 or
more raises OverflowError instead of wrapping.
"""
from __future__ import annotations

import numpy as np


def allreduce_counts(counts, device=None, group=None) -> np.ndarray:
    """Exact sum of uint64 count arrays over the ranks of `group` (the
    default process group if None); device: where the collective's tensors
    live (None = host, e.g. for gloo; a CUDA device for NCCL)."""
    import torch
    import torch.distributed as dist
    c = np.ascontiguousarray(counts, dtype=np.uint64)
    halves = np.stack([(c & np.uint64(0xFFFFFFFF)).astype(np.int64), (c >> np.uint64(32)).astype(np.int64)])
    t = torch.from_numpy(halves)
    if device is not None:
        t = t.to(device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    lo, hi = t.cpu().numpy().astype(object)
    total = [int(h) * (1 << 32) + int(x) for h, x in zip(hi.ravel(), lo.ravel())]
    if any(v >= 1 << 64 for v in total):
        raise OverflowError("a count summed over the ranks exceeds 2^64 - 1")
    return np.array(total, dtype=np.uint64).reshape(c.shape)


def count_sharded(graph, deltas, rank: int, world: int, device=None, group=None) -> np.ndarray:
    """This rank's shard of ``graph.count_batch(deltas)``, summed over the
    ranks: every rank gets the whole graph's counts ([k][8] uint64)."""
    return allreduce_counts(graph.count_shard(deltas, rank, world), device=device, group=group)
