"""Multi-rank helpers: how the work of one graph, or of a batch of graphs, is
split over ranks (one GPU each) and how partial results are combined.

* One graph: every rank builds the same oriented CSR and runs its shard of
  the count (tc_count_shard); the partial total and per-vertex counts are
  summed with one all-reduce of 8(n+1) bytes.  This is the path's only
  exchange step.
* A batch: graphs are independent problems, so ranks take contiguous graph
  ranges of about equal edge count and exchange nothing but the per-graph
  totals at the end (for reporting).

Process groups are plain torch.distributed groups (NCCL on GPUs, gloo on
CPU for the tests).
"""
from __future__ import annotations

import numpy as np


def graph_ranges(edge_off, world: int):
    """Contiguous graph ranges [lo, hi) per rank with about equal edge counts."""
    eo = np.asarray(edge_off, dtype=np.int64)
    G = eo.shape[0] - 1
    if world < 1:
        raise ValueError("world must be >= 1")
    total = int(eo[-1])
    cuts = [0]
    for r in range(1, world):
        target = total * r // world
        cuts.append(int(np.searchsorted(eo[:-1], target, side="left")))
    cuts.append(G)
    for i in range(1, len(cuts)):
        cuts[i] = max(cuts[i], cuts[i - 1])
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def shard_bounds(n_all: int, shard: int, nshards: int):
    """[lo, hi) of a work list of n_all units that shard `shard` of `nshards`
    takes: the same integer arithmetic the count kernels apply to each of their
    work lists (CTA items, warp items, small-class source rows) under
    tc_count_shard, so that the shards cover every unit exactly once."""
    if nshards < 1 or not 0 <= shard < nshards:
        raise ValueError("shard must be in [0, nshards)")
    return n_all * shard // nshards, n_all * (shard + 1) // nshards


def allreduce_counts(total, per_vertex=None, group=None):
    """Sum partial counts over the ranks in place (int64 tensors)."""
    import torch.distributed as dist
    dist.all_reduce(total, op=dist.ReduceOp.SUM, group=group)
    if per_vertex is not None:
        dist.all_reduce(per_vertex, op=dist.ReduceOp.SUM, group=group)
    return total, per_vertex


def count_sharded_one_device(ctx, o, nshards: int, total, per_vertex=None, stream=None):
    """Run every shard of one oriented CSR on this device and add the partial
    results: what the ranks of a multi-GPU count produce together."""
    import torch
    acc_t = torch.zeros_like(total)
    acc_pv = torch.zeros_like(per_vertex) if per_vertex is not None else None
    for sh in range(nshards):
        ctx.count_shard(o, sh, nshards, total, per_vertex, stream)
        acc_t += total
        if acc_pv is not None:
            acc_pv += per_vertex
    total.copy_(acc_t)
    if per_vertex is not None:
        per_vertex.copy_(acc_pv)
    return total, per_vertex
