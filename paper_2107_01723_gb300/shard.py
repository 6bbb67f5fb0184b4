"""Sharding of a batched scan over several GPUs (one process per GPU).

The targets of a scan are independent, so the scan shards with no exchange
during the run: whole targets go to ranks by greedy longest-processing-time
on their electron counts, each rank steps its own batch, and the per-target
tallies are summed over ranks once at the end (an FP64 all-reduce).  Each
target keeps its global index as its Philox stream, so a sharded scan draws
the same random numbers as the unsharded one.
"""
from __future__ import annotations


def lpt_assign(weights, n_ranks: int) -> list:
    """Greedy longest-processing-time: targets in decreasing weight, each to
    the currently lightest rank (ties: lowest rank).  Returns, per rank, the
    sorted list of target indices.  Its largest load is at most 4/3 of the
    best possible (Graham 1969)."""
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    load = [0.0] * n_ranks
    out = [[] for _ in range(n_ranks)]
    for t in sorted(range(len(weights)), key=lambda i: (-float(weights[i]), i)):
        r = min(range(n_ranks), key=lambda k: (load[k], k))
        load[r] += float(weights[t])
        out[r].append(t)
    return [sorted(a) for a in out]


def reduce_tallies(world: int, totals: dict) -> dict:
    """Sum per-rank FP64 tally totals over all ranks (one all-reduce)."""
    if world == 1:
        return dict(totals)
    import torch
    import torch.distributed as dist
    keys = sorted(totals)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(totals[k]) for k in keys], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return dict(zip(keys, t.tolist()))
