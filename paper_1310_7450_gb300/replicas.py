"""Host-side logic of multi-GPU runs: one process per GPU, no collective on the data path.

The single large channel runs as independent replicas (one per GPU, weak scaling).  The batched
sweep partitions its channels across the ranks -- the channels are independent, so the only
communication is the final reduction of the timing and the counts.  Work per channel is taken as
proportional to its node count times its width (the diffusion time grows as ny^2 and the nodes as
ny), and the channels are dealt out largest first to the least loaded rank, a deterministic
assignment that every rank computes for itself.
"""
from __future__ import annotations

import heapq


def partition_channels(nys, world_size: int, rank: int):
    """Indices of the channels that `rank` runs (sorted), balancing sum(ny^2) over the ranks."""
    if world_size < 1 or not 0 <= rank < world_size:
        raise ValueError("bad world_size / rank")
    order = sorted(range(len(nys)), key=lambda c: (-nys[c], c))
    heap = [(0, r) for r in range(world_size)]
    mine = []
    for c in order:
        load, r = heapq.heappop(heap)
        if r == rank:
            mine.append(c)
        heapq.heappush(heap, (load + nys[c] * nys[c], r))
    return sorted(mine)


def reduce_job(values: dict, world_size: int):
    """Whole-job numbers from per-rank ones: times reduce by max (the job ends with the slowest
    rank), counts by sum.  `values` maps name -> (kind, value) with kind "max" or "sum"; needs an
    initialised torch.distributed group when world_size > 1."""
    if world_size <= 1:
        return {k: v for k, (_, v) in values.items()}
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    out = {}
    for k, (kind, v) in values.items():
        t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX if kind == "max" else dist.ReduceOp.SUM)
        out[k] = float(t.item())
    return out
