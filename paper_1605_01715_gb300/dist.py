"""Host-side sharding of independent FMM instances across ranks (one GPU per rank).

The boundary-integral matvecs of different bodies or requests are independent, so
several GPUs run disjoint sets of instances with no collective on the data path
(weak scaling).  The only collectives are the timing barrier and the max-reduce of
the per-rank step time, and the optional gather of per-rank results.
"""
from __future__ import annotations

import heapq


def shard_instances(sizes, world_size):
    """Longest-processing-time partition: instance ids per rank, balanced by size.

    Deterministic (ties broken by instance id, then by rank), so every rank computes
    the same assignment without communicating.
    """
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i], i))
    heap = [(0, r) for r in range(world_size)]
    heapq.heapify(heap)
    out = [[] for _ in range(world_size)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + sizes[i], r))
    for ids in out:
        ids.sort()
    return out


def max_over_ranks(value, group=None):
    """Max of a float over all ranks (the step time the job reports)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def gather_to_rank0(obj, group=None):
    """List of every rank's `obj` on rank 0 (None elsewhere)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return [obj]
    out = [None] * dist.get_world_size(group) if dist.get_rank(group) == 0 else None
    dist.gather_object(obj, out, dst=0, group=group)
    return out
