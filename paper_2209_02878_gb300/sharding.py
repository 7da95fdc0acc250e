"""Host-side sharding of the work across ranks (one process per GPU).

Segments are independent, so a multi-GPU run splits them into contiguous
ranges and replicates the mesh: the forward pass needs no collective.  The
only cross-segment reduction is the vertex gradient of the backward pass,
summed across ranks with one all-reduce.  Batches of meshes are assigned to
ranks whole, longest estimated cost first (LPT), cost ~ N_r log2(N_t).
"""
from __future__ import annotations

import math


def shard_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [lo, hi) of n items for `rank` of `world` (sizes differ by
    at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    q, r = divmod(n, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def batch_cost(n_tri: int, n_seg: int) -> float:
    return n_seg * math.log2(2.0 + n_tri)


def lpt_assign(costs, world: int) -> list[list[int]]:
    """Longest-processing-time-first assignment of items to `world` ranks."""
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for k in sorted(range(len(costs)), key=lambda k: -costs[k]):
        r = min(range(world), key=lambda r: (load[r], r))
        out[r].append(k)
        load[r] += costs[k]
    return out


def allreduce_grad(grad, group=None):
    """Sum a vertex-gradient tensor over all ranks in place (NCCL for CUDA
    tensors, gloo for CPU tensors)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(grad, op=dist.ReduceOp.SUM, group=group)
    return grad
