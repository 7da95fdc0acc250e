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


def _rank_world(group=None):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(group), dist.get_world_size(group)
    return 0, 1


def nearest_backward_shard(V, T, A, B, grad_point=None, grad_tuv=None, bvh=None, group=None,
                           stream=None, forward=None, backward=None):
    """One rank's part of a data-parallel nearest + adjoint step over the
    segments A -> B (every rank passes the same full arrays and the same
    replicated mesh): the rank takes its contiguous shard_range of the
    segments, runs the nearest forward and the adjoint on its own GPU, and
    the vertex gradients are summed over all ranks with one all-reduce (the
    only collective; the segment gradients and the forward outputs stay
    sharded).

    forward(a, b) -> dict with "tri" and backward(tri, a, b, gp, gt) ->
    (grad_V, grad_A, grad_B) default to the CUDA path (BVH.intersect in
    NEAREST mode on `bvh`, built from (V, T) when None, and
    intersect_backward); they are parameters so that the orchestration can
    run on CPU ranks with other implementations of the two steps.

    Returns dict(range=(lo, hi), out=forward outputs of the shard,
    grad_V=summed over ranks, grad_A, grad_B=of the shard)."""
    rank, world = _rank_world(group)
    lo, hi = shard_range(int(A.shape[0]), rank, world)
    a, b = A[lo:hi], B[lo:hi]
    gp = None if grad_point is None else grad_point[lo:hi]
    gt = None if grad_tuv is None else grad_tuv[lo:hi]
    if forward is None or backward is None:
        from . import BVH, intersect_backward
        if bvh is None and forward is None:
            bvh = BVH(V, T, stream=stream)
        if forward is None:
            forward = lambda a_, b_: bvh.intersect(a_, b_, "nearest", stream=stream)  # noqa: E731
        if backward is None:
            backward = lambda tri, a_, b_, gp_, gt_: intersect_backward(  # noqa: E731
                V, T, a_, b_, tri, gp_, gt_, stream=stream)
    out = forward(a, b)
    gV, gA, gB = backward(out["tri"], a, b, gp, gt)
    allreduce_grad(gV, group)
    return {"range": (lo, hi), "out": out, "grad_V": gV, "grad_A": gA, "grad_B": gB}
