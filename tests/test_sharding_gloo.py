"""The multi-rank path on the CPU: two gloo ranks split the segments with
shard_range, compute their shard with the FP64 oracle, and (a) the gathered
forward outputs equal the unsharded ones, (b) the all-reduced vertex
gradient equals the unsharded gradient.  Also the LPT batch assignment."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2209_02878_gb300 import sharding, synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _case():
    mesh, seg, w = synth.workload_diff(n_seg=3000, G=33)
    return mesh, seg, w


def _worker(rank, world, port, out_dir):
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mesh, seg, w = _case()
        lo, hi = sharding.shard_range(seg.n, rank, world)
        o = oracle.brute(mesh.V, mesh.T, seg.A[lo:hi], seg.B[lo:hi], threads=1)
        gV, _, _ = oracle.backward(mesh.V, mesh.T, seg.A[lo:hi], seg.B[lo:hi], o["tri"],
                                   gP=w[lo:hi].astype(np.float64))
        g = torch.from_numpy(gV)
        sharding.allreduce_grad(g)
        parts = [None] * world
        dist.all_gather_object(parts, o["tri"])  # outputs gathered to every rank
        if rank == 0:
            np.save(os.path.join(out_dir, "gV.npy"), g.numpy())
            np.save(os.path.join(out_dir, "tri.npy"), np.concatenate(parts))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_sharding(tmp_path, orc):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    mesh, seg, w = _case()
    full = orc.brute(mesh.V, mesh.T, seg.A, seg.B)
    tri = np.load(tmp_path / "tri.npy")
    np.testing.assert_array_equal(tri, full["tri"])
    gV_full, _, _ = orc.backward(mesh.V, mesh.T, seg.A, seg.B, full["tri"], gP=w.astype(np.float64))
    gV = np.load(tmp_path / "gV.npy")
    assert np.allclose(gV, gV_full, rtol=1e-12, atol=1e-12)


def test_shard_range_covers_everything():
    for n in (0, 1, 7, 10, 1001):
        for world in (1, 2, 3, 8):
            r = [sharding.shard_range(n, k, world) for k in range(world)]
            assert r[0][0] == 0 and r[-1][1] == n
            assert all(r[k][1] == r[k + 1][0] for k in range(world - 1))
            assert max(b - a for a, b in r) - min(b - a for a, b in r) <= 1


def test_lpt_assignment_balances():
    costs = [sharding.batch_cost(t, r) for t, r in
             [(1000, 10**4), (2 * 10**5, 2 * 10**6), (5000, 10**5), (81920, 5 * 10**5),
              (20480, 10**6), (1280, 2 * 10**6)]]
    a = sharding.lpt_assign(costs, 3)
    assert sorted(k for part in a for k in part) == list(range(len(costs)))
    loads = [sum(costs[k] for k in part) for part in a]
    assert max(loads) <= 1.34 * (sum(costs) / 3) + max(costs)
