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


def _step_worker(rank, world, port, out_dir):
    """The product helper nearest_backward_shard on a gloo rank, its two
    compute steps supplied by the FP64 oracle (no GPU here)."""
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mesh, seg, w = _case()
        A, B, W = (torch.from_numpy(x) for x in (seg.A, seg.B, w))
        gt = torch.from_numpy(np.random.default_rng(7).normal(size=(seg.n, 3)).astype(np.float32))

        def forward(a, b):
            return {"tri": oracle.brute(mesh.V, mesh.T, a.numpy(), b.numpy(), threads=1)["tri"]}

        def backward(tri, a, b, gp, g_tuv):
            gV, gA, gB = oracle.backward(mesh.V, mesh.T, a.numpy(), b.numpy(), tri,
                                         gP=gp.numpy().astype(np.float64),
                                         gtuv=g_tuv.numpy().astype(np.float64))
            return torch.from_numpy(gV), torch.from_numpy(gA), torch.from_numpy(gB)

        r = sharding.nearest_backward_shard(None, None, A, B, grad_point=W, grad_tuv=gt,
                                            forward=forward, backward=backward)
        lo, hi = r["range"]
        parts = [None] * world
        dist.all_gather_object(parts, (lo, hi, r["out"]["tri"], r["grad_A"].numpy(),
                                       r["grad_B"].numpy()))
        if rank == 0:
            np.save(os.path.join(out_dir, "step_gV.npy"), r["grad_V"].numpy())
            parts.sort(key=lambda p: p[0])
            assert parts[0][0] == 0 and parts[-1][1] == seg.n
            for k in range(len(parts) - 1):
                assert parts[k][1] == parts[k + 1][0]
            np.save(os.path.join(out_dir, "step_tri.npy"), np.concatenate([p[2] for p in parts]))
            np.save(os.path.join(out_dir, "step_gA.npy"), np.concatenate([p[3] for p in parts]))
            np.save(os.path.join(out_dir, "step_gB.npy"), np.concatenate([p[4] for p in parts]))
        else:
            # every rank holds the summed vertex gradient
            np.save(os.path.join(out_dir, f"step_gV_{rank}.npy"), r["grad_V"].numpy())
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_nearest_backward_step(tmp_path, orc):
    """nearest_backward_shard on two gloo ranks: the shards tile the
    segments, the gathered ids and segment gradients equal the unsharded
    ones, and every rank ends with the unsharded vertex gradient."""
    world = 2
    mp.start_processes(_step_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    mesh, seg, w = _case()
    gt = np.random.default_rng(7).normal(size=(seg.n, 3)).astype(np.float32)
    full = orc.brute(mesh.V, mesh.T, seg.A, seg.B)
    np.testing.assert_array_equal(np.load(tmp_path / "step_tri.npy"), full["tri"])
    gV, gA, gB = orc.backward(mesh.V, mesh.T, seg.A, seg.B, full["tri"],
                              gP=w.astype(np.float64), gtuv=gt.astype(np.float64))
    for name, ref in (("step_gV.npy", gV), ("step_gV_1.npy", gV), ("step_gA.npy", gA),
                      ("step_gB.npy", gB)):
        np.testing.assert_allclose(np.load(tmp_path / name), ref, rtol=1e-12, atol=1e-12,
                                   err_msg=name)


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
