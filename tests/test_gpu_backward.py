"""GPU adjoint (rsi_intersect_backward through RSIFunction) against the FP64
CPU adjoint and FP64 central finite differences, on the differentiable
workload: 257x257 heightfield (131,072 triangles), 262,144 near-vertical
segments, loss = sum_i w_i . P_i with w ~ N(0, I3)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2209_02878_gb300 as rsi
from paper_2209_02878_gb300 import synth

from _util import assert_close

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def rel_l2(g, ref):
    return float(np.linalg.norm(g - ref) / max(np.linalg.norm(ref), 1e-30))


def elementwise_ok(g, ref, idx, rel=1e-5):
    scale = np.maximum(np.abs(ref[idx]), 1e-3 * np.abs(ref).max())
    return np.abs(g[idx] - ref[idx]) <= rel * scale


@pytest.fixture(scope="module")
def diff_case():
    mesh, seg, w = synth.workload_diff()
    assert mesh.n_tri == 131072 and seg.n == 262144
    ref = oracle.CpuBVH(mesh.V, mesh.T).query(seg.A, seg.B)
    V = dev(mesh.V).requires_grad_(True)
    A = dev(seg.A).requires_grad_(True)
    B = dev(seg.B).requires_grad_(True)
    P, tuv, tri = rsi.nearest_hit(V, dev(mesh.T), A, B)
    loss = (P * dev(w)).sum()
    loss.backward()
    torch.cuda.synchronize()
    got = dict(tri=tri.cpu().numpy(), P=P.detach().cpu().numpy(),
               gV=V.grad.cpu().numpy().astype(np.float64),
               gA=A.grad.cpu().numpy().astype(np.float64),
               gB=B.grad.cpu().numpy().astype(np.float64))
    gV, gA, gB = oracle.backward(mesh.V, mesh.T, seg.A, seg.B, ref["tri"], gP=w.astype(np.float64))
    return mesh, seg, w, ref, got, dict(gV=gV, gA=gA, gB=gB)


def test_forward_ids_match(diff_case):
    mesh, seg, w, ref, got, _ = diff_case
    np.testing.assert_array_equal(got["tri"], ref["tri"])
    assert (ref["tri"] >= 0).mean() > 0.99


@pytest.mark.parametrize("key", ["gV", "gA", "gB"])
def test_adjoint_vs_fp64_adjoint(diff_case, key):
    _, _, _, _, got, adj = diff_case
    assert rel_l2(got[key], adj[key]) <= 1e-5
    rng = np.random.default_rng(0)
    flat_g, flat_r = got[key].ravel(), adj[key].ravel()
    nz = np.nonzero(flat_r)[0]
    idx = rng.choice(nz, min(1000, nz.size), replace=False)
    assert elementwise_ok(flat_g, flat_r, idx).all()


def test_adjoint_vs_finite_differences(diff_case):
    mesh, seg, w, ref, got, adj = diff_case
    tri = np.where(ref["neardeg"] == 0, ref["tri"], -1).astype(np.int32)
    V64, A64, B64 = (mesh.V.astype(np.float64), seg.A.astype(np.float64),
                     seg.B.astype(np.float64))
    rng = np.random.default_rng(1)
    w64 = w.astype(np.float64)

    def loss(Vx, Ax, Bx, idx):
        r = oracle.eval_fixed(Vx, mesh.T, Ax[idx], Bx[idx], tri[idx])
        return float(np.sum(r[:, 3:] * w64[idx]))

    def central(f, x0, h):
        # Richardson extrapolation of central differences: error O(h^4)
        d1 = (f(x0 + h) - f(x0 - h)) / (2 * h)
        d2 = (f(x0 + h / 2) - f(x0 - h / 2)) / h
        return (4 * d2 - d1) / 3

    # vertex -> segments whose crossing triangle uses it
    hit = np.nonzero(tri >= 0)[0]
    corners = mesh.T[tri[hit]]
    order = np.argsort(corners.ravel(), kind="stable")
    keys = corners.ravel()[order]
    segs_of = hit[order // 3]
    used = np.unique(keys)
    checks = []
    for vtx in rng.choice(used, 200, replace=False):
        lo, hi = np.searchsorted(keys, vtx), np.searchsorted(keys, vtx, side="right")
        sidx = segs_of[lo:hi]
        for k in range(3):
            def f(x, vtx=vtx, k=k, sidx=sidx):
                Vx = V64.copy()
                Vx[vtx, k] = x
                return loss(Vx, A64, B64, sidx)
            fd = central(f, V64[vtx, k], 1e-5 * max(1.0, abs(V64[vtx, k])))
            checks.append((fd, got["gV"][vtx, k], adj["gV"][vtx, k]))
    for i in rng.choice(hit, 70, replace=False):
        for which, key in ((A64, "gA"), (B64, "gB")):
            for k in range(3):
                o = which[i, k]

                def f(x, which=which, i=i, k=k):
                    which[i, k] = x
                    return loss(V64, A64, B64, [i])
                fd = central(f, o, 1e-5 * max(1.0, abs(o)))
                which[i, k] = o
                checks.append((fd, got[key][i, k], adj[key][i, k]))
    c = np.array(checks)
    assert len(c) >= 1000
    gmax = max(np.abs(got["gV"]).max(), np.abs(got["gA"]).max(), np.abs(got["gB"]).max())
    # FP64 adjoint vs FD (the oracle's own pin, at this size)
    assert np.all(np.abs(c[:, 2] - c[:, 0]) <= 1e-6 * np.maximum(np.abs(c[:, 0]), 1e-3 * gmax) + 1e-9)
    # GPU vs FD
    assert np.all(np.abs(c[:, 1] - c[:, 0]) <= 1e-5 * np.maximum(np.abs(c[:, 0]), 1e-3 * gmax))


def test_translation_invariance(diff_case):
    """Moving the mesh and the segments together moves every crossing point
    with them: the gradients sum to the sum of dL/dP over the hits (per
    axis).  Each gradient entry is within 1e-5 of its value (relative), so
    the sum is within 1e-5 of the sum of their magnitudes."""
    _, _, w, ref, got, _ = diff_case
    terms = [got["gV"], got["gA"], got["gB"]]
    total = sum(t.sum(0) for t in terms)
    mag = sum(np.abs(t).sum(0) for t in terms)
    want = w[ref["tri"] >= 0].astype(np.float64).sum(0)
    assert np.all(np.abs(total - want) <= 1e-5 * mag), (total, want, mag)


def test_sharded_backward_sums_to_unsharded(diff_case):
    """Segments split into shards (as ranks would hold them): the per-shard
    vertex gradients summed equal the unsharded gradient (the all-reduce a
    multi-GPU run would do)."""
    mesh, seg, w, ref, got, _ = diff_case
    V, T = dev(mesh.V), dev(mesh.T)
    tri = dev(ref["tri"])
    bvh = rsi.BVH(V, T)
    o = bvh.intersect(dev(seg.A), dev(seg.B), "nearest")
    acc = torch.zeros_like(V)
    for sl in np.array_split(np.arange(seg.n), 4):
        s = slice(int(sl[0]), int(sl[-1]) + 1)
        rsi.intersect_backward(V, T, dev(seg.A[s]), dev(seg.B[s]), o["tri"][s].contiguous(),
                               grad_point=dev(w[s]), grad_V=acc)
    torch.cuda.synchronize()
    assert rel_l2(acc.cpu().numpy().astype(np.float64), got["gV"]) <= 1e-6
    assert torch.equal(o["tri"], tri)


def test_reused_tree_follows_optimizer_steps():
    """Three SGD steps on the vertices of the differentiable workload with
    one BVH passed to nearest_hit throughout: each step's forward refits the
    tree to the moved vertices (an in-place optimizer update bumps V's
    version), and its outputs and gradients match the oracle on those
    vertices.  A step moves vertices by up to about a grid cell, so a stale
    tree would miss crossings."""
    mesh, seg, w = synth.workload_diff()
    V = dev(mesh.V).requires_grad_(True)
    T, A, B, W = dev(mesh.T), dev(seg.A), dev(seg.B), dev(w)
    bvh = rsi.BVH(V.detach(), T)
    opt = torch.optim.SGD([V], lr=2e-3)
    moved = 0.0
    for step in range(3):
        Vh = V.detach().cpu().numpy()
        P, tuv, tri = rsi.nearest_hit(V, T, A, B, bvh=bvh)
        opt.zero_grad()
        (P * W).sum().backward()
        torch.cuda.synchronize()
        assert bvh.refits == step
        ref = oracle.CpuBVH(Vh, mesh.T).query(seg.A, seg.B)
        np.testing.assert_array_equal(tri.cpu().numpy(), ref["tri"], err_msg=f"step {step}")
        assert_close(P.detach().cpu().numpy(), ref["point"], what=f"step {step} point")
        assert_close(tuv.detach().cpu().numpy(), ref["tuv"], what=f"step {step} tuv")
        gV, _, _ = oracle.backward(Vh, mesh.T, seg.A, seg.B, ref["tri"], gP=w.astype(np.float64))
        g = V.grad.cpu().numpy().astype(np.float64)
        assert rel_l2(g, gV) <= 1e-5, step
        nz = np.nonzero(gV.ravel())[0]
        idx = np.random.default_rng(step).choice(nz, 1000, replace=False)
        assert elementwise_ok(g.ravel(), gV.ravel(), idx).all(), step
        before = V.detach().clone()
        opt.step()
        moved = max(moved, float((V.detach() - before).abs().max()))
    assert bvh.refits == 2
    assert moved > 1e-3, moved


def test_sharded_step_helper_at_one_rank(diff_case):
    """sharding.nearest_backward_shard on its default CUDA path with no
    process group (one rank, the whole range, no collective) gives the
    unsharded forward and gradients."""
    from paper_2209_02878_gb300 import sharding
    mesh, seg, w, ref, got, _ = diff_case
    V, T = dev(mesh.V), dev(mesh.T)
    r = sharding.nearest_backward_shard(V, T, dev(seg.A), dev(seg.B), grad_point=dev(w))
    torch.cuda.synchronize()
    assert r["range"] == (0, seg.n)
    np.testing.assert_array_equal(r["out"]["tri"].cpu().numpy(), ref["tri"])
    for key, g in (("gV", r["grad_V"]), ("gA", r["grad_A"]), ("gB", r["grad_B"])):
        assert rel_l2(g.cpu().numpy().astype(np.float64), got[key]) <= 1e-6, key


def test_reused_tree_rebuilds_for_new_triangles():
    """BVH.sync with another triangle tensor rebuilds the tree (the
    topology changed), and results follow the new triangles."""
    mesh, seg = synth.workload_small_bool(n_seg=3000)
    V, A, B = dev(mesh.V), dev(seg.A), dev(seg.B)
    T1 = dev(mesh.T)
    T2 = dev(mesh.T[::-1].copy())          # the same triangles in reverse order
    bvh = rsi.BVH(V, T1)
    P1, _, tri1 = rsi.nearest_hit(V, T1, A, B, bvh=bvh)
    P2, _, tri2 = rsi.nearest_hit(V, T2, A, B, bvh=bvh)
    torch.cuda.synchronize()
    assert bvh.T is T2 and bvh.refits == 0
    n = mesh.n_tri
    t1, t2 = tri1.cpu().numpy(), tri2.cpu().numpy()
    hit = t1 >= 0
    # the same crossings, triangle ids mapped through the reversal (except
    # ties on t, which go to the lower index of each numbering)
    ref2 = oracle.brute(mesh.V, mesh.T[::-1].copy(), seg.A, seg.B)
    np.testing.assert_array_equal(t2, ref2["tri"])
    assert np.array_equal(t2 >= 0, hit)
    assert (n - 1 - t2[hit] == t1[hit]).mean() > 0.99


def test_autograd_step_replays_from_a_cuda_graph():
    """The whole training step -- an in-place vertex update, nearest_hit with
    a reused tree (which refits it), the backward pass -- captured once with
    torch.cuda.graph and replayed: after every replay the outputs and the
    vertex gradient match the oracle on the moved vertices (the refit is in
    the graph; nothing of the step needs the host)."""
    rng = np.random.default_rng(17)
    mesh = synth.heightfield(65, rng)
    n = 20000
    xy = rng.uniform(0.02, 0.98, size=(n, 2))
    A_np = np.c_[xy, -np.ones(n)].astype(np.float32)
    B_np = np.c_[xy + rng.normal(0.0, 0.02, size=(n, 2)), np.ones(n)].astype(np.float32)
    w = rng.normal(size=(n, 3)).astype(np.float32)
    step_np = (rng.normal(size=mesh.V.shape) * 2e-3).astype(np.float32)
    V = dev(mesh.V).requires_grad_(True)
    T, A, B, W, D = dev(mesh.T), dev(A_np), dev(B_np), dev(w), dev(step_np)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        bvh = rsi.BVH(V.detach(), T, stream=s)
        P, _, _ = rsi.nearest_hit(V, T, A, B, bvh=bvh)      # warm-up, eager
        (P * W).sum().backward()
        s.synchronize()
        V.grad = None
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            with torch.no_grad():
                V.add_(D)
            P, tuv, tri = rsi.nearest_hit(V, T, A, B, bvh=bvh)
            (P * W).sum().backward()
    assert bvh.refits == 1                                   # captured with the step
    for k in range(3):
        g.replay()
        torch.cuda.synchronize()
        Vh = V.detach().cpu().numpy()
        np.testing.assert_allclose(Vh, mesh.V + (k + 1) * step_np, rtol=0, atol=1e-5)
        ref = oracle.brute(Vh, mesh.T, A_np, B_np)
        np.testing.assert_array_equal(tri.cpu().numpy(), ref["tri"], err_msg=f"replay {k}")
        assert_close(P.detach().cpu().numpy(), ref["point"], what=f"replay {k} point")
        gV, _, _ = oracle.backward(Vh, mesh.T, A_np, B_np, ref["tri"], gP=w.astype(np.float64))
        assert rel_l2(V.grad.cpu().numpy().astype(np.float64), gV) <= 1e-5, k
