"""Batched persistent launch (and its CUDA graph) against per-mesh launches
and the oracle, on a scaled-down copy of the 64-mesh workload; plus the
autotuner."""
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


@pytest.fixture(scope="module")
def batch_case():
    items = synth.workload_batched(scale=0.01)
    assert len(items) == 64
    tens = [(dev(m.V), dev(m.T), dev(s.A), dev(s.B), mode) for m, s, mode in items]
    return items, tens


def _np(o):
    return {k: v.cpu().numpy() for k, v in o.items() if isinstance(v, torch.Tensor)}


def test_batched_equals_single_and_oracle(batch_case):
    items, tens = batch_case
    b = rsi.Batch(tens, compact=True)
    outs = b.build().intersect()
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    for k, ((mesh, seg, mode), t) in enumerate(zip(items, tens)):
        got = _np(outs[k])
        single = _np(rsi.BVH(t[0], t[1]).intersect(t[2], t[3], mode))
        key = "flag" if mode == "bool" else "tri"
        np.testing.assert_array_equal(got[key], single[key], err_msg=f"item {k}")
        if mode != "bool":
            np.testing.assert_array_equal(got["tuv"], single["tuv"])
            n = int(got["n_hits"][0])
            assert np.array_equal(np.sort(got["hit_idx"][:n]), np.nonzero(got["tri"] >= 0)[0])
        idx = rng.choice(seg.n, min(200, seg.n), replace=False)
        ref = oracle.brute(mesh.V, mesh.T, seg.A[idx], seg.B[idx])
        if mode == "bool":
            np.testing.assert_array_equal(got["flag"][idx], ref["flag"])
        else:
            np.testing.assert_array_equal(got["tri"][idx], ref["tri"])
            assert_close(got["tuv"][idx], ref["tuv"], what=f"item {k} tuv")
    b.close()


def test_batched_graph_replay(batch_case):
    items, tens = batch_case
    b = rsi.Batch(tens)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        first = [_np(o) for o in b.run_graph(rebuild=True, stream=s)]
        s.synchronize()
        for o in b.outputs:
            for v in o.values():
                if isinstance(v, torch.Tensor):
                    v.zero_()
        again = [_np(o) for o in b.run_graph(rebuild=False, stream=s)]
        s.synchronize()
    for x, y in zip(first, again):
        for k in x:
            np.testing.assert_array_equal(x[k], y[k])
    ref = [_np(o) for o in rsi.Batch(tens).build().intersect()]
    torch.cuda.synchronize()
    for x, y in zip(first, ref):
        for k in x:
            np.testing.assert_array_equal(x[k], y[k])


def test_autotune_returns_valid_config():
    import paper_2209_02878_gb300.tuning as tuning
    mesh, seg = synth.workload_small_bool(n_seg=50000)
    V, T, A, B = dev(mesh.V), dev(mesh.T), dev(seg.A), dev(seg.B)
    bvh = rsi.BVH(V, T)
    best, leaf, table = tuning.autotune(bvh, V, T, A, B, "bool", block_sizes=(128, 256),
                                        stack_depths=(8, 64), smem_nodes=(-1, 511),
                                        leaf_sizes=(1, 4), reps=3, cache=None)
    assert len(table) == 16 + 1  # the grid, then the packet traversal
    assert table[-1].get("packet") == 1 and leaf in (1, 4)
    assert best == {"packet": 1} or best["block_size"] in (128, 256)
    ref = oracle.brute(mesh.V, mesh.T, seg.A, seg.B)
    got = bvh.intersect(A, B, "bool", launch=best)["flag"].cpu().numpy()
    np.testing.assert_array_equal(got, ref["flag"])


def test_batched_full_size_sampled():
    """The full 64-mesh workload (1k-200k triangles, 19.8M segments) in the
    benchmark's configuration (one graph: multi-mesh build + persistent
    traversal), 64 sampled segments per mesh against brute force."""
    items = synth.workload_batched()
    tens = [(dev(m.V), dev(m.T), dev(s.A), dev(s.B), mode) for m, s, mode in items]
    assert sum(s.n for _, s, _ in items) > 10_000_000
    b = rsi.Batch(tens, leaf_size=1, launch=dict(block_size=128, stack_depth=64))
    outs = b.run_graph(rebuild=True)
    torch.cuda.synchronize()
    rng = np.random.default_rng(7)
    for k, (mesh, seg, mode) in enumerate(items):
        idx = np.sort(rng.choice(seg.n, min(64, seg.n), replace=False))
        ref = oracle.brute(mesh.V, mesh.T, seg.A[idx], seg.B[idx])
        if mode == "bool":
            np.testing.assert_array_equal(outs[k]["flag"][idx].cpu().numpy(), ref["flag"],
                                          err_msg=f"item {k}")
        else:
            np.testing.assert_array_equal(outs[k]["tri"][idx].cpu().numpy(), ref["tri"],
                                          err_msg=f"item {k}")
            assert_close(outs[k]["tuv"][idx].cpu().numpy(), ref["tuv"], what=f"item {k} tuv")
    assert b.status() == 0
    b.close()
