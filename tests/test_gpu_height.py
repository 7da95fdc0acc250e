"""The height-field option of the build (rsi_build_opts.height_axis: the
Morton code leaves one axis out): the device tree equals the oracle's LBVH
with the same option exactly, and every output equals the oracle's and the
paper-code tree's, since only the tree's shape changes."""
import numpy as np
import pytest
import torch

import oracle
import paper_2209_02878_gb300 as rsi
from paper_2209_02878_gb300 import synth

from _util import assert_close, tree_check

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def outputs(bvh, A, B):
    o = {m: bvh.intersect(A, B, m) for m in ("bool", "count", "nearest")}
    torch.cuda.synchronize()
    return {m: {k: v.cpu().numpy() for k, v in d.items()} for m, d in o.items()}


@pytest.fixture(scope="module")
def small():
    mesh, seg = synth.workload_small_bool()
    return mesh, seg, oracle.brute(mesh.V, mesh.T, seg.A, seg.B)


@pytest.mark.parametrize("axis", [1, 2, 3])
def test_tree_matches_oracle(small, axis):
    mesh, _, _ = small
    bvh = rsi.BVH(dev(mesh.V), dev(mesh.T), height_axis=axis)
    g = bvh.export()
    r = oracle.lbvh(mesh.V, mesh.T, height_axis=axis)
    np.testing.assert_array_equal(g["bounds"], r["bounds"])
    np.testing.assert_array_equal(g["order"], r["order"].astype(np.int32))
    np.testing.assert_array_equal(g["codes"], r["codes"][r["order"]])
    for k in ("left", "right", "range", "nbox", "lbox"):
        np.testing.assert_array_equal(g[k], r[k], err_msg=k)
    tree_check(g, mesh.n_tri)


def test_outputs_match_oracle_and_paper_code(small):
    mesh, seg, ref = small
    A, B = dev(seg.A), dev(seg.B)
    got = outputs(rsi.BVH(dev(mesh.V), dev(mesh.T), height_axis=3), A, B)
    base = outputs(rsi.BVH(dev(mesh.V), dev(mesh.T)), A, B)
    np.testing.assert_array_equal(got["bool"]["flag"], ref["flag"])
    np.testing.assert_array_equal(got["count"]["count"], ref["count"])
    np.testing.assert_array_equal(got["nearest"]["tri"], ref["tri"])
    assert_close(got["nearest"]["tuv"], ref["tuv"], what="tuv")
    assert_close(got["nearest"]["point"], ref["point"], what="point")
    for m in got:
        for k in got[m]:
            np.testing.assert_array_equal(got[m][k], base[m][k], err_msg=f"{m} {k}")


def test_differentiable_workload_same_outputs():
    # near-vertical segments over a 131,072-triangle terrain: the workload the
    # option is for; outputs bit-identical to the paper-code tree's
    mesh, seg, _ = synth.workload_diff(seed=9, n_seg=50_000)
    A, B = dev(seg.A), dev(seg.B)
    h = rsi.BVH(dev(mesh.V), dev(mesh.T), height_axis=3)
    b = rsi.BVH(dev(mesh.V), dev(mesh.T))
    got, base = outputs(h, A, B), outputs(b, A, B)
    for m in got:
        for k in got[m]:
            np.testing.assert_array_equal(got[m][k], base[m][k], err_msg=f"{m} {k}")
    # fewer node visits: no splits along the height
    sh = h.intersect(A, B, "nearest", stats=True)["stats"]
    sb = b.intersect(A, B, "nearest", stats=True)["stats"]
    assert sh["node_visits"] < 0.8 * sb["node_visits"]
    tree_check(h.export(), mesh.n_tri)


def test_batch_with_height_axis_matches_single_meshes():
    rng = np.random.default_rng(4)
    items, refs = [], []
    for G in (17, 40, 65):
        mesh = synth.heightfield(G, rng)
        seg = synth.segments_box(rng, 3000, [0, 0, -1], [1, 1, -0.8], [0, 0, 0.8], [1, 1, 1])
        V, T, A, B = dev(mesh.V), dev(mesh.T), dev(seg.A), dev(seg.B)
        items.append((V, T, A, B, "nearest"))
        refs.append(rsi.BVH(V, T).intersect(A, B, "nearest"))
    batch = rsi.Batch(items, height_axis=3)
    batch.build()
    outs = batch.intersect()
    torch.cuda.synchronize()
    for o, r in zip(outs, refs):
        for k in ("tri", "tuv", "point", "dist"):
            assert torch.equal(o[k], r[k]), k


def test_bad_height_axis_is_refused(small):
    mesh, _, _ = small
    with pytest.raises(Exception):
        rsi.BVH(dev(mesh.V), dev(mesh.T), height_axis=4)


def test_autotuner_picks_the_height_axis():
    from paper_2209_02878_gb300 import tuning
    mesh, seg, _ = synth.workload_diff(seed=12, n_seg=100_000)
    V, T, A, B = dev(mesh.V), dev(mesh.T), dev(seg.A), dev(seg.B)
    bvh = rsi.BVH(V, T)
    base = bvh.intersect(A, B, "nearest")
    best, ms = tuning.autotune_height_axis(bvh, V, T, A, B, "nearest", reps=5)
    assert best == 3, ms  # a terrain z = f(x, y): leaving z out is clearly fastest
    assert ms[3] < 0.8 * ms[0], ms
    assert bvh.height_axis == 3
    got = bvh.intersect(A, B, "nearest")  # the handle stays built with axis 3
    torch.cuda.synchronize()
    for k in ("tri", "tuv", "point", "dist"):
        assert torch.equal(got[k], base[k]), k
    g = bvh.export()
    r = oracle.lbvh(mesh.V, mesh.T, height_axis=3)
    np.testing.assert_array_equal(g["left"], r["left"])


def test_batch_per_item_height_axis():
    # terrains with the option, icospheres without, in one batch
    rng = np.random.default_rng(6)
    items, refs = [], []
    for k, G in enumerate((33, 50)):
        mesh = synth.heightfield(G, rng)
        seg = synth.segments_random_direction(rng, 4000, mesh.V)
        V, T, A, B = dev(mesh.V), dev(mesh.T), dev(seg.A), dev(seg.B)
        items.append((V, T, A, B, "count", 3))
        refs.append(rsi.BVH(V, T).intersect(A, B, "count")["count"])
        sph = synth.icosphere(3 + k, rng)
        sseg = synth.segments_box(rng, 4000, [-1.5] * 3, [1.5] * 3, [-1.5] * 3, [1.5] * 3)
        V, T, A, B = dev(sph.V), dev(sph.T), dev(sseg.A), dev(sseg.B)
        items.append((V, T, A, B, "count"))
        refs.append(rsi.BVH(V, T).intersect(A, B, "count")["count"])
    batch = rsi.Batch(items)
    outs = batch.run_graph()
    torch.cuda.synchronize()
    assert batch.status() == 0
    for o, r in zip(outs, refs):
        assert torch.equal(o["count"], r)
    with pytest.raises(Exception):
        rsi.Batch([items[0][:5] + (5,)])


@pytest.mark.parametrize("nT", [1, 2, 3, 17, 600])
@pytest.mark.parametrize("axis", [1, 3])
def test_height_axis_small_meshes(nT, axis):
    rng = np.random.default_rng(nT + 10 * axis)
    mesh, seg = synth.random_soup(rng, nT, 2000)
    ref = oracle.brute(mesh.V, mesh.T, seg.A, seg.B)
    bvh = rsi.BVH(dev(mesh.V), dev(mesh.T), height_axis=axis, leaf_size=2)
    got = outputs(bvh, dev(seg.A), dev(seg.B))
    np.testing.assert_array_equal(got["count"]["count"], ref["count"])
    np.testing.assert_array_equal(got["nearest"]["tri"], ref["tri"])
    tree_check(bvh.export(), nT, leaf_size=2)
    if nT > 1:
        r = oracle.lbvh(mesh.V, mesh.T, height_axis=axis)
        g = bvh.export()
        for k in ("left", "right", "range", "nbox", "lbox"):
            np.testing.assert_array_equal(g[k], r[k], err_msg=k)


def test_single_item_batch_with_height_axis():
    rng = np.random.default_rng(21)
    mesh = synth.heightfield(30, rng)
    seg = synth.segments_random_direction(rng, 5000, mesh.V)
    V, T, A, B = dev(mesh.V), dev(mesh.T), dev(seg.A), dev(seg.B)
    ref = rsi.BVH(V, T).intersect(A, B, "nearest")
    for item, batch_axis in (((V, T, A, B, "nearest", 3), 0), ((V, T, A, B, "nearest"), 3)):
        b = rsi.Batch([item], height_axis=batch_axis)
        out = b.run_graph()[0]
        torch.cuda.synchronize()
        for k in ("tri", "tuv", "point", "dist"):
            assert torch.equal(out[k], ref[k]), k
        b.close()
