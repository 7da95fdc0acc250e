"""Warp-cooperative (packet) traversal, launch option `packet`: the same
results as the oracle (and so as the per-segment traversal) in every mode,
with and without the coherent segment order, a treelet root, larger leaves,
compaction, ragged segment counts and an empty mesh."""
import numpy as np
import pytest
import torch

import oracle
import paper_2209_02878_gb300 as rsi
from paper_2209_02878_gb300 import RSIError, synth

from _util import assert_close

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def run_modes(bvh, A, B, launch, compact=False):
    o = {m: bvh.intersect(A, B, m, launch=launch, compact=compact)
         for m in ("bool", "count", "nearest")}
    torch.cuda.synchronize()
    return {m: {k: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for k, v in d.items()}
            for m, d in o.items()}


def check(got, ref, what):
    np.testing.assert_array_equal(got["bool"]["flag"], ref["flag"], err_msg=what + " flag")
    np.testing.assert_array_equal(got["count"]["count"], ref["count"], err_msg=what + " count")
    np.testing.assert_array_equal(got["nearest"]["tri"], ref["tri"], err_msg=what + " tri")
    assert_close(got["nearest"]["tuv"], ref["tuv"], what=what + " tuv")
    assert_close(got["nearest"]["point"], ref["point"], what=what + " point")
    assert_close(got["nearest"]["dist"], ref["dist"], what=what + " dist")


@pytest.fixture(scope="module")
def small():
    mesh, seg = synth.workload_small_bool()
    return mesh, seg, oracle.brute(mesh.V, mesh.T, seg.A, seg.B)


@pytest.mark.parametrize("sort_bits,top_levels,leaf", [(0, 0, 1), (12, 0, 1), (0, 6, 1),
                                                       (24, 0, 4)])
def test_packet_matches_oracle(small, sort_bits, top_levels, leaf):
    mesh, seg, ref = small
    bvh = rsi.BVH(dev(mesh.V), dev(mesh.T), leaf_size=leaf, top_levels=top_levels)
    got = run_modes(bvh, dev(seg.A), dev(seg.B), dict(packet=1, sort_bits=sort_bits))
    check(got, ref, f"packet sort={sort_bits} levels={top_levels} leaf={leaf}")
    assert bvh.status() == 0


def test_packet_closed_sphere_counts_and_ragged_sizes():
    """Crossing counts of 0, 1, 2 and more on a closed icosphere, segment
    counts that end inside a warp."""
    rng = np.random.default_rng(31)
    mesh = synth.icosphere(4, rng)
    seg = synth.segments_box(rng, 20000, [-1.5] * 3, [1.5] * 3, [-1.5] * 3, [1.5] * 3)
    ref = oracle.brute(mesh.V, mesh.T, seg.A, seg.B)
    assert (ref["count"] >= 2).any()
    bvh = rsi.BVH(dev(mesh.V), dev(mesh.T))
    for n in (1, 31, 33, 1007, 20000):
        got = run_modes(bvh, dev(seg.A[:n]), dev(seg.B[:n]), dict(packet=1, sort_bits=18))
        check(got, {k: v[:n] for k, v in ref.items()}, f"sphere n={n}")


def test_packet_compaction_and_stats(small):
    mesh, seg, ref = small
    bvh = rsi.BVH(dev(mesh.V), dev(mesh.T))
    A, B = dev(seg.A), dev(seg.B)
    got = run_modes(bvh, A, B, dict(packet=1), compact=True)
    for m in ("count", "nearest"):
        n = int(got[m]["n_hits"][0])
        assert n == int((ref["count"] > 0).sum())
        idx = got[m]["hit_idx"][:n]
        assert np.array_equal(np.sort(idx), np.nonzero(ref["count"] > 0)[0])
    np.testing.assert_array_equal(got["nearest"]["hit_tri"][:n], ref["tri"][idx])
    # a warp visits the union of its lanes' paths: at least each lane's own
    per_lane = bvh.intersect(A, B, "count", stats=True)["stats"]
    packet = bvh.intersect(A, B, "count", stats=True, launch=dict(packet=1))["stats"]
    assert packet["segments"] == per_lane["segments"] == seg.n
    assert packet["tri_tests"] >= per_lane["tri_tests"]
    assert packet["node_visits"] >= per_lane["node_visits"]


def test_packet_empty_mesh_and_bad_options(small):
    mesh, seg, _ = small
    V = dev(mesh.V)
    T = torch.zeros((0, 3), dtype=torch.int32, device=DEV)
    bvh = rsi.BVH(V, T)
    o = run_modes(bvh, dev(seg.A), dev(seg.B), dict(packet=1))
    assert not o["bool"]["flag"].any() and not o["count"]["count"].any()
    assert (o["nearest"]["tri"] == -1).all()
    bvh = rsi.BVH(V, dev(mesh.T), top_levels=6)
    for bad in (dict(packet=2), dict(packet=1, node_width=4), dict(packet=1, smem_nodes=64)):
        with pytest.raises(RSIError):
            bvh.intersect(dev(seg.A), dev(seg.B), "bool", launch=bad)
