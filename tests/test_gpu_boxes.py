"""The box pass of the device build (bottom-up boxes of Sec. 3.1, computed
per block of sorted leaves plus a pass over the nodes that cross block
boundaries) against the oracle's LBVH, exactly: meshes whose trees have
nodes spanning many blocks (more than a warp's worth, so the block unions
take several rounds), leaf sizes above 1, sizes at the block edges, and a
refit after the vertices move (leaf boxes of the moved triangles, every
node the union over its leaf range)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2209_02878_gb300 as rsi
from paper_2209_02878_gb300 import synth

from _util import tree_check

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def same_tree(g, r, what=""):
    for k in ("left", "right", "range", "nbox", "lbox"):
        np.testing.assert_array_equal(g[k], r[k], err_msg=f"{what} {k}")


@pytest.mark.parametrize("level", [5, 6])
def test_icosphere_boxes_many_blocks(level):
    # 20,480 / 81,920 triangles: 40 / 160 blocks of 512 sorted leaves
    rng = np.random.default_rng(level)
    mesh = synth.icosphere(level, rng)
    r = oracle.lbvh(mesh.V, mesh.T)
    for leaf in (1, 3):
        bvh = rsi.BVH(dev(mesh.V), dev(mesh.T), leaf_size=leaf)
        g = bvh.export()
        same_tree(g, r, f"L{level} leaf {leaf}")
        tree_check(g, mesh.n_tri, leaf_size=leaf)
        assert bvh.status() == 0


@pytest.mark.parametrize("n", [511, 512, 513, 1024, 1537])
def test_block_edge_sizes(n):
    rng = np.random.default_rng(n)
    mesh, _ = synth.random_soup(rng, n, 1)
    r = oracle.lbvh(mesh.V, mesh.T)
    bvh = rsi.BVH(dev(mesh.V), dev(mesh.T))
    g = bvh.export()
    same_tree(g, r, f"n={n}")
    tree_check(g, n)


def test_refit_equals_fresh_build():
    mesh, seg, _ = synth.workload_diff(seed=5, n_seg=1000, G=129)  # 32,768 triangles
    V = dev(mesh.V)
    T = dev(mesh.T)
    bvh = rsi.BVH(V, T)
    rng = np.random.default_rng(1)
    moved = (mesh.V + rng.normal(0, 1e-3, mesh.V.shape)).astype(np.float32)
    Vm = dev(moved)
    bvh.refit(Vm)
    g = bvh.export()
    r = oracle.lbvh(mesh.V, mesh.T)  # topology of the original build
    for k in ("left", "right", "range"):
        np.testing.assert_array_equal(g[k], r[k], err_msg=k)
    # boxes of the moved vertices over the same topology: the leaf boxes from
    # the moved triangles, every node the union of its leaf range
    P = moved[mesh.T.reshape(-1)].reshape(-1, 3, 3).astype(np.float32)
    tb = np.concatenate([P.min(1), P.max(1)], 1)[r["order"]]
    np.testing.assert_array_equal(g["lbox"], tb)
    rg = r["range"]
    want = np.stack([np.r_[tb[a:b + 1, :3].min(0), tb[a:b + 1, 3:].max(0)] for a, b in rg])
    np.testing.assert_array_equal(g["nbox"], want)
    tree_check(g, mesh.n_tri)
