"""A processing order computed once (rsi_segment_order, the paper's
Morton-sorted rays of Sec. 4.1) and passed to later traversals through
rsi_launch_opts.order: outputs identical to the input-order traversal in
every mode, checked against the oracle on a sample; entries outside
[0, nR) are skipped and reported; the calls that cannot take an order
refuse it."""
import numpy as np
import pytest
import torch

import oracle
import paper_2209_02878_gb300 as rsi
from paper_2209_02878_gb300 import synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
RSI_ERR_BAD_INDEX = 4


def t(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


@pytest.fixture(scope="module")
def diff_case():
    # the differentiable workload's heightfield and segment shapes, fewer segments
    mesh, seg, _ = synth.workload_diff(seed=11, n_seg=40_000, G=129)
    V, T = t(mesh.V), t(mesh.T)
    return mesh, seg, V, T, t(seg.A), t(seg.B)


def _same(a, b):
    for k in a:
        if k == "stats":
            continue
        assert torch.equal(a[k], b[k]), k


def test_order_is_a_permutation(diff_case):
    _, seg, V, T, A, B = diff_case
    bvh = rsi.BVH(V, T)
    for bits in (0, 12, 30):
        order = bvh.segment_order(A, B, bits=bits)
        torch.cuda.synchronize()
        assert order.dtype == torch.int32 and order.shape == (seg.n,)
        assert torch.equal(torch.sort(order.long())[0], torch.arange(seg.n, device=DEV))
    with pytest.raises(Exception):
        bvh.segment_order(A, B, bits=5)


@pytest.mark.parametrize("mode", ["bool", "count", "nearest"])
@pytest.mark.parametrize("packet", [0, 1])
def test_ordered_outputs_match_input_order(diff_case, mode, packet):
    _, _, V, T, A, B = diff_case
    bvh = rsi.BVH(V, T)
    order = bvh.segment_order(A, B)
    ref = bvh.intersect(A, B, mode)
    got = bvh.intersect(A, B, mode, launch={"order": order, "packet": packet})
    torch.cuda.synchronize()
    _same(ref, got)
    assert bvh.status() == 0


def test_ordered_nearest_against_oracle(diff_case):
    mesh, seg, V, T, A, B = diff_case
    bvh = rsi.BVH(V, T)
    order = bvh.segment_order(A, B)
    got = bvh.intersect(A, B, "nearest", launch={"order": order})
    rng = np.random.default_rng(5)
    idx = np.sort(rng.choice(seg.n, 3000, replace=False))
    ref = oracle.intersect(mesh.V, mesh.T, seg.A[idx], seg.B[idx])
    tri = got["tri"].cpu().numpy()[idx]
    assert np.array_equal(tri, ref["tri"])
    hit = tri >= 0
    assert hit.mean() > 0.9
    for k in ("tuv", "point"):
        x = got[k].cpu().numpy()[idx][hit].astype(np.float64)
        r = ref[k][hit]
        assert np.all(np.abs(x - r) <= 1e-5 * np.maximum(1.0, np.abs(r))), k


def test_ordered_compaction(diff_case):
    _, _, V, T, A, B = diff_case
    bvh = rsi.BVH(V, T)
    order = bvh.segment_order(A, B)
    ref = bvh.intersect(A, B, "nearest", compact=True)
    got = bvh.intersect(A, B, "nearest", compact=True, launch={"order": order})
    torch.cuda.synchronize()
    n = int(ref["n_hits"].item())
    assert int(got["n_hits"].item()) == n
    ri, gi = ref["hit_idx"][:n].long(), got["hit_idx"][:n].long()
    rs, gs = torch.argsort(ri), torch.argsort(gi)
    assert torch.equal(ri[rs], gi[gs])
    assert torch.equal(ref["hit_tri"][:n][rs], got["hit_tri"][:n][gs])
    assert torch.equal(ref["hit_point"][:n][rs], got["hit_point"][:n][gs])


def test_order_entries_out_of_range_are_skipped(diff_case):
    _, seg, V, T, A, B = diff_case
    bvh = rsi.BVH(V, T)
    order = bvh.segment_order(A, B)
    ref = bvh.intersect(A, B, "count")
    torch.cuda.synchronize()
    bad = order.clone()
    lost = bad[:2].long().cpu().numpy()
    bad[0] = seg.n
    bad[1] = -1
    assert bvh.status() == 0
    got = bvh.intersect(A, B, "count", launch={"order": bad})
    torch.cuda.synchronize()
    assert bvh.status() == RSI_ERR_BAD_INDEX
    keep = torch.ones(seg.n, dtype=torch.bool, device=DEV)
    keep[torch.from_numpy(lost).to(DEV)] = False
    assert torch.equal(ref["count"][keep], got["count"][keep])
    # the handle stays usable
    again = bvh.intersect(A, B, "count", launch={"order": order})
    torch.cuda.synchronize()
    assert torch.equal(ref["count"], again["count"])


def test_calls_without_order_support_refuse_it(diff_case):
    _, _, V, T, A, B = diff_case
    bvh = rsi.BVH(V, T)
    order = bvh.segment_order(A, B)
    with pytest.raises(Exception):
        bvh.intersect_host(A.cpu(), B.cpu(), "bool", launch={"order": order})
    with pytest.raises(Exception):
        bvh.points_inside(A, launch={"order": order})
    with pytest.raises(ValueError):
        bvh.intersect(A, B, "bool", launch={"order": order[:-1]})


def test_nearest_hit_with_order_same_gradients(diff_case):
    _, seg, V, T, A, B = diff_case
    rng = np.random.default_rng(2)
    W = t(rng.normal(size=(seg.n, 3)).astype(np.float32))
    grads = []
    for use_order in (False, True):
        Vp = V.clone().requires_grad_(True)
        bvh = rsi.BVH(Vp.detach(), T)
        order = bvh.segment_order(A, B) if use_order else None
        P, _, tri = rsi.nearest_hit(Vp, T, A, B, bvh=bvh, order=order)
        (P * W).sum().backward()
        grads.append((P.detach(), tri, Vp.grad.clone()))
    torch.cuda.synchronize()
    assert torch.equal(grads[0][0], grads[1][0])
    assert torch.equal(grads[0][1], grads[1][1])
    # the adjoint sums the same per-segment terms in FP64 (atomics): equal to
    # rounding of the FP64 sums
    g0, g1 = grads[0][2], grads[1][2]
    assert torch.allclose(g0, g1, rtol=1e-6, atol=1e-9)


@pytest.mark.parametrize("nT,nR", [(0, 5), (1, 1), (2, 33), (17, 1000)])
def test_order_edge_sizes(nT, nR):
    rng = np.random.default_rng(nT * 7 + nR)
    if nT == 0:
        V = np.zeros((3, 3), np.float32)
        T = np.zeros((0, 3), np.int32)
        A = rng.uniform(0, 1, (nR, 3)).astype(np.float32)
        B = rng.uniform(0, 1, (nR, 3)).astype(np.float32)
    else:
        mesh, seg = synth.random_soup(rng, nT, nR)
        V, T, A, B = mesh.V, mesh.T, seg.A, seg.B
    bvh = rsi.BVH(t(V), t(T))
    order = bvh.segment_order(t(A), t(B))
    torch.cuda.synchronize()
    assert torch.equal(torch.sort(order.long())[0], torch.arange(nR, device=DEV))
    for mode in ("bool", "count", "nearest"):
        ref = bvh.intersect(t(A), t(B), mode)
        got = bvh.intersect(t(A), t(B), mode, launch={"order": order})
        torch.cuda.synchronize()
        _same(ref, got)
    assert bvh.status() == 0
