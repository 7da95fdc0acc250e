"""GPU parity on the hand-derived cases of tests/golden/: the CUDA path
(through the C ABI binding), one small mesh per case.  Flags, counts and
nearest triangles must match exactly; (t, u, v), points, distances and
gradients within relative 1e-5 (the parity tolerance of the FP32 outputs)."""
import numpy as np
import pytest
import torch

import paper_2209_02878_gb300 as rsi

from _golden import load_backward_cases, load_inside_case, load_lbvh_case, load_mt_cases
from _util import assert_close

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


@pytest.mark.parametrize("case", load_mt_cases(), ids=lambda c: c["name"])
def test_golden_hand_cases(case):
    bvh = rsi.BVH(dev(case["V"]), dev(case["T"]))
    A, B = dev(case["A"]), dev(case["B"])
    o = {m: bvh.intersect(A, B, m) for m in ("bool", "count", "nearest")}
    torch.cuda.synchronize()
    got = (int(o["bool"]["flag"][0]), int(o["count"]["count"][0]), int(o["nearest"]["tri"][0]))
    assert got == (case["flag"], case["count"], case["tri"]), case["name"]
    if "tuv" in case:
        n = o["nearest"]
        assert_close(n["tuv"].cpu().numpy()[0], case["tuv"], what=case["name"] + " tuv")
        assert_close(n["point"].cpu().numpy()[0], case["point"], what=case["name"] + " point")
        assert_close(n["dist"].cpu().numpy()[:1], [case["dist"]], what=case["name"] + " dist")
    assert bvh.status() == 0
    bvh.close()


@pytest.mark.parametrize("case", load_backward_cases(), ids=lambda c: c["name"])
def test_golden_backward_cases(case):
    V, T, A, B = dev(case["V"]), dev(case["T"]), dev(case["A"]), dev(case["B"])
    tri = torch.zeros(1, dtype=torch.int32, device=DEV)
    gP = dev(case["gP"].astype(np.float32))
    gtuv = dev(case["gtuv"].astype(np.float32))
    gV, gA, gB = rsi.intersect_backward(V, T, A, B, tri, grad_point=gP, grad_tuv=gtuv)
    torch.cuda.synchronize()
    assert_close(gA.cpu().numpy(), case["gA"], what=case["name"] + " gA")
    assert_close(gB.cpu().numpy(), case["gB"], what=case["name"] + " gB")
    assert_close(gV.cpu().numpy(), case["gV"], what=case["name"] + " gV")


def test_golden_lbvh_build():
    """The hand-worked build of tests/golden/lbvh_hand_case.txt on the
    device: bounds, codes (exported in sorted order), order, children,
    ranges and internal boxes exactly."""
    c = load_lbvh_case()
    bvh = rsi.BVH(dev(c["V"]), dev(c["T"]))
    g = bvh.export()
    assert list(g["bounds"]) == c["bounds"]
    assert list(g["order"]) == c["order"]
    assert list(g["codes"]) == [c["codes"][i] for i in c["order"]]
    assert list(g["left"]) == c["left"]
    assert list(g["right"]) == c["right"]
    assert g["range"].tolist() == c["range"]
    for k in (0, 3, 4):
        assert g["nbox"][k].tolist() == c[f"nbox{k}"]
    bvh.close()


def test_golden_cube_inside():
    """rsi_points_inside on the closed cube of tests/golden/cube_inside_cases.txt."""
    c = load_inside_case()
    bvh = rsi.BVH(dev(c["V"]), dev(c["T"]))
    got = bvh.points_inside(dev(c["P"]))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(got.cpu().numpy(), c["inside"])
    bvh.close()
