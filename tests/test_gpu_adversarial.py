"""GPU parity on adversarial crossings (Sec. 2 definition, nearest mode of
Sec. 2.4, and the adjoint of the nearest outputs): small meshes of four
triangles sharing a frame (scales and offsets over 24 binades), each with
128 segments aimed within 1e-9 .. 1e-3 of an edge, a vertex or a segment
end, or nearly parallel to the plane (grazing crossings).  Every segment
goes through rsi_intersect in the BOOL, COUNT and NEAREST modes (one mesh
per call, the handle rebuilt per mesh) and every crossing through
rsi_intersect_backward; each result is compared element by element with the
FP64 oracle: flags, counts and triangle ids bit-exactly (near-degenerate
segments included, and counted), (t, u, v), points and distances within
|x - x_ref| <= 1e-5 max(1, |x_ref|), gradients within
|g - g_ref| <= 1e-5 max(|g_ref|, 1e-3 max |g_ref|) per segment (endpoint
gradients) and per triangle (vertex gradients of one crossing each), plus
the relative L2 rule per tensor."""
import numpy as np
import pytest
import torch

import oracle
import paper_2209_02878_gb300 as rsi
from _adversarial import adversarial_groups
from _util import close

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
N_GROUPS, K, M = 2000, 4, 128


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


@pytest.fixture(scope="module")
def adv():
    rng = np.random.default_rng(31)
    V, A, B, _ = adversarial_groups(rng, N_GROUPS, K, M)
    T = np.arange(3 * K, dtype=np.int32).reshape(K, 3)
    parts = [oracle.brute(V[g], T, A[g], B[g]) for g in range(N_GROUPS)]
    ref = {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}
    return V, T, A, B, ref


def run_groups(V, T, A, B, modes, launch=None, groups=None):
    """Each group as its own mesh through rsi_intersect (one handle, rebuilt
    per group, every call queued on one stream); outputs land in slices of
    full-size tensors.  Returns host arrays and the summed traversal
    counters when launch asks for stats."""
    groups = range(N_GROUPS) if groups is None else groups
    n = M * len(groups)
    Vd, Td = dev(V.reshape(-1, 3)), dev(T)
    Ad, Bd = dev(A.reshape(-1, 3)), dev(B.reshape(-1, 3))
    out = {}
    for m in modes:
        if m == "bool":
            out[m] = {"flag": torch.empty(n, dtype=torch.uint8, device=DEV)}
        elif m == "count":
            out[m] = {"count": torch.empty(n, dtype=torch.int32, device=DEV)}
        else:
            out[m] = {"tri": torch.empty(n, dtype=torch.int32, device=DEV),
                      "tuv": torch.empty((n, 3), dtype=torch.float32, device=DEV),
                      "point": torch.empty((n, 3), dtype=torch.float32, device=DEV),
                      "dist": torch.empty(n, dtype=torch.float32, device=DEV)}
    bvh = rsi.BVH(Vd[:3 * K], Td)
    stats = None
    for q, g in enumerate(groups):
        bvh.build(Vd[3 * K * g:3 * K * (g + 1)], Td)
        a, b = Ad[M * g:M * (g + 1)], Bd[M * g:M * (g + 1)]
        for m in modes:
            o = {k: v[M * q:M * (q + 1)] for k, v in out[m].items()}
            r = bvh.intersect(a, b, m, out=o, launch=launch, stats=bool(launch and
                                                                         launch.get("stats")))
            if "stats" in r:
                stats = r["stats"] if stats is None else {k: stats[k] + r["stats"][k]
                                                          for k in stats}
    assert bvh.status() == 0
    torch.cuda.synchronize()
    return {m: {k: v.cpu().numpy() for k, v in d.items()} for m, d in out.items()}, stats


def sel_ref(ref, groups):
    idx = np.concatenate([np.arange(M * g, M * (g + 1)) for g in groups])
    return {k: v[idx] for k, v in ref.items()}


def check_nearest(got, ref, what):
    nd = int(ref["neardeg"].sum())
    hit = ref["tri"] >= 0
    np.testing.assert_array_equal(got["tri"], ref["tri"],
                                  err_msg=f"{what}: tri ({nd} near-degenerate segments)")
    for k in ("tuv", "point", "dist"):
        bad = close(got[k], ref[k])
        if bad.ndim == 2:
            bad = bad.any(axis=1)
        assert not (hit & bad).any(), \
            f"{what}: {k} outside 1e-5 on {int((hit & bad).sum())} of {int(hit.sum())} hits " \
            f"({nd} near-degenerate segments); first {np.argmax(hit & bad)}"


def test_adversarial_all_modes(adv):
    V, T, A, B, ref = adv
    got, _ = run_groups(V, T, A, B, ("bool", "count", "nearest"))
    hits = int((ref["tri"] >= 0).sum())
    nd = int(ref["neardeg"].sum())
    assert hits >= 100_000, hits
    assert nd > 10_000, nd            # the inputs do reach the near-degenerate band
    np.testing.assert_array_equal(got["bool"]["flag"], ref["flag"], err_msg="flag")
    np.testing.assert_array_equal(got["count"]["count"], ref["count"], err_msg="count")
    check_nearest(got["nearest"], ref, "nearest")


def test_adversarial_takes_the_fp64_value_path(adv):
    """The counters of the same calls: grazing crossings and long segments
    do go to the FP64 recomputation of the outputs."""
    V, T, A, B, ref = adv
    groups = range(0, N_GROUPS, 4)
    got, st = run_groups(V, T, A, B, ("nearest",), launch={"stats": 1}, groups=groups)
    check_nearest(got["nearest"], sel_ref(ref, groups), "nearest (stats)")
    assert st["fp64_values"] > 100 and st["df_refines"] > 100, st


@pytest.mark.parametrize("launch", [{"packet": 1}, {"node_width": 4, "stack_depth": 8},
                                    {"sort_bits": 24}, {"block_size": 32}])
def test_adversarial_launch_variants(adv, launch):
    V, T, A, B, ref = adv
    groups = range(1, N_GROUPS, 5)
    got, _ = run_groups(V, T, A, B, ("count", "nearest"), launch=launch, groups=groups)
    r = sel_ref(ref, groups)
    np.testing.assert_array_equal(got["count"]["count"], r["count"], err_msg=f"{launch} count")
    check_nearest(got["nearest"], r, str(launch))


def test_adversarial_batched(adv):
    """The same meshes as items of one batch (one multi-mesh build, one
    persistent traversal launch)."""
    V, T, A, B, ref = adv
    groups = list(range(2, N_GROUPS, 4))
    Td = dev(T)
    items = [(dev(V[g]), Td, dev(A[g]), dev(B[g]), "nearest") for g in groups]
    b = rsi.Batch(items)
    outs = b.build().intersect()
    assert b.status() == 0
    got = {k: np.concatenate([o[k].cpu().numpy() for o in outs])
           for k in ("tri", "tuv", "point", "dist")}
    b.close()
    check_nearest(got, sel_ref(ref, groups), "batched")


def test_adversarial_backward(adv):
    V, T, A, B, ref = adv
    rng = np.random.default_rng(32)
    n = N_GROUPS * M
    Vs = V.reshape(-1, 3)
    Ts = (T[None, :, :] + 3 * K * np.arange(N_GROUPS)[:, None, None]).reshape(-1, 3)
    Ts = Ts.astype(np.int32)
    group = np.repeat(np.arange(N_GROUPS), M)
    tri = np.where(ref["tri"] >= 0, ref["tri"] + K * group, -1).astype(np.int32)
    As, Bs = A.reshape(-1, 3), B.reshape(-1, 3)
    gP = rng.normal(size=(n, 3)).astype(np.float32)
    gt = rng.normal(size=(n, 3)).astype(np.float32)
    hit = tri >= 0

    def both(tri_sel):
        gV, gA, gB = rsi.intersect_backward(dev(Vs), dev(Ts), dev(As), dev(Bs), dev(tri_sel),
                                            grad_point=dev(gP), grad_tuv=dev(gt))
        torch.cuda.synchronize()
        r = oracle.backward(Vs, Ts, As, Bs, tri_sel, gP=gP.astype(np.float64),
                            gtuv=gt.astype(np.float64))
        return [x.cpu().numpy().astype(np.float64) for x in (gV, gA, gB)], r

    (gV, gA, gB), (rV, rA, rB) = both(tri)
    # endpoint gradients, per segment
    got = np.concatenate([gA, gB], axis=1)[hit]
    want = np.concatenate([rA, rB], axis=1)[hit]
    scale = np.maximum(np.abs(want), 1e-3 * np.abs(want).max(axis=1, keepdims=True))
    err = np.abs(got - want) / scale
    assert err.max() <= 1e-5, f"endpoint gradients: {int((err > 1e-5).any(1).sum())} segments"
    assert np.all(gA[~hit] == 0) and np.all(gB[~hit] == 0)
    for g, r, name in ((gV, rV, "gV"), (gA, rA, "gA"), (gB, rB, "gB")):
        rel = np.linalg.norm(g - r) / max(np.linalg.norm(r), 1e-300)
        assert rel <= 1e-5, (name, rel)
    # vertex gradients of every mesh, with that mesh's floor
    gVg, rVg = gV.reshape(N_GROUPS, -1), rV.reshape(N_GROUPS, -1)
    scale = np.maximum(np.abs(rVg), 1e-3 * np.abs(rVg).max(axis=1, keepdims=True))
    ok = (np.abs(gVg - rVg) <= 1e-5 * scale) | (rVg == 0) & (gVg == 0)
    assert ok.all(), f"vertex gradients: {int((~ok).any(1).sum())} meshes"
    # one crossing per triangle: each vertex gradient is a single
    # contribution, checked per triangle
    first = np.full(Ts.shape[0], -1)
    seg = np.nonzero(hit)[0]
    first[tri[seg[::-1]]] = seg[::-1]
    one = np.full(n, -1, np.int32)
    used = first[first >= 0]
    one[used] = tri[used]
    (gV1, _, _), (rV1, _, _) = both(one)
    t_ids = np.unique(one[one >= 0])
    got = gV1[Ts[t_ids]].reshape(len(t_ids), 9)
    want = rV1[Ts[t_ids]].reshape(len(t_ids), 9)
    scale = np.maximum(np.abs(want), 1e-3 * np.abs(want).max(axis=1, keepdims=True))
    err = np.abs(got - want) / scale
    assert len(t_ids) > 4_000
    assert err.max() <= 1e-5, f"single-crossing vertex gradients: {int((err > 1e-5).any(1).sum())}"
