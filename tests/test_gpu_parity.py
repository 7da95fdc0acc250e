"""GPU parity: the CUDA path (through the C ABI binding) against the FP64 CPU
oracle, element by element on the same seeded inputs.

Flags, counts and triangle ids must match bit-exactly (the kernels recompute
every decision their FP32 error bound cannot settle in FP64 with the
definition's operation order); (t, u, v), points and distances within
relative 1e-5 of the oracle's FP64 values (|x - x_ref| <= 1e-5 max(1,|x_ref|)).
Near-degenerate segments are counted and must match too."""
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


def run_all_modes(bvh, A, B, launch=None, compact=False):
    o = {m: bvh.intersect(A, B, m, launch=launch, compact=compact) for m in ("bool", "count", "nearest")}
    torch.cuda.synchronize()
    return {m: {k: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for k, v in d.items()}
            for m, d in o.items()}


def compare(got, ref, idx=None, what=""):
    sel = slice(None) if idx is None else idx
    np.testing.assert_array_equal(got["bool"]["flag"], ref["flag"][sel], err_msg=what + " flag")
    np.testing.assert_array_equal(got["count"]["count"], ref["count"][sel], err_msg=what + " count")
    np.testing.assert_array_equal(got["nearest"]["tri"], ref["tri"][sel], err_msg=what + " tri")
    assert_close(got["nearest"]["tuv"], ref["tuv"][sel], what=what + " tuv")
    assert_close(got["nearest"]["point"], ref["point"][sel], what=what + " point")
    assert_close(got["nearest"]["dist"], ref["dist"][sel], what=what + " dist")


# ------------------------------------------------------------ small, full
@pytest.fixture(scope="module")
def small():
    mesh, seg = synth.workload_small_bool()
    ref = oracle.brute(mesh.V, mesh.T, seg.A, seg.B)
    return mesh, seg, ref


def test_small_heightfield_all_modes(small):
    mesh, seg, ref = small
    bvh = rsi.BVH(dev(mesh.V), dev(mesh.T))
    got = run_all_modes(bvh, dev(seg.A), dev(seg.B))
    compare(got, ref, what="1922 tris x 10k")
    assert bvh.status() == 0
    assert ref["flag"].mean() > 0.3  # the workload does cross the surface


@pytest.mark.parametrize("leaf,levels", [(1, 0), (1, -1), (1, 10), (2, 4), (4, 10), (8, 12)])
def test_small_build_options(small, leaf, levels):
    mesh, seg, ref = small
    bvh = rsi.BVH(dev(mesh.V), dev(mesh.T), leaf_size=leaf, top_levels=levels)
    compare(run_all_modes(bvh, dev(seg.A), dev(seg.B)), ref, what=f"leaf {leaf} levels {levels}")
    tree_check(bvh.export(), mesh.n_tri, leaf_size=leaf)


@pytest.mark.parametrize("launch", [
    dict(block_size=32), dict(block_size=128, smem_nodes=-1), dict(block_size=512),
    dict(block_size=1024, smem_nodes=2047), dict(stack_depth=8), dict(stack_depth=32),
    dict(smem_nodes=1), dict(sort_bits=24), dict(sort_bits=6), dict(sort_bits=30),
    dict(sort_bits=-1), dict(sort_bits=15, stack_depth=8, block_size=64),
    dict(node_width=2), dict(node_width=4, stack_depth=8), dict(node_width=2, sort_bits=21)])
def test_small_launch_options(small, launch):
    mesh, seg, ref = small
    # shared-memory staging needs the breadth-first treelet
    levels = 11 if launch.get("smem_nodes", 0) > 0 else 0
    bvh = rsi.BVH(dev(mesh.V), dev(mesh.T), top_levels=levels)
    compare(run_all_modes(bvh, dev(seg.A), dev(seg.B), launch=launch), ref, what=str(launch))


def test_build_steps_match_definition(small):
    mesh, _, _ = small
    bvh = rsi.BVH(dev(mesh.V), dev(mesh.T))
    g = bvh.export()
    r = oracle.lbvh(mesh.V, mesh.T)
    np.testing.assert_array_equal(g["bounds"], r["bounds"])
    np.testing.assert_array_equal(g["order"], r["order"].astype(np.int32))
    np.testing.assert_array_equal(g["codes"], r["codes"][r["order"]])
    np.testing.assert_array_equal(g["left"], r["left"])
    np.testing.assert_array_equal(g["right"], r["right"])
    np.testing.assert_array_equal(g["range"], r["range"])
    np.testing.assert_array_equal(g["nbox"], r["nbox"])
    np.testing.assert_array_equal(g["lbox"], r["lbox"])
    tree_check(g, mesh.n_tri)


@pytest.mark.parametrize("seed", range(3))
def test_build_steps_duplicate_codes(seed):
    # clustered centroids force equal Morton codes (index tie-break)
    rng = np.random.default_rng(seed)
    n = 5000
    base = rng.uniform(0, 1, size=(50, 3))
    cen = base[rng.integers(0, 50, n)] + rng.normal(0, 1e-6, size=(n, 3))
    V = (cen[:, None, :] + rng.normal(0, 1e-3, size=(n, 3, 3))).reshape(-1, 3).astype(np.float32)
    T = np.arange(3 * n, dtype=np.int32).reshape(n, 3)
    bvh = rsi.BVH(dev(V), dev(T))
    g = bvh.export()
    r = oracle.lbvh(V, T)
    assert len(np.unique(r["codes"])) < n  # duplicates present
    for k in ("left", "right", "range", "nbox", "lbox"):
        np.testing.assert_array_equal(g[k], r[k], err_msg=k)
    np.testing.assert_array_equal(g["order"], r["order"].astype(np.int32))
    tree_check(g, n)
    A = rng.uniform(-0.1, 1.1, size=(20000, 3)).astype(np.float32)
    B = (A + rng.normal(0, 0.2, size=A.shape)).astype(np.float32)
    compare(run_all_modes(bvh, dev(A), dev(B)), oracle.brute(V, T, A, B), what="clustered")


def test_icosphere_build_and_counts():
    rng = np.random.default_rng(7)
    mesh = synth.icosphere(4, rng)
    seg = synth.segments_box(rng, 20000, [-1.5] * 3, [1.5] * 3, [-1.5] * 3, [1.5] * 3)
    bvh = rsi.BVH(dev(mesh.V), dev(mesh.T))
    g = bvh.export()
    r = oracle.lbvh(mesh.V, mesh.T)
    for k in ("left", "right", "range", "nbox", "lbox"):
        np.testing.assert_array_equal(g[k], r[k], err_msg=k)
    ref = oracle.brute(mesh.V, mesh.T, seg.A, seg.B)
    compare(run_all_modes(bvh, dev(seg.A), dev(seg.B)), ref, what="icosphere L4")
    assert ref["count"].max() >= 2


# ------------------------------------------------------------ edge cases
@pytest.mark.parametrize("nR", [1, 31, 32, 33, 1007])
@pytest.mark.parametrize("nT", [1, 2, 3, 17])
def test_ragged_sizes(nR, nT):
    rng = np.random.default_rng(nR * 100 + nT)
    mesh, seg = synth.random_soup(rng, nT, nR)
    ref = oracle.brute(mesh.V, mesh.T, seg.A, seg.B)
    for leaf in (1, 4):
        bvh = rsi.BVH(dev(mesh.V), dev(mesh.T), leaf_size=leaf)
        compare(run_all_modes(bvh, dev(seg.A), dev(seg.B)), ref, what=f"nT={nT} nR={nR}")
        tree_check(bvh.export(), nT, leaf_size=leaf)


def test_empty_inputs():
    V = dev(np.zeros((3, 3), np.float32))
    T = dev(np.zeros((0, 3), np.int32))
    A = dev(np.zeros((5, 3), np.float32))
    B = dev(np.ones((5, 3), np.float32))
    bvh = rsi.BVH(V, T)
    got = run_all_modes(bvh, A, B, compact=True)
    assert not got["bool"]["flag"].any() and not got["count"]["count"].any()
    assert np.all(got["nearest"]["tri"] == -1)
    assert got["nearest"]["n_hits"][0] == 0
    mesh, _ = synth.workload_small_bool()
    bvh = rsi.BVH(dev(mesh.V), dev(mesh.T))
    e = dev(np.zeros((0, 3), np.float32))
    got = run_all_modes(bvh, e, e)
    assert got["bool"]["flag"].size == 0


def test_degenerate_and_special_segments():
    mesh, seg = synth.workload_small_bool(n_seg=2000)
    V = mesh.V.copy()
    T = mesh.T.copy()
    # degenerate triangles: collapse some (zero edge) and flatten others (collinear)
    T[5] = [T[5][0], T[5][0], T[5][1]]
    T[9] = [0, 1, 2]
    V_extra = np.array([[0.5, 0.5, 0.0], [0.6, 0.5, 0.0], [0.7, 0.5, 0.0]], np.float32)
    T = np.concatenate([T, np.array([[len(V), len(V) + 1, len(V) + 2]], np.int32)])
    V = np.concatenate([V, V_extra])
    # duplicate triangle (tie on t: lower index wins)
    T = np.concatenate([T, T[100:101]])
    A, B = seg.A.copy(), seg.B.copy()
    A[0] = [np.nan, 0.5, -1]
    B[1] = [np.inf, 0.5, 1]
    A[2] = B[2]                                   # zero-length segment
    A[3], B[3] = V[T[100][0]], V[T[100][1]]      # along a triangle edge
    A[4] = V[T[200][0]] - [0, 0, 0.5]            # through a vertex
    B[4] = V[T[200][0]] + [0, 0, 0.5]
    c = V[T[100]].mean(0)                         # through the duplicated triangle
    A[5], B[5] = c - [0, 0, 0.5], c + [0, 0, 0.5]
    A[6], B[6] = [1e-25, 0.3, 0.5], [2e-25, 0.3, -0.5]       # |d_x| < 2^-60
    ref = oracle.brute(V, T, A, B)
    bvh = rsi.BVH(dev(V), dev(T))
    compare(run_all_modes(bvh, dev(A), dev(B)), ref, what="special")
    assert ref["tri"][5] == 100 and ref["count"][5] >= 2


def test_bad_index_sets_status():
    mesh, seg = synth.workload_small_bool(n_seg=100)
    T = mesh.T.copy()
    T[7, 1] = len(mesh.V) + 5
    T[8, 0] = -1
    bvh = rsi.BVH(dev(mesh.V), dev(T))
    o = bvh.intersect(dev(seg.A), dev(seg.B), "count")
    assert bvh.status() == 4          # RSI_ERR_BAD_INDEX
    assert bvh.status() == 0          # cleared
    # the bad triangles never hit (the oracle sees them as degenerate)
    good = np.ones(len(T), bool)
    good[[7, 8]] = False
    ref = oracle.brute(mesh.V, np.where(good[:, None], T, 0), seg.A, seg.B)
    np.testing.assert_array_equal(o["count"].cpu().numpy(), ref["count"])


def test_compaction(small):
    mesh, seg, ref = small
    bvh = rsi.BVH(dev(mesh.V), dev(mesh.T))
    got = run_all_modes(bvh, dev(seg.A), dev(seg.B), compact=True)
    for m in ("count", "nearest"):
        g = got[m]
        n = int(g["n_hits"][0])
        assert n == int((ref["count"] > 0).sum())
        idx = g["hit_idx"][:n]
        assert np.array_equal(np.sort(idx), np.nonzero(ref["count"] > 0)[0])
        if m == "count":
            np.testing.assert_array_equal(g["hit_count"][:n], ref["count"][idx])
        else:
            np.testing.assert_array_equal(g["hit_tri"][:n], ref["tri"][idx])
            assert_close(g["hit_dist"][:n], ref["dist"][idx], what="hit_dist")
            assert_close(g["hit_point"][:n], ref["point"][idx], what="hit_point")
    # capacity smaller than the number of hits: total still counted, no overrun
    o = bvh.intersect(dev(seg.A), dev(seg.B), "nearest", compact=True, hit_cap=7)
    torch.cuda.synchronize()
    assert int(o["n_hits"][0]) == int((ref["count"] > 0).sum())


def test_stats_counters(small):
    mesh, seg, ref = small
    bvh = rsi.BVH(dev(mesh.V), dev(mesh.T))
    o = bvh.intersect(dev(seg.A), dev(seg.B), "count", stats=True)
    st = o["stats"]
    assert st["segments"] == seg.n
    assert st["tri_tests"] >= ref["count"].sum()
    assert st["node_visits"] >= seg.n
    assert st["fp64_tests"] <= 0.01 * st["tri_tests"] + 10
    np.testing.assert_array_equal(o["count"].cpu().numpy(), ref["count"])


def test_refit_moves_with_vertices(small):
    mesh, seg, _ = small
    bvh = rsi.BVH(dev(mesh.V), dev(mesh.T))
    rng = np.random.default_rng(3)
    V2 = (mesh.V + rng.normal(0, 0.02, size=mesh.V.shape)).astype(np.float32)
    bvh.refit(dev(V2))
    ref = oracle.brute(V2, mesh.T, seg.A, seg.B)
    compare(run_all_modes(bvh, dev(seg.A), dev(seg.B)), ref, what="refit")
    tree_check(bvh.export(), mesh.n_tri)


@pytest.mark.parametrize("chunk,pin", [(0, "both"), (1000, "both"), (4103, "none"),
                                       (10**9, "both"), (777, "A only"), (0, "offset")])
def test_intersect_from_host_buffers(small, chunk, pin):
    """Both host paths: page-locked inputs read in place by the kernel
    ("both", and "offset": views starting inside a pinned allocation) and
    inputs staged by copies ("none", and "A only", where one of the two
    arrays is pageable)."""
    mesh, seg, ref = small
    bvh = rsi.BVH(dev(mesh.V), dev(mesh.T))
    A = torch.from_numpy(seg.A)
    B = torch.from_numpy(seg.B)
    if pin == "both":
        A, B = A.pin_memory(), B.pin_memory()
    elif pin == "A only":
        A = A.pin_memory()
    elif pin == "offset":
        k = 5
        A = torch.cat([torch.zeros(k, 3), A]).pin_memory()[k:]
        B = torch.cat([torch.zeros(k, 3), B]).pin_memory()[k:]
        assert A.is_contiguous() and A.is_pinned()
    s = torch.cuda.Stream()
    got = {}
    for m in ("bool", "count", "nearest"):
        got[m] = bvh.intersect_host(A, B, m, chunk=chunk, stream=s)
    s.synchronize()
    got = {m: {k: v.numpy() for k, v in d.items()} for m, d in got.items()}
    compare(got, ref, what=f"host chunk={chunk}")


def test_points_inside_star_shaped_sphere():
    """Odd parity against the independent radial truth of a star-shaped
    closed surface: p is inside iff |p| < radius of the surface along p."""
    rng = np.random.default_rng(9)
    mesh = synth.icosphere(5, rng)
    P = rng.uniform(-1.3, 1.3, size=(20000, 3)).astype(np.float32)
    bvh = rsi.BVH(dev(mesh.V), dev(mesh.T))
    got = bvh.points_inside(dev(P)).cpu().numpy()
    rmax = float(np.linalg.norm(mesh.V.astype(np.float64), axis=1).max())
    u = P.astype(np.float64) / np.linalg.norm(P.astype(np.float64), axis=1, keepdims=True)
    r = oracle.brute(mesh.V, mesh.T, np.zeros_like(P), (u * rmax * 1.5).astype(np.float32))
    rs = np.linalg.norm(r["point"], axis=1)
    rp = np.linalg.norm(P.astype(np.float64), axis=1)
    ok = (r["count"] == 1) & (r["neardeg"] == 0) & (np.abs(rp - rs) > 1e-4)
    assert ok.mean() > 0.98
    np.testing.assert_array_equal(got[ok], (rp < rs)[ok].astype(np.uint8))
    assert 0.2 < got.mean() < 0.8


@pytest.mark.parametrize("levels", [0, 10])
def test_stack_overflow_reruns_with_deep_stack(levels):
    """An 8-entry stack overflows on a deep tree; the overflowed segments are
    re-run with the 64-entry stack and the results do not change.  With a
    top treelet (levels > 0) binary traversal re-runs from the treelet root
    and 4-wide traversal from the global root."""
    rng = np.random.default_rng(12)
    mesh = synth.icosphere(7, rng)                 # 327,680 triangles
    seg = synth.segments_box(rng, 20000, [-1.5] * 3, [1.5] * 3, [-1.5] * 3, [1.5] * 3)
    bvh = rsi.BVH(dev(mesh.V), dev(mesh.T), top_levels=levels)
    A, B = dev(seg.A), dev(seg.B)
    deep = {m: bvh.intersect(A, B, m) for m in ("count", "nearest")}
    for w in (2, 4):
        small = {m: bvh.intersect(A, B, m, launch=dict(stack_depth=8, node_width=w), stats=True)
                 for m in ("count", "nearest")}
        assert small["count"]["stats"]["overflows"] > 0
        assert torch.equal(small["count"]["count"], deep["count"]["count"])
        assert torch.equal(small["nearest"]["tri"], deep["nearest"]["tri"])
        assert torch.equal(small["nearest"]["tuv"], deep["nearest"]["tuv"])
    idx = np.random.default_rng(0).choice(seg.n, 300, replace=False)
    ref = oracle.brute(mesh.V, mesh.T, seg.A[idx], seg.B[idx])
    np.testing.assert_array_equal(deep["count"]["count"].cpu().numpy()[idx], ref["count"])


# ------------------------------------------------------------ full sizes
@pytest.fixture(scope="module")
def paper_scale():
    mesh, seg = synth.workload_paper_bool()
    return mesh, seg


def test_paper_scale_all_modes_sampled(paper_scale):
    """29,768 triangles x 10M segments in the benchmark's launch
    configuration, all three modes; 20k sampled segments against brute
    force (flags, counts and triangle ids exactly, nearest values within
    1e-5), invariants on all 10M."""
    mesh, seg = paper_scale
    assert mesh.n_tri == 29768 and seg.n == 10_000_000
    bvh = rsi.BVH(dev(mesh.V), dev(mesh.T))
    A, B = dev(seg.A), dev(seg.B)
    flag = bvh.intersect(A, B, "bool")["flag"].cpu().numpy()
    cnt = bvh.intersect(A, B, "count")["count"].cpu().numpy()
    near = {k: v.cpu().numpy() for k, v in bvh.intersect(A, B, "nearest").items()}
    assert np.array_equal(flag, (cnt > 0).astype(np.uint8))      # holds at any size
    assert np.array_equal(near["tri"] >= 0, cnt > 0)
    hit = near["tri"] >= 0
    assert np.all((near["tuv"][hit] >= 0) & (near["tuv"][hit] <= 1))
    idx = np.random.default_rng(0).choice(seg.n, 20000, replace=False)
    ref = oracle.brute(mesh.V, mesh.T, seg.A[idx], seg.B[idx])
    nd = int(ref["neardeg"].sum())
    np.testing.assert_array_equal(flag[idx], ref["flag"], err_msg=f"flag ({nd} near-degenerate)")
    np.testing.assert_array_equal(cnt[idx], ref["count"], err_msg=f"count ({nd} near-degenerate)")
    np.testing.assert_array_equal(near["tri"][idx], ref["tri"], err_msg=f"tri ({nd} near-degenerate)")
    for k in ("tuv", "point", "dist"):
        assert_close(near[k][idx], ref[k], what=f"{k} ({nd} near-degenerate)")
    assert 0.05 < flag.mean() < 0.95


def test_sphere_scale_count_nearest_sampled():
    """1,310,720-triangle icosphere x 1M segments, count + nearest; 20k
    sampled segments against the oracle (its CPU BVH, pinned to brute force,
    over the FP64 test), parity invariant on all."""
    mesh, seg = synth.workload_sphere()
    assert mesh.n_tri == 1_310_720 and mesh.n_vert == 655_362
    bvh = rsi.BVH(dev(mesh.V), dev(mesh.T))
    A, B = dev(seg.A), dev(seg.B)
    cnt = bvh.intersect(A, B, "count")["count"].cpu().numpy()
    o = bvh.intersect(A, B, "nearest", compact=True)
    tri = o["tri"].cpu().numpy()
    assert np.array_equal(tri >= 0, cnt > 0)
    assert int(o["n_hits"][0].item()) == int((cnt > 0).sum())
    idx = np.random.default_rng(1).choice(seg.n, 20000, replace=False)
    ref = oracle.CpuBVH(mesh.V, mesh.T).query(seg.A[idx], seg.B[idx])
    nd = int(ref["neardeg"].sum())
    np.testing.assert_array_equal(cnt[idx], ref["count"], err_msg=f"count ({nd} near-degenerate)")
    np.testing.assert_array_equal(tri[idx], ref["tri"], err_msg=f"tri ({nd} near-degenerate)")
    assert_close(o["tuv"].cpu().numpy()[idx], ref["tuv"], what=f"tuv ({nd} near-degenerate)")
    assert_close(o["point"].cpu().numpy()[idx], ref["point"], what=f"point ({nd} near-degenerate)")
    assert_close(o["dist"].cpu().numpy()[idx], ref["dist"], what=f"dist ({nd} near-degenerate)")
    # closed surface: both ends outside the bounding sphere -> even count
    rmax = np.linalg.norm(mesh.V.astype(np.float64), axis=1).max()
    out = (np.linalg.norm(seg.A, axis=1) > rmax) & (np.linalg.norm(seg.B, axis=1) > rmax)
    assert np.all(cnt[out] % 2 == 0)
    assert cnt.max() >= 4


def test_host_calls_alternate_streams_growing(small):
    """Host-buffer calls on one handle alternating between two streams, each
    ordered after the previous call by an event (the handle's rule), with
    growing segment counts so that the staging is reallocated between calls
    (freed on the current call's stream, which follows every earlier use):
    every result matches the oracle, in every mode and host path."""
    mesh, seg, ref = small
    V, T = dev(mesh.V), dev(mesh.T)
    bvh = rsi.BVH(V, T)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    calls = []
    prev = None
    for k, n in enumerate([500, 1500, 3000, 6007, 10000]):
        s = streams[k % 2]
        if prev is not None:
            s.wait_event(prev)
        A = torch.from_numpy(seg.A[:n]).pin_memory()
        B = torch.from_numpy(seg.B[:n]).pin_memory()
        mode = ("bool", "count", "nearest")[k % 3]
        # the streamed BOOL path, the in-place path and the staged path (pageable)
        if k == 3:
            A, B = torch.from_numpy(seg.A[:n].copy()), torch.from_numpy(seg.B[:n].copy())
        calls.append((n, mode, bvh.intersect_host(A, B, mode, chunk=1024, stream=s), A, B))
        prev = torch.cuda.Event()
        prev.record(s)
    for s in streams:
        s.synchronize()
    for n, mode, o, _, _ in calls:
        key = {"bool": "flag", "count": "count", "nearest": "tri"}[mode]
        np.testing.assert_array_equal(o[key].numpy(), ref[key][:n], err_msg=f"{mode} n={n}")
    assert bvh.status(streams[0]) == 0


def test_host_calls_back_to_back(small):
    """Streamed BOOL calls, in-place COUNT / NEAREST calls and rebuilds
    queued on one stream without synchronising in between, with inputs of
    different sizes: every result matches (the staging is shared, and a
    streamed call's copies start as soon as the previous streamed call is
    done with it)."""
    mesh, seg, ref = small
    V, T = dev(mesh.V), dev(mesh.T)
    bvh = rsi.BVH(V, T)
    A, B = torch.from_numpy(seg.A).pin_memory(), torch.from_numpy(seg.B).pin_memory()
    n2 = 6007
    A2, B2 = A[:n2].clone().pin_memory(), B[:n2].clone().pin_memory()
    s = torch.cuda.Stream()
    outs = []
    for it in range(3):
        bvh.build(V, T, stream=s)
        outs.append(("bool", None, bvh.intersect_host(A, B, "bool", chunk=1024, stream=s)))
        outs.append(("count", None, bvh.intersect_host(A, B, "count", stream=s)))
        outs.append(("bool", n2, bvh.intersect_host(A2, B2, "bool", stream=s)))
        outs.append(("nearest", n2, bvh.intersect_host(A2, B2, "nearest", stream=s)))
        outs.append(("bool", None, bvh.intersect_host(A, B, "bool", chunk=4096, stream=s)))
    s.synchronize()
    for mode, n, o in outs:
        sel = slice(None) if n is None else slice(0, n)
        key = {"bool": "flag", "count": "count", "nearest": "tri"}[mode]
        np.testing.assert_array_equal(o[key].numpy(), ref[key][sel], err_msg=f"{mode} n={n}")
    assert bvh.status() == 0


def test_streamed_calls_alternate_staging_slots(small):
    """Streamed BOOL calls only, back to back on one stream with different
    segments, sizes and chunks and a rebuild now and then: consecutive calls
    use the two staging slots in turn and a call's copies overlap the
    previous call's traversal; every result matches the oracle's flags."""
    mesh, seg, ref = small
    V, T = dev(mesh.V), dev(mesh.T)
    bvh = rsi.BVH(V, T)
    rng = np.random.default_rng(5)
    s = torch.cuda.Stream()
    calls = []
    for k, (n, chunk) in enumerate([(10000, 0), (6007, 1024), (9000, 64), (33, 0), (10000, 512),
                                    (1, 0), (7777, 2048), (4096, 32), (10000, 0)]):
        idx = rng.permutation(seg.n)[:n]
        A = torch.from_numpy(seg.A[idx]).pin_memory()
        B = torch.from_numpy(seg.B[idx]).pin_memory()
        if k % 3 == 2:
            bvh.build(V, T, stream=s)
        calls.append((idx, bvh.intersect_host(A, B, "bool", chunk=chunk, stream=s), A, B))
    s.synchronize()
    for idx, o, _, _ in calls:
        np.testing.assert_array_equal(o["flag"].numpy(), ref["flag"][idx], err_msg=f"n={idx.size}")
    assert bvh.status() == 0


_BLOCKING_CHILD = r"""
import numpy as np, torch
import paper_2209_02878_gb300 as rsi
from paper_2209_02878_gb300 import synth
mesh, seg = synth.workload_small_bool()
V, T = torch.from_numpy(mesh.V).cuda(), torch.from_numpy(mesh.T).cuda()
A, B = torch.from_numpy(seg.A).pin_memory(), torch.from_numpy(seg.B).pin_memory()
bvh = rsi.BVH(V, T)
want = bvh.intersect(A.cuda(), B.cuda(), "bool")["flag"].cpu()
outs = [bvh.intersect_host(A, B, "bool", chunk=1024) for _ in range(3)]
torch.cuda.synchronize()
assert all(torch.equal(o["flag"], want) for o in outs)
assert bvh.status() == 0, bvh.status()
print("ok")
"""


def test_streamed_call_with_blocking_launches():
    """With CUDA_LAUNCH_BLOCKING=1 a launch returns only when its kernel has
    ended, so the streamed path must queue the chunk copies before the
    traversal that waits for them: the calls finish with correct flags and
    no timeout in the status."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, CUDA_LAUNCH_BLOCKING="1",
               PYTHONPATH=root + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", _BLOCKING_CHILD], cwd=root, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr
