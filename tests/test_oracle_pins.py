"""Pins for the FP64 CPU oracle, each against something other than the oracle
itself: hand-derived values, closed forms, an independent construction, brute
force, or invariants the mathematics fixes.  CPU only."""
import math

import numpy as np
import pytest

from paper_2209_02878_gb300 import synth

from _golden import load_inside_case, load_lbvh_case, load_mt_cases

UNIT = ([0, 0, 0], [1, 0, 0], [0, 1, 0])


# ---------------------------------------------------------------- hand cases
def test_axis_aligned_hit_exact(orc):
    # d=(0,0,2), e1=(1,0,0), e2=(0,1,0): p=(-2,0,0), det=-2 -> 2;
    # s0=(.25,.25,-1), q=(0,-1,-.25): nU=.5, nV=.5, nT=1 after the sign flip.
    hit, det, nu, nv, nt = orc.mt([0.25, 0.25, -1], [0.25, 0.25, 1], *UNIT)
    assert hit and (det, nu, nv, nt) == (2.0, 0.5, 0.5, 1.0)
    o = orc.brute(np.array(UNIT, np.float32), np.array([[0, 1, 2]]),
                  np.array([[0.25, 0.25, -1]]), np.array([[0.25, 0.25, 1]]))
    assert o["flag"][0] == 1 and o["count"][0] == 1 and o["tri"][0] == 0
    assert tuple(o["tuv"][0]) == (0.5, 0.25, 0.25)
    assert tuple(o["point"][0]) == (0.25, 0.25, 0.0)
    assert o["dist"][0] == 1.0
    assert o["neardeg"][0] == 0


@pytest.mark.parametrize("case", load_mt_cases(), ids=lambda c: c["name"])
def test_golden_hand_cases(orc, case):
    """tests/golden/mt_hand_cases.txt: hand-derived flags, counts, nearest
    triangles and exact (t, u, v), points and distances (dyadic inputs, so
    FP64 reproduces them exactly)."""
    o = orc.brute(case["V"], case["T"], case["A"], case["B"])
    assert (o["flag"][0], o["count"][0], o["tri"][0]) == \
        (case["flag"], case["count"], case["tri"]), case["name"]
    if "tuv" in case:
        assert list(o["tuv"][0]) == list(case["tuv"]), case["name"]
        assert list(o["point"][0]) == list(case["point"]), case["name"]
        assert o["dist"][0] == case["dist"], case["name"]


@pytest.mark.parametrize("a,b,why", [
    ([0.75, 0.75, -1], [0.75, 0.75, 1], "beside: u+v=1.5"),
    ([0.25, 0.25, -1], [0.25, 0.25, -0.5], "stops short: t=2"),
    ([0.25, 0.25, 0.5], [0.25, 0.25, 1], "starts past: t<0"),
    ([0.25, 0.25, 1], [0.5, 0.25, 1], "parallel: det=0"),
])
def test_misses(orc, a, b, why):
    hit, det, *_ = orc.mt(a, b, *UNIT)
    assert not hit, why
    if "parallel" in why:
        assert det == 0.0


def test_coplanar_is_miss_and_near_degenerate(orc):
    V = np.array(UNIT, np.float32)
    o = orc.brute(V, np.array([[0, 1, 2]]), np.array([[-0.5, 0.25, 0]]),
                  np.array([[1.5, 0.25, 0]]))
    assert o["flag"][0] == 0 and o["neardeg"][0] == 1


def test_edge_band(orc):
    # float32(1e-9) > 0: just inside the v=0 edge -> hit; just outside -> miss;
    # both inside the 1e-6 near-degenerate band.
    V = np.array(UNIT, np.float32)
    T = np.array([[0, 1, 2]])
    A = np.array([[0.5, 1e-9, -1], [0.5, -1e-9, -1]], np.float32)
    B = np.array([[0.5, 1e-9, 1], [0.5, -1e-9, 1]], np.float32)
    o = orc.brute(V, T, A, B)
    assert list(o["flag"]) == [1, 0]
    assert list(o["neardeg"]) == [1, 1]


def test_endpoint_on_plane_is_hit(orc):
    hit, det, nu, nv, nt = orc.mt([0.25, 0.25, -1], [0.25, 0.25, 0], *UNIT)
    assert hit and nt == det  # t = 1 exactly, closed interval


@pytest.mark.parametrize("tri", [
    ([0, 0, 0], [1, 0, 0], [2, 0, 0]),
    ([0, 0, 0], [0, 0, 0], [0, 1, 0]),
    ([0.5, 0.5, 0], [0.5, 0.5, 0], [0.5, 0.5, 0]),
])
def test_degenerate_triangle_never_hits(orc, tri):
    hit, det, *_ = orc.mt([0.5, 0.0, -1], [0.5, 0.0, 1], *tri)
    assert not hit and det == 0.0


def test_reversed_winding_same_hit(orc):
    f = orc.mt([0.2, 0.3, -1], [0.2, 0.3, 1], [0, 0, 0], [1, 0, 0], [0, 1, 0])
    r = orc.mt([0.2, 0.3, -1], [0.2, 0.3, 1], [0, 0, 0], [0, 1, 0], [1, 0, 0])
    assert f[0] and r[0]
    assert f[4] / f[1] == r[4] / r[1]          # same t
    assert f[2] / f[1] == r[3] / r[1]          # u and v swap
    assert f[3] / f[1] == r[2] / r[1]


def test_nan_segment_is_miss(orc):
    V = np.array(UNIT, np.float32)
    o = orc.brute(V, np.array([[0, 1, 2]]), np.array([[np.nan, 0.25, -1]]),
                  np.array([[0.25, 0.25, 1]]))
    assert o["flag"][0] == 0 and o["tri"][0] == -1


def test_non_finite_never_hits(orc):
    # without the rule, an infinite start gives det = nT = inf and a "hit"
    V = np.array(UNIT, np.float32)
    T = np.array([[0, 1, 2]])
    A = np.array([[0.25, 0.25, -np.inf], [0.25, 0.25, -1]], np.float32)
    B = np.array([[0.25, 0.25, 1], [0.25, 0.25, 1]], np.float32)
    o = orc.brute(V, T, A, B)
    assert list(o["flag"]) == [0, 1]
    V2 = V.copy()
    V2[1, 0] = np.inf
    assert orc.brute(V2, T, A[1:], B[1:])["flag"][0] == 0


def test_nearest_tie_goes_to_lower_index(orc):
    # two copies of the same triangle: equal t, the smaller index wins
    V = np.array(UNIT, np.float32)
    T = np.array([[0, 1, 2], [0, 1, 2]])
    o = orc.brute(V, T, np.array([[0.2, 0.2, -1]]), np.array([[0.2, 0.2, 1]]))
    assert o["count"][0] == 2 and o["tri"][0] == 0


def test_nearest_picks_min_t(orc):
    # planes z=0 (tri 0) and z=-0.5 (tri 1); segment from z=-1 upward
    V = np.array(UNIT + ([0, 0, -0.5], [1, 0, -0.5], [0, 1, -0.5]), np.float32)
    T = np.array([[0, 1, 2], [3, 4, 5]])
    o = orc.brute(V, T, np.array([[0.2, 0.2, -1]]), np.array([[0.2, 0.2, 1]]))
    assert o["count"][0] == 2 and o["tri"][0] == 1 and o["tuv"][0][0] == 0.25


def test_bad_index_rejected(orc):
    with pytest.raises(ValueError):
        orc.brute(np.array(UNIT, np.float32), np.array([[0, 1, 3]]),
                  np.zeros((1, 3)), np.ones((1, 3)))


# ---------------------------------------------------------------- closed forms
def _plane_z(p0, p1, p2, x, y):
    """Height at (x,y) of the plane through three points (float64, Cramer)."""
    M = np.array([[p1[0] - p0[0], p2[0] - p0[0]], [p1[1] - p0[1], p2[1] - p0[1]]])
    l1, l2 = np.linalg.solve(M, [x - p0[0], y - p0[1]])
    return p0[2] + l1 * (p1[2] - p0[2]) + l2 * (p2[2] - p0[2]), l1, l2


def test_heightfield_vertical_segment_hits_once(orc):
    rng = np.random.default_rng(11)
    G = 17
    mesh = synth.heightfield(G, rng)
    V, T = mesh.V.astype(np.float64), mesh.T
    n = 3000
    xy = rng.uniform(0.001, 0.999, size=(n, 2)).astype(np.float32)
    zlo, zhi = V[:, 2].min() - 1, V[:, 2].max() + 1
    A = np.c_[xy, np.full(n, zlo)].astype(np.float32)
    B = np.c_[xy, np.full(n, zhi)].astype(np.float32)
    o = orc.brute(mesh.V, T, A, B)
    ok = o["neardeg"] == 0
    assert ok.mean() > 0.99
    assert np.all(o["count"][ok] == 1)
    # independent expected triangle and height from the grid cell + diagonal
    for k in np.nonzero(ok)[0][:500]:
        x, y = float(xy[k, 0]), float(xy[k, 1])
        i = min(int(x * (G - 1)), G - 2)
        j = min(int(y * (G - 1)), G - 2)
        # the float32 grid coordinates are not exactly i/(G-1): step to the cell
        while V[j * G + i + 1, 0] < x:
            i += 1
        while V[j * G + i, 0] > x:
            i -= 1
        while V[(j + 1) * G + i, 1] < y:
            j += 1
        while V[j * G + i, 1] > y:
            j -= 1
        v00, v10 = j * G + i, j * G + i + 1
        v01, v11 = (j + 1) * G + i, (j + 1) * G + i + 1
        z1, a1, b1 = _plane_z(V[v00], V[v10], V[v11], x, y)
        inside1 = a1 >= 0 and b1 >= 0 and a1 + b1 <= 1
        z2, a2, b2 = _plane_z(V[v00], V[v11], V[v01], x, y)
        q = 2 * (j * (G - 1) + i)
        exp_tri, exp_z = (q, z1) if inside1 else (q + 1, z2)
        assert o["tri"][k] == exp_tri
        assert abs(o["point"][k][2] - exp_z) <= 1e-12 * max(1.0, abs(exp_z))
        assert o["point"][k][0] == x and o["point"][k][1] == y


def test_icosphere_star_shaped_counts_and_parity(orc):
    rng = np.random.default_rng(5)
    mesh = synth.icosphere(3, rng)
    V, T = mesh.V, mesh.T
    rmax = float(np.linalg.norm(V.astype(np.float64), axis=1).max())
    n = 4000
    # radial segments from the origin cross exactly once
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    far = (d * (rmax * 1.5)).astype(np.float32)
    o = orc.brute(V, T, np.zeros((n, 3), np.float32), far)
    ok = o["neardeg"] == 0
    assert ok.mean() > 0.99 and np.all(o["count"][ok] == 1)
    # both ends outside the bounding sphere: even count
    A = (rng.normal(size=(n, 3)))
    A = (A / np.linalg.norm(A, axis=1, keepdims=True) * rmax * 1.2).astype(np.float32)
    B = (-A * rng.uniform(0.8, 1.0, size=(n, 1))).astype(np.float32)
    B = (B / np.linalg.norm(B, axis=1, keepdims=True) * rmax * 1.2).astype(np.float32)
    o = orc.brute(V, T, A, B)
    ok = o["neardeg"] == 0
    assert np.all(o["count"][ok] % 2 == 0)
    # parity = inside(a) xor inside(b), inside() from the radial hit radius
    A = rng.uniform(-1.5, 1.5, size=(n, 3)).astype(np.float32)
    B = rng.uniform(-1.5, 1.5, size=(n, 3)).astype(np.float32)
    o = orc.brute(V, T, A, B)

    def inside(P):
        u = P.astype(np.float64) / np.linalg.norm(P.astype(np.float64), axis=1, keepdims=True)
        r = orc.brute(V, T, np.zeros_like(P), (u * rmax * 1.5).astype(np.float32))
        rs = np.linalg.norm(r["point"], axis=1)
        good = (r["count"] == 1) & (r["neardeg"] == 0)
        return np.linalg.norm(P.astype(np.float64), axis=1) < rs, good, rs

    ia, ga, ra = inside(A)
    ib, gb, rb = inside(B)
    margin = (np.abs(np.linalg.norm(A.astype(np.float64), axis=1) - ra) > 1e-6) & \
             (np.abs(np.linalg.norm(B.astype(np.float64), axis=1) - rb) > 1e-6)
    ok = (o["neardeg"] == 0) & ga & gb & margin
    assert ok.mean() > 0.98
    assert np.all((o["count"][ok] % 2 == 1) == (ia[ok] ^ ib[ok]))
    assert (o["count"] > 1).any()  # the workload really has multiple crossings


# ---------------------------------------------------------------- brute vs BVH
def _same(o1, o2):
    for k in ("flag", "count", "tri", "neardeg"):
        np.testing.assert_array_equal(o1[k], o2[k], err_msg=k)
    for k in ("tuv", "point", "dist"):
        np.testing.assert_array_equal(o1[k], o2[k], err_msg=k)


def test_cpu_bvh_equals_brute_on_small_heightfield(orc):
    mesh, seg = synth.workload_small_bool()
    assert mesh.n_tri == 1922 and seg.n == 10_000
    _same(orc.brute(mesh.V, mesh.T, seg.A, seg.B),
          orc.CpuBVH(mesh.V, mesh.T).query(seg.A, seg.B))


@pytest.mark.parametrize("seed", range(6))
def test_cpu_bvh_equals_brute_on_tiny_soups(orc, seed):
    rng = np.random.default_rng(100 + seed)
    mesh, seg = synth.random_soup(rng, int(rng.integers(1, 51)), 10_000)
    b = orc.brute(mesh.V, mesh.T, seg.A, seg.B)
    _same(b, orc.CpuBVH(mesh.V, mesh.T).query(seg.A, seg.B))
    assert b["count"].max() >= 1


def test_cpu_bvh_equals_brute_on_random_direction_sample(orc):
    mesh, seg = synth.workload_paper_bool(n_seg=4000, G=40)
    _same(orc.brute(mesh.V, mesh.T, seg.A, seg.B),
          orc.CpuBVH(mesh.V, mesh.T).query(seg.A, seg.B))


# ---------------------------------------------------------------- invariants
def test_output_invariants(orc):
    mesh, seg = synth.workload_sphere(n_seg=2000, level=3)
    o = orc.brute(mesh.V, mesh.T, seg.A, seg.B)
    assert np.all(o["count"] >= o["flag"])
    assert np.all(o["flag"] == (o["count"] > 0))
    assert np.all((o["tri"] >= 0) == (o["flag"] == 1))
    h = o["tri"] >= 0
    t, u, v = o["tuv"][h].T
    assert np.all((t >= 0) & (t <= 1) & (u >= 0) & (v >= 0) & (u + v <= 1))
    for k in np.nonzero(h)[0][:200]:
        j = o["tri"][k]
        tri = mesh.V[mesh.T[j]]
        assert orc.mt(seg.A[k], seg.B[k], *tri)[0]
        # the reported hit point lies on the segment and on the triangle plane
        P = o["point"][k]
        p0, p1, p2 = tri.astype(np.float64)
        nrm = np.cross(p1 - p0, p2 - p0)
        assert abs(np.dot(nrm, P - p0)) <= 1e-12 * np.linalg.norm(nrm) * 4


# ---------------------------------------------------------------- Morton / LBVH
def test_morton_interleave_known_values(orc):
    assert orc.morton3(1, 0, 0) == 4
    assert orc.morton3(0, 1, 0) == 2
    assert orc.morton3(0, 0, 1) == 1
    assert orc.morton3(3, 0, 0) == 4 + 32
    assert orc.morton3(0, 0, 1023) == int("001" * 10, 2)
    assert orc.morton3(1023, 1023, 1023) == (1 << 30) - 1
    assert orc.morton3(512, 0, 0) == 1 << 29


def _point_mesh(points):
    # degenerate "triangles" whose three corners coincide: centroid = point
    P = np.asarray(points, np.float32)
    V = np.repeat(P, 3, axis=0)
    T = np.arange(3 * len(P), dtype=np.int32).reshape(-1, 3)
    return V, T


def test_lbvh_hand_example(orc):
    """tests/golden/lbvh_hand_case.txt: six centroids at binary fractions, so
    the quantised coordinates, codes, order, radix tree and boxes are exact
    (derivation in the file)."""
    c = load_lbvh_case()
    o = orc.lbvh(c["V"], c["T"])
    assert list(o["bounds"]) == c["bounds"]
    assert list(o["codes"]) == c["codes"]
    assert list(o["order"]) == c["order"]
    assert list(o["left"]) == c["left"]
    assert list(o["right"]) == c["right"]
    assert o["range"].tolist() == c["range"]
    for k in (0, 3, 4):
        assert o["nbox"][k].tolist() == c[f"nbox{k}"]


def _trie_tree(keys):
    """Independent construction: insert the keys into a binary trie bit by
    bit, then drop nodes with a single child.  Returns {(f,l): split}."""
    root = {}
    for i, k in enumerate(keys):
        node = root
        for bit in range(63, -1, -1):
            node = node.setdefault((k >> bit) & 1, {})
        node["leaf"] = i
    out = {}

    def walk(node):  # returns (first, last) leaf of the subtree
        if "leaf" in node:
            return node["leaf"], node["leaf"]
        kids = [node[b] for b in (0, 1) if b in node]
        if len(kids) == 1:
            return walk(kids[0])
        f0, l0 = walk(kids[0])
        f1, l1 = walk(kids[1])
        out[(f0, l1)] = l0
        return f0, l1

    walk(root)
    return out


@pytest.mark.parametrize("seed", range(4))
def test_lbvh_radix_tree_matches_trie(orc, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 300))
    pts = rng.uniform(0, 1, size=(n, 3))
    dup = rng.integers(0, n, size=n // 4)           # force duplicate codes
    pts[rng.integers(0, n, size=n // 4)] = pts[dup]
    V, T = _point_mesh(pts)
    o = orc.lbvh(V, T)
    codes = o["codes"][o["order"]].astype(np.uint64)
    assert np.all(np.diff(codes.astype(np.int64)) >= 0)
    keys = [(int(c) << 32) | i for i, c in enumerate(codes)]
    want = _trie_tree(keys)
    got = {}
    for node in range(n - 1):
        f, l = o["range"][node]
        L = o["left"][node]
        split = (-L - 1) if L < 0 else o["range"][L][1]
        got[(int(f), int(l))] = int(split)
        assert node in (f, l) or node == 0  # Karras numbering
    assert got == want
    # boxes: every internal box is the union of its leaves' boxes
    for node in range(n - 1):
        f, l = o["range"][node]
        lb = o["lbox"][f:l + 1]
        assert np.array_equal(o["nbox"][node][:3], lb[:, :3].min(0))
        assert np.array_equal(o["nbox"][node][3:], lb[:, 3:].max(0))


def test_lbvh_quantisation_against_float32_numpy(orc):
    mesh, _ = synth.workload_small_bool()
    o = orc.lbvh(mesh.V, mesh.T)
    P = mesh.V[mesh.T]                                     # [n,3,3] float32
    c = ((P[:, 0] + P[:, 1]) + P[:, 2]) / np.float32(3)
    lo, hi = c.min(0), c.max(0)
    q = np.clip(np.floor(((c - lo) / (hi - lo)) * np.float32(1024)), 0, 1023).astype(np.uint32)

    def spread(x):  # bit k -> bit 3k
        r = np.zeros_like(x)
        for k in range(10):
            r |= ((x >> k) & 1) << (3 * k)
        return r

    codes = (spread(q[:, 0]) << 2) | (spread(q[:, 1]) << 1) | spread(q[:, 2])
    np.testing.assert_array_equal(o["codes"], codes)
    np.testing.assert_array_equal(o["bounds"], np.r_[lo, hi])
    np.testing.assert_array_equal(o["order"], np.lexsort((np.arange(len(codes)), codes)))


def test_morton2_interleave_known_values(orc):
    # height-field variant: first kept axis on the odd bits, 15 bits each
    assert orc.morton2(1, 0) == 2
    assert orc.morton2(0, 1) == 1
    assert orc.morton2(3, 0) == 2 + 8
    assert orc.morton2(0, 32767) == int("01" * 15, 2)
    assert orc.morton2(32767, 32767) == (1 << 30) - 1
    assert orc.morton2(16384, 0) == 1 << 29


@pytest.mark.parametrize("height_axis", [1, 2, 3])
def test_lbvh_height_axis_codes_against_float32_numpy(orc, height_axis):
    """The height-field option of the code: the coordinate along the height
    axis left out, the other two quantised to 2^15 levels (float32, as in
    the paper's quantisation) and interleaved bit by bit, first kept axis
    high; order by (code, index) and the radix tree as for the paper's code."""
    mesh, _ = synth.workload_small_bool()
    o = orc.lbvh(mesh.V, mesh.T, height_axis=height_axis)
    P = mesh.V[mesh.T]
    c = ((P[:, 0] + P[:, 1]) + P[:, 2]) / np.float32(3)
    lo, hi = c.min(0), c.max(0)
    q = np.clip(np.floor(((c - lo) / (hi - lo)) * np.float32(32768)), 0, 32767).astype(np.uint32)
    a, b = [k for k in range(3) if k != height_axis - 1]
    codes = np.zeros(len(q), np.uint32)
    for k in range(15):
        codes |= ((q[:, a] >> k) & 1) << (2 * k + 1)
        codes |= ((q[:, b] >> k) & 1) << (2 * k)
    np.testing.assert_array_equal(o["codes"], codes)
    np.testing.assert_array_equal(o["order"], np.lexsort((np.arange(len(codes)), codes)))
    keys = [(int(x) << 32) | i for i, x in enumerate(codes[o["order"]])]
    want = _trie_tree(keys)
    got = {}
    for node in range(len(codes) - 1):
        f, l = o["range"][node]
        L = o["left"][node]
        got[(int(f), int(l))] = int((-L - 1) if L < 0 else o["range"][L][1])
    assert got == want
    with pytest.raises(ValueError):
        orc.lbvh(mesh.V, mesh.T, height_axis=4)


def test_golden_cube_parity(orc):
    """tests/golden/cube_inside_cases.txt: the crossing count of a segment
    from each point along (0.31, 0.57, 0.76), 10 long, is odd exactly for
    the points inside the closed cube."""
    c = load_inside_case()
    u = np.array([0.31, 0.57, 0.76])
    B = (c["P"] + 10.0 * u / np.linalg.norm(u)).astype(np.float32)
    o = orc.brute(c["V"], c["T"], c["P"], B)
    np.testing.assert_array_equal(o["count"] % 2, c["inside"])
