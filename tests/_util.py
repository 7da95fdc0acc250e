"""Shared helpers of the GPU tests: tolerance checks and the host-side tree
validator.  No arithmetic of the method lives here."""
import numpy as np

REL = 1e-5  # points, (t, u, v), distances and gradients: relative 1e-5


def close(x, ref, rel=REL):
    """|x - ref| <= rel * max(1, |ref|) elementwise; returns the bad mask."""
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    return np.abs(x - ref) > rel * np.maximum(1.0, np.abs(ref))


def assert_close(x, ref, rel=REL, what=""):
    bad = close(x, ref, rel)
    assert not bad.any(), f"{what}: {int(bad.sum())} of {bad.size} outside rel {rel}; " \
                          f"first at {np.argwhere(bad)[:3].tolist()}"


def tree_check(exp, nT, leaf_size=1, max_depth=64):
    """Validate an exported traversal tree (rsi_bvh_export `nodes`):
    every leaf position reached exactly once from the root slot, child boxes
    equal to the union of what lies below, leaves within leaf_size, depth
    bounded.  Returns the depth."""
    if nT == 0:
        return 0
    f = exp["nodes"]
    ii = exp["nodes_i"]
    lbox = exp["lbox"]
    seen = np.zeros(nT, np.int64)
    depth = 0
    root = nT - 1
    stack = [(root, 0)]
    while stack:
        node, d = stack.pop()
        depth = max(depth, d)
        assert d <= max_depth, "tree deeper than the stack bound"
        for k in range(2):
            # children interleaved: lo.x0 lo.x1 lo.y0 lo.y1 lo.z0 lo.z1 hi.x0 ...
            box = f[node, [k, 2 + k, 4 + k, 6 + k, 8 + k, 10 + k]]
            ref, cnt = int(ii[node, 12 + k]), int(ii[node, 14 + k])
            if cnt > 0:
                assert cnt <= leaf_size or node == root, "leaf larger than leaf_size"
                seen[ref:ref + cnt] += 1
                lb = lbox[ref:ref + cnt]
                union = np.r_[lb[:, :3].min(0), lb[:, 3:].max(0)]
                assert np.array_equal(box, union), "leaf box is not the union of its triangles"
            elif ref >= 0:
                sub = f[ref]
                b0 = sub[[0, 2, 4, 6, 8, 10]]
                b1 = sub[[1, 3, 5, 7, 9, 11]]
                lo = np.minimum(b0[:3], b1[:3])
                hi = np.maximum(b0[3:], b1[3:])
                # an empty second child (root slot) is stored at +inf
                if np.isinf(b1).all():
                    lo, hi = b0[:3], b0[3:]
                assert np.array_equal(box, np.r_[lo, hi]), "internal box is not its children's union"
                stack.append((ref, d + 1))
            else:
                assert node == root and k == 1 and np.isinf(box).all()
    assert np.all(seen == 1), "some leaf position not reached exactly once"
    return depth
