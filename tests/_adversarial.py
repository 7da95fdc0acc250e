"""Seeded adversarial inputs for the segment / triangle test: triangles over
many binades and segments whose exact crossing sits near an edge, a vertex
or a segment end, or that run nearly parallel to the triangle's plane (a
crossing at a grazing angle).  Input generation only: no arithmetic of the
method (the Moller-Trumbore test, its error bounds or its outputs) lives
here.

`adversarial` gives one segment per triangle (independent pairs, for the
CPU emulations); `adversarial_groups` gives small meshes of a few triangles
that share a frame, each with many segments aimed at its triangles (for the
GPU path, one mesh per group, where a segment may cross several triangles
of its group)."""
import numpy as np

F = np.float32


def _frames(rng, n):
    """Per-row scale and offset over 24 binades each."""
    scale = 2.0 ** rng.uniform(-12, 12, n)[:, None]
    offset = rng.normal(size=(n, 3)) * 2.0 ** rng.uniform(-12, 12, n)[:, None]
    return scale, offset


def _segments_near(rng, v0, v1, v2, scale):
    """One segment per row aimed at triangle (v0, v1, v2) (float64 arrays):
    kind 0-2 cross within delta (1e-9 .. 1e-3, barycentric units) of an edge,
    kind 3 of the vertex v0, kind 4 end within delta of the plane, kind 5
    runs nearly parallel to the plane (normal component delta), on either
    side of the boundary; the rest are ordinary crossings."""
    n = v0.shape[0]
    delta = 10.0 ** rng.uniform(-9, -3, n)
    kind = rng.integers(0, 6, n)
    u = rng.uniform(0, 1, n)
    v = rng.uniform(0, 1, n) * (1 - u)
    sgn = rng.choice([-1.0, 1.0], n)
    u = np.where(kind == 0, sgn * delta, u)                       # near the edge u = 0
    v = np.where(kind == 1, sgn * delta, v)                       # near the edge v = 0
    v = np.where(kind == 2, 1 - u + sgn * delta, v)               # near the edge u + v = 1
    u = np.where(kind == 3, sgn * delta, u)                       # near the vertex v0
    v = np.where(kind == 3, rng.choice([-1.0, 1.0], n) * delta, v)
    X = v0 + u[:, None] * (v1 - v0) + v[:, None] * (v2 - v0)
    nrm = np.cross(v1 - v0, v2 - v0)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    dirn = rng.normal(size=(n, 3))
    dirn /= np.linalg.norm(dirn, axis=1, keepdims=True)
    # nearly parallel: the in-plane part of a direction plus a tiny normal part
    par = dirn - np.sum(dirn * nrm, axis=1, keepdims=True) * nrm
    par = par / np.linalg.norm(par, axis=1, keepdims=True) + sgn[:, None] * delta[:, None] * nrm
    dirn = np.where((kind == 5)[:, None], par, dirn)
    length = scale * 2.0 ** rng.uniform(-3, 3, n)[:, None]
    t0 = rng.uniform(0, 1, n)
    t0 = np.where(kind == 4, rng.choice([0.0, 1.0], n) + sgn * delta, t0)  # near a segment end
    a = X - t0[:, None] * length * dirn
    b = a + length * dirn
    return a, b


def adversarial(rng, n):
    """n independent (segment, triangle) pairs: float32 (a, b, v0, v1, v2)."""
    scale, offset = _frames(rng, n)
    v0 = offset + scale * rng.normal(size=(n, 3))
    v1 = offset + scale * rng.normal(size=(n, 3))
    v2 = offset + scale * rng.normal(size=(n, 3))
    a, b = _segments_near(rng, v0, v1, v2, scale)
    return tuple(x.astype(F) for x in (a, b, v0, v1, v2))


def adversarial_groups(rng, n_groups, k, m):
    """n_groups meshes of k triangles sharing one frame (scale, offset), and
    m segments per mesh, each aimed at one of its triangles.  Returns float32
    V [n_groups, 3k, 3] (triangle j of a group = its vertices 3j, 3j+1,
    3j+2), float32 A, B [n_groups, m, 3] and the aimed-at triangle
    int [n_groups, m]."""
    scale, offset = _frames(rng, n_groups)
    V = offset[:, None, :] + scale[:, None, :] * rng.normal(size=(n_groups, 3 * k, 3))
    V = V.astype(F).astype(np.float64)   # aim at the float32 triangles
    target = rng.integers(0, k, size=(n_groups, m))
    g = np.repeat(np.arange(n_groups), m)
    j = target.ravel()
    v0, v1, v2 = (V[g, 3 * j + q] for q in range(3))
    a, b = _segments_near(rng, v0, v1, v2, scale[g])
    return (V.astype(F), a.reshape(n_groups, m, 3).astype(F),
            b.reshape(n_groups, m, 3).astype(F), target)
