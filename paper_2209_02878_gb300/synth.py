"""Seeded synthetic inputs for segment / triangle-mesh intersection.

This module only draws random numbers and lays out meshes; it contains none of
the intersection arithmetic.  Both the CUDA path and the CPU oracle consume the
arrays it returns (float32 vertices / segment endpoints, int32 triangle
indices, all C-contiguous AoS xyz), which is the input layout of the paper's
program (Sec. 2.5: vertices f32[N_v*3], triangles i32[N_t*3], rayFrom / rayTo
f32[N_r*3]).

The paper's own test surface (29,284 triangles) and its 10M random rays are not
available, so these recipes stand in for them:

* ``heightfield``  -- G x G vertex grid on [0,1]^2, each quad split on the
  (i,j)-(i+1,j+1) diagonal, z = 0.2 * sum_{k=1..3} sin(2 pi k (cos th_k x +
  sin th_k y) + phi_k) + N(0, 0.01), th, phi ~ U[0, 2 pi).
* ``icosphere``    -- icosahedron subdivided L times (midpoints projected to
  the unit sphere at every level), radius 1 + 0.05 n_v with n ~ N(0,1)
  smoothed by 10 Jacobi sweeps (0.5 self + 0.5 neighbour mean).
* segment recipes for each workload (see the ``workload_*`` functions).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TWO_PI = 2.0 * math.pi


@dataclass
class Mesh:
    V: np.ndarray  # float32 [N_v, 3]
    T: np.ndarray  # int32   [N_t, 3]
    kind: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_tri(self) -> int:
        return int(self.T.shape[0])

    @property
    def n_vert(self) -> int:
        return int(self.V.shape[0])


@dataclass
class Segments:
    A: np.ndarray  # float32 [N_r, 3] start points
    B: np.ndarray  # float32 [N_r, 3] end points

    @property
    def n(self) -> int:
        return int(self.A.shape[0])


# --------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------
def grid_triangles(G: int) -> np.ndarray:
    """Triangle indices of a G x G vertex grid (vertex (i,j) = j*G + i)."""
    i, j = np.meshgrid(np.arange(G - 1), np.arange(G - 1), indexing="xy")
    i = i.ravel()
    j = j.ravel()
    v00 = j * G + i
    v10 = j * G + i + 1
    v01 = (j + 1) * G + i
    v11 = (j + 1) * G + i + 1
    t0 = np.stack([v00, v10, v11], axis=1)
    t1 = np.stack([v00, v11, v01], axis=1)
    T = np.empty((2 * t0.shape[0], 3), dtype=np.int32)
    T[0::2] = t0
    T[1::2] = t1
    return T


def heightfield(G: int, rng: np.random.Generator) -> Mesh:
    """Sinusoid terrain on [0,1]^2 with N(0, 0.01) vertex noise."""
    theta = rng.uniform(0.0, TWO_PI, 3)
    phi = rng.uniform(0.0, TWO_PI, 3)
    noise = rng.normal(0.0, 0.01, G * G)
    xs = np.arange(G, dtype=np.float64) / (G - 1)
    x, y = np.meshgrid(xs, xs, indexing="xy")
    x = x.ravel()
    y = y.ravel()
    z = np.zeros_like(x)
    for k in range(3):
        z += np.sin(TWO_PI * (k + 1) * (math.cos(theta[k]) * x + math.sin(theta[k]) * y) + phi[k])
    z = 0.2 * z + noise
    V = np.stack([x, y, z], axis=1).astype(np.float32)
    return Mesh(V=V, T=grid_triangles(G), kind="heightfield",
                meta={"G": G, "theta": theta, "phi": phi})


def _icosahedron():
    t = (1.0 + math.sqrt(5.0)) / 2.0
    V = np.array([
        [-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
        [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
        [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    T = np.array([
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    return V, T


def icosphere_topology(level: int):
    """Unit icosphere after `level` midpoint subdivisions (float64, int64)."""
    V, T = _icosahedron()
    for _ in range(level):
        nv = V.shape[0]
        e = np.concatenate([T[:, [0, 1]], T[:, [1, 2]], T[:, [2, 0]]], axis=0)
        lo = np.minimum(e[:, 0], e[:, 1])
        hi = np.maximum(e[:, 0], e[:, 1])
        key = lo * nv + hi
        uniq, inv = np.unique(key, return_inverse=True)
        ulo = uniq // nv
        uhi = uniq % nv
        mid = 0.5 * (V[ulo] + V[uhi])
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        V = np.concatenate([V, mid], axis=0)
        nt = T.shape[0]
        m01 = nv + inv[0:nt]
        m12 = nv + inv[nt:2 * nt]
        m20 = nv + inv[2 * nt:3 * nt]
        a, b, c = T[:, 0], T[:, 1], T[:, 2]
        T = np.concatenate([
            np.stack([a, m01, m20], 1),
            np.stack([m01, b, m12], 1),
            np.stack([m20, m12, c], 1),
            np.stack([m01, m12, m20], 1)], axis=0)
    return V, T


def icosphere(level: int, rng: np.random.Generator, amp: float = 0.05,
              sweeps: int = 10) -> Mesh:
    """Closed, radially displaced icosphere (star-shaped about the origin)."""
    U, T = icosphere_topology(level)
    nv = U.shape[0]
    n = rng.normal(0.0, 1.0, nv)
    e = np.concatenate([T[:, [0, 1]], T[:, [1, 2]], T[:, [2, 0]]], axis=0)
    src = np.concatenate([e[:, 0], e[:, 1]])
    dst = np.concatenate([e[:, 1], e[:, 0]])
    # every undirected edge appears twice (once per adjacent triangle)
    deg = np.bincount(dst, minlength=nv).astype(np.float64)
    for _ in range(sweeps):
        nb = np.bincount(dst, weights=n[src], minlength=nv) / deg
        n = 0.5 * n + 0.5 * nb
    r = 1.0 + amp * n
    V = (U * r[:, None]).astype(np.float32)
    return Mesh(V=V, T=T.astype(np.int32), kind="icosphere", meta={"level": level})


# --------------------------------------------------------------------------
# segment recipes
# --------------------------------------------------------------------------
def segments_box(rng, n, lo_a, hi_a, lo_b, hi_b) -> Segments:
    A = rng.uniform(lo_a, hi_a, size=(n, 3)).astype(np.float32)
    B = rng.uniform(lo_b, hi_b, size=(n, 3)).astype(np.float32)
    return Segments(A, B)


def segments_raster(g: int, z0=-1.0, z1=1.0) -> Segments:
    """A g x g raster of vertical segments over [0,1]^2 (pixel centres, row
    by row): the coherent input of an orthographic view, where neighbouring
    segments take nearly the same path through the tree."""
    xs = (np.arange(g, dtype=np.float64) + 0.5) / g
    x, y = np.meshgrid(xs, xs, indexing="xy")
    n = g * g
    A = np.stack([x.ravel(), y.ravel(), np.full(n, z0)], axis=1).astype(np.float32)
    B = np.stack([x.ravel(), y.ravel(), np.full(n, z1)], axis=1).astype(np.float32)
    return Segments(A, B)


def segments_random_direction(rng, n, V: np.ndarray, expand=0.10,
                              len_lo=0.01, len_hi=1.0, chunk=1 << 21) -> Segments:
    """Start uniform in the mesh bbox grown by `expand` of its extent per side,
    direction uniform on the sphere, length log-uniform in [len_lo, len_hi]."""
    lo = V.min(axis=0).astype(np.float64)
    hi = V.max(axis=0).astype(np.float64)
    ext = hi - lo
    lo = lo - expand * ext
    hi = hi + expand * ext
    A = np.empty((n, 3), np.float32)
    B = np.empty((n, 3), np.float32)
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        a = rng.uniform(lo, hi, size=(m, 3))
        d = rng.normal(0.0, 1.0, size=(m, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        L = np.exp(rng.uniform(math.log(len_lo), math.log(len_hi), size=m))
        A[s:s + m] = a
        B[s:s + m] = a + d * L[:, None]
    return Segments(A, B)


# --------------------------------------------------------------------------
# workloads (sizes of the paper's experiments and their extensions)
# --------------------------------------------------------------------------
def workload_small_bool(seed: int = 0, n_seg: int = 10_000):
    """32x32 heightfield (1,922 triangles), 10k segments crossing z=0 band."""
    rng = np.random.default_rng(seed)
    mesh = heightfield(32, rng)
    seg = segments_box(rng, n_seg, [0, 0, -0.5], [1, 1, 0], [0, 0, 0], [1, 1, 0.5])
    return mesh, seg


def workload_paper_bool(seed: int = 1, n_seg: int = 10_000_000, G: int = 123):
    """123x123 heightfield (29,768 triangles), 10M random-direction segments."""
    rng = np.random.default_rng(seed)
    mesh = heightfield(G, rng)
    seg = segments_random_direction(rng, n_seg, mesh.V)
    return mesh, seg


def workload_sphere(seed: int = 2, n_seg: int = 1_000_000, level: int = 8):
    """Level-8 icosphere (1,310,720 triangles), 1M segments in a cube of side 3."""
    rng = np.random.default_rng(seed)
    mesh = icosphere(level, rng)
    seg = segments_box(rng, n_seg, [-1.5] * 3, [1.5] * 3, [-1.5] * 3, [1.5] * 3)
    return mesh, seg


def workload_diff(seed: int = 3, n_seg: int = 262_144, G: int = 257):
    """257x257 heightfield (131,072 triangles), near-vertical segments and
    loss weights w ~ N(0, I3) for loss = sum_i w_i . P_i."""
    rng = np.random.default_rng(seed)
    mesh = heightfield(G, rng)
    xy = rng.uniform(0.02, 0.98, size=(n_seg, 2))
    dxy = rng.normal(0.0, 0.02, size=(n_seg, 2))
    A = np.concatenate([xy, -np.ones((n_seg, 1))], axis=1).astype(np.float32)
    B = np.concatenate([xy + dxy, np.ones((n_seg, 1))], axis=1).astype(np.float32)
    w = rng.normal(0.0, 1.0, size=(n_seg, 3)).astype(np.float32)
    return mesh, Segments(A, B), w


def workload_raster(seed: int = 1, g: int = 3163, G: int = 123):
    """The paper-scale heightfield (seed 1, 29,768 triangles) under a
    3163 x 3163 raster of vertical segments (10,004,569, row by row)."""
    rng = np.random.default_rng(seed)
    mesh = heightfield(G, rng)
    return mesh, segments_raster(g)


ICO_LEVELS = (3, 4, 5, 6)  # 1,280 / 5,120 / 20,480 / 81,920 triangles


def workload_batched(seed: int = 4, n_mesh: int = 64, nt_lo=1e3, nt_hi=2e5,
                     nr_lo=1e4, nr_hi=2e6, scale: float = 1.0):
    """64 independent meshes of log-uniform size, each with its own segments.

    Even items are heightfields (grid size from N_t), odd items icospheres at the
    subdivision level nearest (in log) to N_t.  Modes alternate bool / nearest.
    `scale` shrinks segment counts (tests use a small scale)."""
    rng = np.random.default_rng(seed)
    items = []
    for m in range(n_mesh):
        nt = math.exp(rng.uniform(math.log(nt_lo), math.log(nt_hi)))
        nr = int(math.exp(rng.uniform(math.log(nr_lo), math.log(nr_hi))) * scale)
        nr = max(nr, 1)
        if m % 2 == 0:
            G = max(2, int(round(math.sqrt(nt / 2.0))) + 1)
            mesh = heightfield(G, rng)
            seg = segments_random_direction(rng, nr, mesh.V)
        else:
            lev = min(ICO_LEVELS, key=lambda L: abs(math.log(20 * 4 ** L) - math.log(nt)))
            mesh = icosphere(lev, rng)
            seg = segments_box(rng, nr, [-1.5] * 3, [1.5] * 3, [-1.5] * 3, [1.5] * 3)
        mode = "bool" if m % 2 == 0 else "nearest"
        items.append((mesh, seg, mode))
    return items


def random_soup(rng: np.random.Generator, n_tri: int, n_seg: int, scale=1.0):
    """Unstructured triangle soup in the unit cube plus random segments
    (tiny brute-force cases)."""
    V = rng.uniform(0, scale, size=(3 * n_tri, 3)).astype(np.float32)
    T = np.arange(3 * n_tri, dtype=np.int32).reshape(n_tri, 3)
    A = rng.uniform(-0.2 * scale, 1.2 * scale, size=(n_seg, 3)).astype(np.float32)
    B = rng.uniform(-0.2 * scale, 1.2 * scale, size=(n_seg, 3)).astype(np.float32)
    return Mesh(V=V, T=T, kind="soup"), Segments(A, B)
