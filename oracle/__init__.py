"""FP64 CPU oracle for segment / triangle-mesh intersection (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: imported by the test-suite, by the smoke check in
``__graft_entry__`` and by the CPU-baseline leg of ``bench.py``.  The product
package never imports it and shares no code with it.

The arithmetic lives in ``rsi_oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off``); this module only compiles it, marshals numpy arrays and
returns numpy results.  Each function names the passage of the paper it
follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rsi_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None


def compile_oracle(force: bool = False) -> str:
    """Compile rsi_oracle.c into liborc.so next to it (gcc, OpenMP if present)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
            "-std=c11", "-o", _LIB_PATH + ".tmp", _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def _bind(lib):
    """Set the ctypes prototypes of the oracle's entry points on `lib`."""
    P = C.c_void_p
    L = C.c_long
    lib.orc_brute.argtypes = [P, L, P, L, P, P, L, C.c_int] + [P] * 7
    lib.orc_brute.restype = C.c_int
    lib.orc_bvh_build.argtypes = [P, L, P, L, C.c_double]
    lib.orc_bvh_build.restype = P
    lib.orc_bvh_free.argtypes = [P]
    lib.orc_bvh_nodes.argtypes = [P]
    lib.orc_bvh_nodes.restype = L
    lib.orc_bvh_query.argtypes = [P, P, L, P, P, P, L, C.c_int] + [P] * 7
    lib.orc_bvh_query.restype = C.c_int
    lib.orc_backward.argtypes = [P, L, P, L, P, P, L, P, P, P, P, P, P]
    lib.orc_backward.restype = C.c_int
    lib.orc_eval_fixed.argtypes = [P, L, P, P, P, L, P, P]
    lib.orc_eval_fixed.restype = C.c_int
    lib.orc_lbvh.argtypes = [P, L, P, L] + [P] * 8
    lib.orc_lbvh.restype = C.c_int
    lib.orc_mt.argtypes = [P] * 6
    lib.orc_morton3.argtypes = [C.c_uint32] * 3
    lib.orc_morton3.restype = C.c_uint32
    lib.orc_morton2.argtypes = [C.c_uint32] * 2
    lib.orc_morton2.restype = C.c_uint32
    lib.orc_lbvh_h.argtypes = [P, L, P, L, C.c_int] + [P] * 8
    lib.orc_lbvh_h.restype = C.c_int
    lib.orc_num_threads.restype = C.c_int
    return lib


def _get():
    global _lib
    with _lock:
        if _lib is None:
            compile_oracle()
            _lib = _bind(C.CDLL(_LIB_PATH))
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def num_threads() -> int:
    return int(_get().orc_num_threads())


def mt(a, b, v0, v1, v2):
    """One Moller-Trumbore test (Sec. 2), FP64 from float inputs.
    Returns (hit, det, nU, nV, nT), sign-normalised."""
    out = np.zeros(5, np.float64)
    args = [_f32(x) for x in (a, b, v0, v1, v2)]
    _get().orc_mt(*[_p(x) for x in args], _p(out))
    return bool(out[0]), out[1], out[2], out[3], out[4]


def morton3(x: int, y: int, z: int) -> int:
    """30-bit Morton interleave (Sec. 2: bit-wise interleaving of q_j)."""
    return int(_get().orc_morton3(x, y, z))


def morton2(x: int, y: int) -> int:
    """30-bit interleave of two 15-bit coordinates, the first one high: the
    height-field variant of the code (a library option, not the paper's)."""
    return int(_get().orc_morton2(x, y))


def _alloc_outputs(nR):
    return dict(
        flag=np.zeros(nR, np.uint8), count=np.zeros(nR, np.int32),
        tri=np.zeros(nR, np.int32), tuv=np.zeros((nR, 3), np.float64),
        point=np.zeros((nR, 3), np.float64), dist=np.zeros(nR, np.float64),
        neardeg=np.zeros(nR, np.uint8))


def brute(V, T, A, B, threads: int = 0) -> dict:
    """All N_t x N_r Moller-Trumbore tests (Sec. 1 problem, Sec. 2 test);
    returns flag / count / nearest (tri, tuv, point, dist) / neardeg."""
    V, T, A, B = _f32(V), _i32(T), _f32(A), _f32(B)
    nR = A.shape[0]
    o = _alloc_outputs(nR)
    rc = _get().orc_brute(_p(V), V.shape[0], _p(T), T.shape[0], _p(A), _p(B), nR,
                          threads, _p(o["flag"]), _p(o["count"]), _p(o["tri"]),
                          _p(o["tuv"]), _p(o["point"]), _p(o["dist"]),
                          _p(o["neardeg"]))
    if rc:
        raise ValueError("oracle: triangle index out of range")
    return o


class CpuBVH:
    """Median-split CPU BVH; a candidate filter in front of the same FP64 test."""

    def __init__(self, V, T, margin: float | None = None):
        self.V, self.T = _f32(V), _i32(T)
        if margin is None:
            ext = float(np.max(self.V.max(0) - self.V.min(0))) if self.V.size else 1.0
            margin = 1e-5 * max(ext, 1e-30)
        self._h = _get().orc_bvh_build(_p(self.V), self.V.shape[0], _p(self.T),
                                       self.T.shape[0], float(margin))

    def __del__(self):
        try:
            if self._h:
                _get().orc_bvh_free(self._h)
                self._h = None
        except Exception:
            pass

    def query(self, A, B, threads: int = 0) -> dict:
        A, B = _f32(A), _f32(B)
        nR = A.shape[0]
        o = _alloc_outputs(nR)
        rc = _get().orc_bvh_query(self._h, _p(self.V), self.V.shape[0], _p(self.T),
                                  _p(A), _p(B), nR, threads, _p(o["flag"]),
                                  _p(o["count"]), _p(o["tri"]), _p(o["tuv"]),
                                  _p(o["point"]), _p(o["dist"]), _p(o["neardeg"]))
        if rc:
            raise ValueError("oracle: triangle index out of range")
        return o


def intersect(V, T, A, B, threads: int = 0, brute_limit: float = 2e8) -> dict:
    """Brute force when N_t*N_r is small, the CPU BVH otherwise."""
    if T.shape[0] * A.shape[0] <= brute_limit:
        return brute(V, T, A, B, threads)
    return CpuBVH(V, T).query(A, B, threads)


def backward(V, T, A, B, tri, gP=None, gtuv=None):
    """FP64 adjoint of the nearest hit with the triangle held fixed.
    Returns (gV, gA, gB) as float64 arrays."""
    V, T, A, B, tri = _f32(V), _i32(T), _f32(A), _f32(B), _i32(tri)
    nR = A.shape[0]
    gP = None if gP is None else np.ascontiguousarray(gP, np.float64)
    gtuv = None if gtuv is None else np.ascontiguousarray(gtuv, np.float64)
    gV = np.zeros_like(V, dtype=np.float64)
    gA = np.zeros((nR, 3), np.float64)
    gB = np.zeros((nR, 3), np.float64)
    rc = _get().orc_backward(_p(V), V.shape[0], _p(T), T.shape[0], _p(A), _p(B), nR,
                             _p(tri), _p(gP), _p(gtuv), _p(gV), _p(gA), _p(gB))
    if rc:
        raise ValueError("oracle: index out of range")
    return gV, gA, gB


def eval_fixed(V64, T, A64, B64, tri):
    """(t, u, v, P) for a fixed triangle per segment, FP64 inputs (for finite
    differences).  Returns float64 [N_r, 6]."""
    V64 = np.ascontiguousarray(V64, np.float64)
    A64 = np.ascontiguousarray(A64, np.float64)
    B64 = np.ascontiguousarray(B64, np.float64)
    T, tri = _i32(T), _i32(tri)
    out = np.zeros((A64.shape[0], 6), np.float64)
    rc = _get().orc_eval_fixed(_p(V64), V64.shape[0], _p(T), _p(A64), _p(B64),
                               A64.shape[0], _p(tri), _p(out))
    if rc:
        raise ValueError("oracle: index out of range")
    return out


def lbvh(V, T, height_axis: int = 0) -> dict:
    """LBVH build by its plain definition (Sec. 2: centroids, support interval,
    quantisation, Morton codes, sort, radix tree, boxes).  height_axis 1, 2
    or 3: the library's height-field option (that coordinate left out of the
    code, the other two quantised to 15 bits each); 0: the paper's code."""
    V, T = _f32(V), _i32(T)
    n = T.shape[0]
    o = dict(bounds=np.zeros(6, np.float32), codes=np.zeros(n, np.uint32),
             order=np.zeros(n, np.uint32), left=np.zeros(max(n - 1, 0), np.int32),
             right=np.zeros(max(n - 1, 0), np.int32),
             range=np.zeros((max(n - 1, 0), 2), np.int32),
             nbox=np.zeros((max(n - 1, 0), 6), np.float32),
             lbox=np.zeros((n, 6), np.float32))
    rc = _get().orc_lbvh_h(_p(V), V.shape[0], _p(T), n, int(height_axis), _p(o["bounds"]),
                           _p(o["codes"]), _p(o["order"]), _p(o["left"]), _p(o["right"]),
                           _p(o["range"]), _p(o["nbox"]), _p(o["lbox"]))
    if rc == 2:
        raise ValueError("oracle: height_axis must be 0, 1, 2 or 3")
    if rc:
        raise ValueError("oracle: triangle index out of range")
    return o
