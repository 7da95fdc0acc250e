"""GB300 line-segment / triangle-mesh intersection (arXiv 2209.02878).

Thin Python binding over the C ABI of ``librsi.so`` (include/rsi.h).  PyTorch
supplies device memory and streams; every step of the computation runs in the
library's CUDA kernels.  The binding fails loudly if the library is missing:
there is no CPU path.

Modes (Sec. 1 and Sec. 2.4 of the paper): ``"bool"`` crossing flag,
``"count"`` number of crossings (``intercept_count``), ``"nearest"`` nearest
crossing with triangle id, (t, u, v), point and distance (``barycentric``).
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _abi
from ._abi import MODES, RSIError

__all__ = ["BVH", "Batch", "intersect", "intersect_backward", "nearest_hit", "RSIFunction",
           "RSIError", "MODES", "load_library", "library_version", "fp32_peak",
           "set_allocator", "use_torch_allocator"]


def load_library():
    return _abi.load()


def library_version() -> str:
    return _abi.load().rsi_version().decode()


def fp32_peak(iters: int = 1 << 16, stream=None) -> float:
    """Measured FP32 rate of the current device in TFLOP/s (rsi_fp32_peak:
    an FMA-only kernel over every SM, event-timed).  Synchronises."""
    v = C.c_double(0.0)
    _abi.check(_abi.load().rsi_fp32_peak(int(iters), C.byref(v), _stream(stream)),
               "rsi_fp32_peak")
    return v.value


_keep = []  # every ctypes callback pair ever set (handles may still free through one)


def set_allocator(alloc=None, free=None):
    """Route the library's device allocations through Python callables
    (rsi_set_allocator): alloc(nbytes, device, stream) -> int pointer (0 when
    it cannot), free(ptr, device, stream).  Streams are raw cudaStream_t
    values (0 = the legacy default stream).  Both None restores
    cudaMallocAsync / cudaFreeAsync.  Handles keep the allocator that was set
    when they were created."""
    lib = _abi.load()
    if alloc is None and free is None:
        _abi.check(lib.rsi_set_allocator(None, None, None), "rsi_set_allocator")
        return
    if alloc is None or free is None:
        raise ValueError("set both alloc and free, or neither")

    def _a(nbytes, device, stream, ctx):
        return int(alloc(int(nbytes), int(device), int(stream or 0)) or 0) or None

    def _f(p, device, stream, ctx):
        free(int(p), int(device), int(stream or 0))

    ca, cf = _abi.ALLOC_FN(_a), _abi.FREE_FN(_f)
    _abi.check(lib.rsi_set_allocator(C.cast(ca, C.c_void_p), C.cast(cf, C.c_void_p), None),
               "rsi_set_allocator")
    # handles created under these callbacks free through them later: keep
    # every pair alive for the life of the process
    _keep.append((ca, cf))


def use_torch_allocator(enable: bool = True):
    """Take the library's device memory from PyTorch's caching allocator
    (it then shows in torch.cuda.memory_allocated and can be reused by
    torch), or go back to cudaMallocAsync."""
    if not enable:
        set_allocator(None, None)
        return

    def alloc(nbytes, device, stream):
        try:
            return torch.cuda.caching_allocator_alloc(nbytes, device=device, stream=stream)
        except RuntimeError:
            return 0

    def free(p, device, stream):
        torch.cuda.caching_allocator_delete(p)

    set_allocator(alloc, free)


def _vp(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _check_tensor(t, name, dtype, cols=3):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (no CPU path)")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if cols and (t.dim() != 2 or t.shape[1] != cols):
        raise ValueError(f"{name} must have shape [n, {cols}], got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _mode(mode) -> int:
    if isinstance(mode, int):
        return mode
    try:
        return MODES[mode]
    except KeyError:
        raise ValueError(f"unknown mode {mode!r}; use one of {sorted(MODES)}") from None


def _launch(launch, n=None, device=None):
    """rsi_launch_opts from a dict; "order" is an int32 CUDA tensor of n
    entries (a processing order, e.g. from BVH.segment_order)."""
    lo = _abi.rsi_launch_opts()
    if launch:
        for k, v in launch.items():
            if k == "order":
                if v is None:
                    continue
                _check_tensor(v, "order", torch.int32, cols=0)
                if v.dim() != 1 or (n is not None and v.shape[0] != n):
                    raise ValueError("order must be a 1-D int32 tensor with one entry per segment")
                if device is not None and v.device != device:
                    raise ValueError("order must be on the segments' device")
                lo.order = v.data_ptr()
            else:
                setattr(lo, k, int(v))
    return lo


def _alloc_outputs(mode: int, n: int, dev, compact: bool, hit_cap):
    o = {}
    if mode == _abi.RSI_MODE_BOOL:
        o["flag"] = torch.empty(n, dtype=torch.uint8, device=dev)
    elif mode == _abi.RSI_MODE_COUNT:
        o["count"] = torch.empty(n, dtype=torch.int32, device=dev)
    else:
        o["tri"] = torch.empty(n, dtype=torch.int32, device=dev)
        o["tuv"] = torch.empty((n, 3), dtype=torch.float32, device=dev)
        o["point"] = torch.empty((n, 3), dtype=torch.float32, device=dev)
        o["dist"] = torch.empty(n, dtype=torch.float32, device=dev)
    if compact and mode != _abi.RSI_MODE_BOOL:
        cap = n if hit_cap is None else int(hit_cap)
        o["hit_idx"] = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
        o["n_hits"] = torch.zeros(1, dtype=torch.int64, device=dev)
        o["hit_cap"] = cap
        if mode == _abi.RSI_MODE_COUNT:
            o["hit_count"] = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
        else:
            o["hit_tri"] = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
            o["hit_dist"] = torch.empty(max(cap, 1), dtype=torch.float32, device=dev)
            o["hit_point"] = torch.empty((max(cap, 1), 3), dtype=torch.float32, device=dev)
    return o


def _rsi_output(o) -> _abi.rsi_output:
    r = _abi.rsi_output()
    for k in ("flag", "count", "tri", "tuv", "point", "dist", "hit_idx", "n_hits", "hit_tri",
              "hit_dist", "hit_point", "hit_count"):
        if k in o and o[k] is not None:
            setattr(r, k, o[k].data_ptr())
    r.hit_cap = int(o.get("hit_cap", 0))
    return r


class BVH:
    """LBVH of one indexed triangle mesh on the current CUDA device
    (rsi_bvh_create + rsi_bvh_build).  V: float32 [nV,3], T: int32 [nT,3].
    height_axis: 0 for the paper's Morton code over x, y, z; 1, 2 or 3 for a
    mesh that is a height field along that axis (a terrain z = f(x, y): 3),
    whose code then leaves that coordinate out (same results, a tree better
    suited to the surface)."""

    def __init__(self, V, T, leaf_size: int = 0, top_levels: int = 0, stream=None,
                 height_axis: int = 0):
        self._lib = _abi.load()
        _check_tensor(V, "V", torch.float32)
        _check_tensor(T, "T", torch.int32)
        self.nV, self.nT = int(V.shape[0]), int(T.shape[0])
        self.device = V.device
        self.leaf_size, self.top_levels, self.height_axis = leaf_size, top_levels, height_axis
        opts = _abi.rsi_build_opts(int(leaf_size), int(top_levels), int(height_axis))
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            _abi.check(self._lib.rsi_bvh_create(self.nV, self.nT, C.byref(opts), _stream(stream),
                                                C.byref(h)), "rsi_bvh_create")
        self._h = h
        self.T = T
        self.refits = 0
        self._vkey = None
        self.build(V, T, stream)

    @staticmethod
    def _key(V):
        # storage, in-place version and shape of the vertices the tree holds:
        # an optimizer step on V (in place) bumps the version, a new tensor
        # has another storage
        return (V.data_ptr(), V._version, tuple(V.shape))

    def build(self, V, T=None, stream=None):
        """Rebuild from vertices V (and triangles T, same sizes)."""
        T = self.T if T is None else T
        _check_tensor(V, "V", torch.float32)
        _check_tensor(T, "T", torch.int32)
        if V.shape[0] != self.nV or T.shape[0] != self.nT:
            raise ValueError("build: sizes differ from the handle's")
        with torch.cuda.device(self.device):
            _abi.check(self._lib.rsi_bvh_build(self._h, _vp(V), _vp(T), _stream(stream)),
                       "rsi_bvh_build")
        self.T = T
        self._tkey = T._version
        self._vkey = self._key(V)
        return self

    def refit(self, V, stream=None):
        """Refit the boxes to moved vertices (same triangles as the last build)."""
        _check_tensor(V, "V", torch.float32)
        if V.shape[0] != self.nV:
            raise ValueError("refit: vertex count differs from the handle's")
        with torch.cuda.device(self.device):
            _abi.check(self._lib.rsi_refit(self._h, _vp(V), _vp(self.T), _stream(stream)),
                       "rsi_refit")
        self._vkey = self._key(V)
        self.refits += 1
        return self

    def sync(self, V, T=None, stream=None):
        """Make the tree describe vertices V (and triangles T): a rebuild when
        T is not the tensor the tree was built from, a refit (the bottom-up
        box pass, Sec. 2) when V is another tensor or was changed in place
        since the last build or refit, nothing otherwise."""
        if T is not None and (T.data_ptr() != self.T.data_ptr() or T.shape != self.T.shape
                              or T._version != self._tkey):
            return self.build(V, T, stream)
        if self._key(V) != self._vkey:
            self.refit(V, stream)
        return self

    def status(self, stream=None) -> int:
        """Synchronise and return (then clear) the device-side status word."""
        with torch.cuda.device(self.device):
            return int(self._lib.rsi_bvh_status(self._h, _stream(stream)))

    def info(self) -> dict:
        i = _abi.rsi_bvh_info()
        _abi.check(self._lib.rsi_bvh_get_info(self._h, C.byref(i)), "rsi_bvh_get_info")
        return {k: getattr(i, k) for k, _ in i._fields_}

    def intersect(self, A, B, mode="bool", *, compact=False, hit_cap=None, launch=None,
                  stats=False, stream=None, out=None):
        """Test segments A[i] -> B[i] (float32 [nR,3], CUDA) against the mesh.
        Returns a dict of output tensors (see rsi_output in include/rsi.h);
        with stats=True also a dict of traversal counters (synchronises)."""
        _check_tensor(A, "A", torch.float32)
        _check_tensor(B, "B", torch.float32)
        if A.shape != B.shape:
            raise ValueError("A and B must have the same shape")
        m = _mode(mode)
        n = int(A.shape[0])
        o = out if out is not None else _alloc_outputs(m, n, A.device, compact, hit_cap)
        ro = _rsi_output(o)
        lo = _launch(launch, n, A.device)
        with torch.cuda.device(self.device):
            if stats:
                st = _abi.rsi_stats()
                _abi.check(self._lib.rsi_intersect_stats(self._h, _vp(A), _vp(B), n, m,
                                                         C.byref(ro), C.byref(lo),
                                                         _stream(stream), C.byref(st)),
                           "rsi_intersect_stats")
                o["stats"] = {k: getattr(st, k) for k, _ in st._fields_}
            else:
                _abi.check(self._lib.rsi_intersect(self._h, _vp(A), _vp(B), n, m, C.byref(ro),
                                                   C.byref(lo), _stream(stream)),
                           "rsi_intersect")
        return o

    def segment_order(self, A, B, bits=0, stream=None):
        """Coherent processing order of the segments A[i] -> B[i] (float32
        [nR,3], CUDA) with rsi_segment_order: an int32 permutation to pass as
        launch={"order": ...} to later intersect calls on the same segments
        (bits 6..30, 0 -> 30)."""
        _check_tensor(A, "A", torch.float32)
        _check_tensor(B, "B", torch.float32)
        if A.shape != B.shape:
            raise ValueError("A and B must have the same shape")
        n = int(A.shape[0])
        order = torch.empty(n, dtype=torch.int32, device=A.device)
        with torch.cuda.device(self.device):
            _abi.check(self._lib.rsi_segment_order(self._h, _vp(A), _vp(B), n, int(bits),
                                                   _vp(order), _stream(stream)),
                       "rsi_segment_order")
        return order

    def intersect_host(self, A, B, mode="bool", *, out=None, chunk=0, launch=None,
                       stream=None):
        """Test segments held in HOST memory (float32 [nR,3] CPU tensors) with
        rsi_intersect_host: pinned inputs are streamed to the device under
        one running traversal (BOOL) or read in place by the kernel (COUNT,
        NEAREST); pageable ones go through chunked copies.  `chunk` sets the
        copy / launch chunk in segments (0: the library's choice).  Returns a
        dict of host output tensors (pinned when allocated here), complete
        once `stream` (default current) is synchronised; A and B must stay
        unchanged until then.  The streamed BOOL copies start without
        waiting for `stream` (they overlap the work already queued there),
        so pinned A and B must hold their data when this is called."""
        for t, nme in ((A, "A"), (B, "B")):
            if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != torch.float32 or \
                    t.dim() != 2 or t.shape[1] != 3 or not t.is_contiguous():
                raise ValueError(f"{nme} must be a contiguous float32 [n,3] CPU tensor")
        m = _mode(mode)
        n = int(A.shape[0])
        if out is None:
            pin = torch.cuda.is_available()
            if m == _abi.RSI_MODE_BOOL:
                out = {"flag": torch.empty(n, dtype=torch.uint8, pin_memory=pin)}
            elif m == _abi.RSI_MODE_COUNT:
                out = {"count": torch.empty(n, dtype=torch.int32, pin_memory=pin)}
            else:
                out = {"tri": torch.empty(n, dtype=torch.int32, pin_memory=pin),
                       "tuv": torch.empty((n, 3), dtype=torch.float32, pin_memory=pin),
                       "point": torch.empty((n, 3), dtype=torch.float32, pin_memory=pin),
                       "dist": torch.empty(n, dtype=torch.float32, pin_memory=pin)}
        ro = _rsi_output(out)
        lo = _launch(launch)
        with torch.cuda.device(self.device):
            _abi.check(self._lib.rsi_intersect_host(self._h, _vp(A), _vp(B), n, m, C.byref(ro),
                                                    int(chunk), C.byref(lo), _stream(stream)),
                       "rsi_intersect_host")
        return out

    def points_inside(self, P, *, launch=None, stream=None):
        """Odd-parity inside test of points P (float32 [n,3], CUDA) against
        a closed mesh (rsi_points_inside); returns uint8 [n] (1 = inside)."""
        _check_tensor(P, "P", torch.float32)
        out = torch.empty(int(P.shape[0]), dtype=torch.uint8, device=P.device)
        lo = _launch(launch)
        with torch.cuda.device(self.device):
            _abi.check(self._lib.rsi_points_inside(self._h, _vp(P), int(P.shape[0]), _vp(out),
                                                   C.byref(lo), _stream(stream)),
                       "rsi_points_inside")
        return out

    def export(self, stream=None) -> dict:
        """Copy the tree to host numpy arrays (synchronises); for validation."""
        n = self.nT
        o = dict(bounds=np.zeros(6, np.float32), codes=np.zeros(n, np.uint32),
                 order=np.zeros(n, np.int32), left=np.zeros(max(n - 1, 0), np.int32),
                 right=np.zeros(max(n - 1, 0), np.int32),
                 range=np.zeros((max(n - 1, 0), 2), np.int32),
                 nbox=np.zeros((max(n - 1, 0), 6), np.float32),
                 lbox=np.zeros((n, 6), np.float32), nodes=np.zeros((max(n, 1), 16), np.float32))
        p = {k: v.ctypes.data_as(C.c_void_p) for k, v in o.items()}
        with torch.cuda.device(self.device):
            _abi.check(self._lib.rsi_bvh_export(self._h, _stream(stream), p["bounds"], p["codes"],
                                                p["order"], p["left"], p["right"], p["range"],
                                                p["nbox"], p["lbox"], p["nodes"]),
                       "rsi_bvh_export")
        o["nodes_i"] = o["nodes"].view(np.int32)
        return o

    def close(self):
        if getattr(self, "_h", None):
            try:
                self._lib.rsi_bvh_destroy(self._h)
            finally:
                self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def intersect(V, T, A, B, mode="bool", **kw):
    """Build a BVH for (V, T) and test the segments (one-shot convenience)."""
    bvh = BVH(V, T, leaf_size=kw.pop("leaf_size", 0), top_levels=kw.pop("top_levels", 0),
              height_axis=kw.pop("height_axis", 0))
    try:
        return bvh.intersect(A, B, mode, **kw)
    finally:
        torch.cuda.current_stream().synchronize()
        bvh.close()


def intersect_backward(V, T, A, B, tri, grad_point=None, grad_tuv=None, grad_V=None,
                       stream=None):
    """Adjoint of the nearest outputs with the triangle held fixed
    (rsi_intersect_backward).  Returns (grad_V, grad_A, grad_B); grad_V is
    accumulated into when given."""
    lib = _abi.load()
    for t, nme in ((V, "V"), (A, "A"), (B, "B")):
        _check_tensor(t, nme, torch.float32)
    _check_tensor(T, "T", torch.int32)
    _check_tensor(tri, "tri", torch.int32, cols=0)
    n = int(A.shape[0])
    if grad_point is not None:
        grad_point = _check_tensor(grad_point.contiguous().float(), "grad_point", torch.float32)
    if grad_tuv is not None:
        grad_tuv = _check_tensor(grad_tuv.contiguous().float(), "grad_tuv", torch.float32)
    gV = grad_V if grad_V is not None else torch.zeros_like(V)
    gA = torch.empty_like(A)
    gB = torch.empty_like(B)
    with torch.cuda.device(V.device):
        _abi.check(lib.rsi_intersect_backward(_vp(V), int(V.shape[0]), _vp(T), int(T.shape[0]),
                                              _vp(A), _vp(B), n, _vp(tri), _vp(grad_point),
                                              _vp(grad_tuv), _vp(gV), _vp(gA), _vp(gB),
                                              _stream(stream)),
                   "rsi_intersect_backward")
    return gV, gA, gB


class RSIFunction(torch.autograd.Function):
    """Nearest crossing as a differentiable function of (V, A, B): returns
    (point [nR,3], tuv [nR,3], tri [nR]); hit/miss and the triangle are held
    fixed in the backward pass (rsi_intersect_backward).  With a `bvh` passed
    the tree is reused across calls and kept current: refit when V is
    another tensor or was changed in place (an optimizer step) since the
    tree last saw it, rebuilt when T is another tensor (BVH.sync).  `order`:
    a processing order of the segments (BVH.segment_order), reused while A
    and B stay the same."""

    @staticmethod
    def forward(ctx, V, A, B, T, bvh, order=None):
        if bvh is None:
            bvh = BVH(V.detach(), T)
        else:
            bvh.sync(V.detach(), T)
        o = bvh.intersect(A.detach(), B.detach(), "nearest",
                          launch={"order": order} if order is not None else None)
        ctx.save_for_backward(V.detach(), A.detach(), B.detach(), T, o["tri"])
        ctx.mark_non_differentiable(o["tri"])
        return o["point"], o["tuv"], o["tri"]

    @staticmethod
    def backward(ctx, g_point, g_tuv, g_tri):
        V, A, B, T, tri = ctx.saved_tensors
        gV, gA, gB = intersect_backward(V, T, A, B, tri, g_point, g_tuv)
        return (gV if ctx.needs_input_grad[0] else None,
                gA if ctx.needs_input_grad[1] else None,
                gB if ctx.needs_input_grad[2] else None, None, None, None)


def nearest_hit(V, T, A, B, bvh=None, order=None):
    """Differentiable nearest crossing: (point, tuv, tri).  Pass a BVH of
    (V, T) to reuse it across steps: it is refit whenever V has moved.  Pass
    order=bvh.segment_order(A, B) to traverse fixed segments in a coherent
    order computed once."""
    return RSIFunction.apply(V, A, B, T, bvh, order)


class Batch:
    """Many independent (mesh, segments, mode) problems: one multi-mesh build
    and one persistent traversal launch, optionally replayed as a CUDA graph
    (rsi_batch_create / _build / _intersect / _run_graph).  Items are
    (V, T, A, B, mode) or (V, T, A, B, mode, height_axis); height_axis as for
    BVH, per item, or for every item without its own."""

    def __init__(self, items, leaf_size=0, launch=None, compact=False, stream=None,
                 height_axis=0):
        self._lib = _abi.load()
        self.items = []
        self.outputs = []
        arr = (_abi.rsi_batch_item * len(items))()
        for k, item in enumerate(items):
            V, T, A, B, mode = item[:5]
            item_axis = int(item[5]) if len(item) > 5 else 0
            _check_tensor(V, "V", torch.float32)
            _check_tensor(T, "T", torch.int32)
            _check_tensor(A, "A", torch.float32)
            _check_tensor(B, "B", torch.float32)
            m = _mode(mode)
            o = _alloc_outputs(m, int(A.shape[0]), A.device, compact, None)
            self.outputs.append(o)
            self.items.append((V, T, A, B, m))
            it = arr[k]
            it.dV, it.nV, it.dT, it.nT = V.data_ptr(), V.shape[0], T.data_ptr(), T.shape[0]
            it.dA, it.dB, it.nR, it.mode = A.data_ptr(), B.data_ptr(), A.shape[0], m
            it.height_axis = item_axis
            it.out = _rsi_output(o)
        self._arr = arr
        bo = _abi.rsi_build_opts(int(leaf_size), 0, int(height_axis))
        lo = _launch(launch)
        h = C.c_void_p()
        _abi.check(self._lib.rsi_batch_create(arr, len(items), C.byref(bo), C.byref(lo),
                                              _stream(stream), C.byref(h)), "rsi_batch_create")
        self._h = h

    def build(self, stream=None):
        _abi.check(self._lib.rsi_batch_build(self._h, _stream(stream)), "rsi_batch_build")
        return self

    def intersect(self, stream=None):
        _abi.check(self._lib.rsi_batch_intersect(self._h, _stream(stream)),
                   "rsi_batch_intersect")
        return self.outputs

    def run_graph(self, rebuild=True, stream=None):
        _abi.check(self._lib.rsi_batch_run_graph(self._h, int(bool(rebuild)), _stream(stream)),
                   "rsi_batch_run_graph")
        return self.outputs

    def status(self, stream=None) -> int:
        """Synchronise and return (then clear) the batch's device-side status."""
        return int(self._lib.rsi_batch_status(self._h, _stream(stream)))

    def close(self):
        if getattr(self, "_h", None):
            try:
                self._lib.rsi_batch_destroy(self._h)
            finally:
                self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
