"""rsi_intersect_backward_static, the allocation-free adjoint, called through
the C ABI: two calls in a row must give what rsi_intersect_backward gives
(same FP64 accumulation, so within the gradient tolerance of the other GPU
tests), and an oversized mesh must be rejected.

The entry point exists for callers that may not allocate device memory while
they run (fixed memory budgets, graph capture into a pool they do not own,
allocator callbacks); it keeps its accumulator in a fixed array inside the
library.  With counting allocator hooks installed, the two calls must make
no allocation through the library's allocator (the allocating variant, the
control, does).  This file sorts last so that a run stopping at the first
failure has already run every other test; it also passes on its own."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2209_02878_gb300 import _abi, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _case():
    rng = np.random.default_rng(21)
    mesh = synth.heightfield(65, rng)          # 4,225 vertices, 8,192 triangles
    n = 20000
    xy = rng.uniform(0.02, 0.98, size=(n, 2))
    dxy = rng.normal(0.0, 0.02, size=(n, 2))
    A = np.c_[xy, -np.ones(n)].astype(np.float32)
    B = np.c_[xy + dxy, np.ones(n)].astype(np.float32)
    w = rng.normal(size=(n, 3)).astype(np.float32)
    wt = rng.normal(size=(n, 3)).astype(np.float32)
    return [torch.from_numpy(x).to(DEV) for x in (mesh.V, mesh.T, A, B, w, wt)]


def _backward(lib, fn, V, T, A, B, tri, w, wt):
    gV = torch.zeros_like(V)
    gA = torch.empty_like(A)
    gB = torch.empty_like(B)
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = getattr(lib, fn)(_p(V), V.shape[0], _p(T), T.shape[0], _p(A), _p(B), A.shape[0],
                          _p(tri), _p(w), _p(wt), _p(gV), _p(gA), _p(gB), s)
    assert rc == _abi.RSI_OK, (fn, rc)
    torch.cuda.synchronize()
    return [x.cpu().numpy().astype(np.float64) for x in (gV, gA, gB)]


def test_static_backward_matches_allocating_backward_twice():
    import paper_2209_02878_gb300 as rsi
    lib = _abi.load()
    V, T, A, B, w, wt = _case()
    tri = rsi.BVH(V, T).intersect(A, B, "nearest")["tri"]
    torch.cuda.synchronize()
    assert (tri >= 0).float().mean() > 0.9
    ref = _backward(lib, "rsi_intersect_backward", V, T, A, B, tri, w, wt)
    for call in range(2):
        got = _backward(lib, "rsi_intersect_backward_static", V, T, A, B, tri, w, wt)
        for g, r, name in zip(got, ref, ("gV", "gA", "gB")):
            rel = np.linalg.norm(g - r) / max(np.linalg.norm(r), 1e-30)
            assert rel <= 1e-5, (call, name, rel)
            scale = np.maximum(np.abs(r), 1e-3 * np.abs(r).max())
            assert np.all(np.abs(g - r) <= 1e-5 * scale), (call, name)


def test_static_backward_rejects_oversized_mesh():
    lib = _abi.load()
    n = _abi.RSI_STATIC_MAX_VERTICES + 1
    V = torch.zeros((n, 3), dtype=torch.float32, device=DEV)
    T = torch.zeros((1, 3), dtype=torch.int32, device=DEV)
    A = torch.zeros((4, 3), dtype=torch.float32, device=DEV)
    tri = torch.full((4,), -1, dtype=torch.int32, device=DEV)
    g = torch.zeros_like(V)
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.rsi_intersect_backward_static(_p(V), n, _p(T), 1, _p(A), _p(A), 4, _p(tri), None,
                                           None, _p(g), None, None, s)
    assert rc == _abi.RSI_ERR_CAPACITY


def test_static_backward_allocates_nothing():
    """Counting hooks on the library's allocator (rsi_set_allocator): after
    one warm-up call (which looks up the array, and under lazy loading loads
    its module), two static calls make no allocation or free; the allocating
    entry point, as a control, makes one of each."""
    import paper_2209_02878_gb300 as rsi
    lib = _abi.load()
    V, T, A, B, w, wt = _case()
    tri = rsi.BVH(V, T).intersect(A, B, "nearest")["tri"]
    torch.cuda.synchronize()
    _backward(lib, "rsi_intersect_backward_static", V, T, A, B, tri, w, wt)
    calls = {"alloc": 0, "free": 0}
    live = {}

    def alloc(nbytes, device, stream):
        calls["alloc"] += 1
        p = torch.cuda.caching_allocator_alloc(nbytes, device=device, stream=stream)
        live[p] = True
        return p

    def free(p, device, stream):
        calls["free"] += 1
        live.pop(p)
        torch.cuda.caching_allocator_delete(p)

    rsi.set_allocator(alloc, free)
    try:
        for _ in range(2):
            _backward(lib, "rsi_intersect_backward_static", V, T, A, B, tri, w, wt)
        assert calls == {"alloc": 0, "free": 0}, calls
        _backward(lib, "rsi_intersect_backward", V, T, A, B, tri, w, wt)
        assert calls == {"alloc": 1, "free": 1}, calls
    finally:
        rsi.set_allocator(None, None)
