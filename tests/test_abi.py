"""The C ABI library: it builds for sm_103a, loads, and exports every entry
point include/rsi.h declares; the binding refuses CPU tensors.  CPU only (no
compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rsi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rsi_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2209_02878_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = _declared()
    for n in ("rsi_build_bvh", "rsi_intersect", "rsi_intersect_backward", "rsi_batch_create",
              "rsi_refit", "rsi_bvh_destroy", "rsi_status_string", "rsi_autotune"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_prototypes_cover_header():
    from paper_2209_02878_gb300 import _abi
    assert sorted(_abi.EXPORTS) == _declared()


def test_status_strings_without_gpu(lib):
    lib.rsi_status_string.restype = ctypes.c_char_p
    lib.rsi_status_string.argtypes = [ctypes.c_int]
    assert lib.rsi_status_string(0) == b"ok"
    assert lib.rsi_status_string(4) == b"triangle index out of range"
    lib.rsi_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.rsi_version()


def test_library_is_built_for_sm_103a(lib):
    from paper_2209_02878_gb300 import _build
    assert "arch=compute_103a,code=sm_103a" in _build.ARCH


def test_missing_library_fails_loudly(tmp_path):
    from paper_2209_02878_gb300 import _abi
    saved = _abi._lib
    _abi._lib = None
    try:
        with pytest.raises(RuntimeError, match="librsi.so not found"):
            _abi.load(str(tmp_path / "nope.so"))
    finally:
        _abi._lib = saved


def test_cpu_tensors_are_refused():
    import torch
    import paper_2209_02878_gb300 as rsi
    V = torch.zeros((3, 3), dtype=torch.float32)
    T = torch.zeros((1, 3), dtype=torch.int32)
    with pytest.raises(ValueError, match="CUDA"):
        rsi.BVH(V, T)


def test_argument_validation_without_gpu(lib):
    """Calls that fail validation return RSI_ERR_ARG before touching CUDA."""
    from paper_2209_02878_gb300 import _abi
    L = _abi.load()
    out = _abi.rsi_output()
    lo = _abi.rsi_launch_opts()
    assert L.rsi_intersect(None, None, None, 10, 0, ctypes.byref(out), ctypes.byref(lo),
                           None) == _abi.RSI_ERR_ARG
    assert L.rsi_intersect_backward(None, -1, None, 0, None, None, 1, None, None, None, None,
                                    None, None, None) == _abi.RSI_ERR_ARG
    assert L.rsi_intersect_backward_static(None, 10**9, None, 0, None, None, 1, None, None,
                                           None, None, None, None,
                                           None) == _abi.RSI_ERR_CAPACITY
    assert L.rsi_batch_create(None, 0, None, None, None, ctypes.byref(ctypes.c_void_p())) \
        == _abi.RSI_ERR_ARG
    h = ctypes.c_void_p()
    assert L.rsi_bvh_create(-1, 10, None, None, ctypes.byref(h)) == _abi.RSI_ERR_ARG
    assert L.rsi_bvh_create(3, 1 << 31, None, None, ctypes.byref(h)) == _abi.RSI_ERR_ARG
    bo = _abi.rsi_build_opts(9, 0)
    assert L.rsi_bvh_create(3, 1, ctypes.byref(bo), None, ctypes.byref(h)) == _abi.RSI_ERR_ARG
    assert L.rsi_points_inside(None, None, 5, None, None, None) == _abi.RSI_ERR_ARG
    assert L.rsi_intersect_host(None, None, None, 5, 0, ctypes.byref(out), 0, None,
                                None) == _abi.RSI_ERR_ARG
    assert L.rsi_bvh_destroy(None) == _abi.RSI_ERR_ARG
    assert L.rsi_batch_status(None, None) == _abi.RSI_ERR_ARG
    v = ctypes.c_double(0.0)
    assert L.rsi_fp32_peak(0, ctypes.byref(v), None) == _abi.RSI_ERR_ARG
    assert L.rsi_fp32_peak(10, None, None) == _abi.RSI_ERR_ARG
    cb = _abi.ALLOC_FN(lambda n, d, s, c: None)
    assert L.rsi_set_allocator(ctypes.cast(cb, ctypes.c_void_p), None, None) == _abi.RSI_ERR_ARG
    assert L.rsi_set_allocator(None, None, None) == _abi.RSI_OK
    st = ctypes.c_int32(0)
    assert L.rsi_selftest_wait(0, None, ctypes.byref(st)) == _abi.RSI_ERR_ARG
    assert L.rsi_selftest_wait(10, None, None) == _abi.RSI_ERR_ARG
