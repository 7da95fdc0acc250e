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
