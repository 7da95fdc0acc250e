"""ctypes mirror of include/rsi.h (structures, enums, prototypes).

Argument marshalling only: every computation happens in librsi.so.  Loading
fails loudly when the library has not been built; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "librsi.so")

RSI_OK = 0
RSI_ERR_ARG = 1
RSI_ERR_CUDA = 2
RSI_ERR_OOM = 3
RSI_ERR_BAD_INDEX = 4
RSI_ERR_STACK_OVERFLOW = 5
RSI_ERR_TIMEOUT = 6
RSI_ERR_NOT_BUILT = 7
RSI_ERR_INTERNAL = 8
RSI_ERR_CAPACITY = 9
RSI_STATIC_MAX_VERTICES = 262144

RSI_MODE_BOOL = 0
RSI_MODE_COUNT = 1
RSI_MODE_NEAREST = 2

MODES = {"bool": RSI_MODE_BOOL, "count": RSI_MODE_COUNT, "nearest": RSI_MODE_NEAREST,
         "barycentric": RSI_MODE_NEAREST, "intercept_count": RSI_MODE_COUNT}

vp = C.c_void_p
i32 = C.c_int32
i64 = C.c_int64


class rsi_build_opts(C.Structure):
    _fields_ = [("leaf_size", i32), ("top_levels", i32), ("height_axis", i32)]


# rsi_alloc_fn / rsi_free_fn (pass as c_void_p after ctypes.cast)
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_int, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p)


class rsi_launch_opts(C.Structure):
    _fields_ = [("block_size", i32), ("stack_depth", i32), ("smem_nodes", i32), ("stats", i32),
                ("sort_bits", i32), ("node_width", i32), ("packet", i32), ("order", vp)]


class rsi_output(C.Structure):
    _fields_ = [("flag", vp), ("count", vp), ("tri", vp), ("tuv", vp), ("point", vp),
                ("dist", vp), ("hit_idx", vp), ("hit_cap", i64), ("n_hits", vp),
                ("hit_tri", vp), ("hit_dist", vp), ("hit_point", vp), ("hit_count", vp)]


class rsi_bvh_info(C.Structure):
    _fields_ = [("n_vertices", i64), ("n_triangles", i64), ("leaf_size", i32),
                ("treelet_nodes", i32), ("device_bytes", i64)]


class rsi_stats(C.Structure):
    _fields_ = [("segments", i64), ("node_visits", i64), ("tri_tests", i64),
                ("fp64_tests", i64), ("df_refines", i64), ("overflows", i64),
                ("fp64_values", i64)]


class rsi_batch_item(C.Structure):
    _fields_ = [("dV", vp), ("nV", i64), ("dT", vp), ("nT", i64), ("dA", vp), ("dB", vp),
                ("nR", i64), ("mode", i32), ("height_axis", i32), ("out", rsi_output)]


class rsi_tune_entry(C.Structure):
    _fields_ = [("block_size", i32), ("stack_depth", i32), ("smem_nodes", i32),
                ("leaf_size", i32), ("ms", C.c_float)]


P = C.POINTER
_PROTOS = {
    "rsi_version": (C.c_char_p, []),
    "rsi_status_string": (C.c_char_p, [C.c_int]),
    "rsi_bvh_create": (C.c_int, [i64, i64, P(rsi_build_opts), vp, P(vp)]),
    "rsi_bvh_build": (C.c_int, [vp, vp, vp, vp]),
    "rsi_build_bvh": (C.c_int, [vp, i64, vp, i64, P(rsi_build_opts), vp, P(vp)]),
    "rsi_refit": (C.c_int, [vp, vp, vp, vp]),
    "rsi_bvh_status": (C.c_int, [vp, vp]),
    "rsi_batch_status": (C.c_int, [vp, vp]),
    "rsi_bvh_get_info": (C.c_int, [vp, P(rsi_bvh_info)]),
    "rsi_bvh_destroy": (C.c_int, [vp]),
    "rsi_bvh_export": (C.c_int, [vp, vp] + [vp] * 9),
    "rsi_intersect": (C.c_int, [vp, vp, vp, i64, C.c_int, P(rsi_output), P(rsi_launch_opts), vp]),
    "rsi_segment_order": (C.c_int, [vp, vp, vp, i64, i32, vp, vp]),
    "rsi_intersect_host": (C.c_int, [vp, vp, vp, i64, C.c_int, P(rsi_output), i64,
                                     P(rsi_launch_opts), vp]),
    "rsi_points_inside": (C.c_int, [vp, vp, i64, vp, P(rsi_launch_opts), vp]),
    "rsi_intersect_stats": (C.c_int, [vp, vp, vp, i64, C.c_int, P(rsi_output),
                                      P(rsi_launch_opts), vp, P(rsi_stats)]),
    "rsi_intersect_backward": (C.c_int, [vp, i64, vp, i64, vp, vp, i64, vp, vp, vp, vp, vp,
                                         vp, vp]),
    "rsi_intersect_backward_static": (C.c_int, [vp, i64, vp, i64, vp, vp, i64, vp, vp, vp, vp,
                                                vp, vp, vp]),
    "rsi_batch_create": (C.c_int, [P(rsi_batch_item), i32, P(rsi_build_opts),
                                   P(rsi_launch_opts), vp, P(vp)]),
    "rsi_batch_build": (C.c_int, [vp, vp]),
    "rsi_batch_intersect": (C.c_int, [vp, vp]),
    "rsi_batch_run_graph": (C.c_int, [vp, i32, vp]),
    "rsi_batch_destroy": (C.c_int, [vp]),
    "rsi_autotune_height_axis": (C.c_int, [vp, vp, vp, vp, vp, i64, C.c_int, P(rsi_output),
                                           P(rsi_launch_opts), i32, vp, P(C.c_float),
                                           P(i32)]),
    "rsi_autotune": (C.c_int, [vp, vp, vp, vp, vp, i64, C.c_int, P(rsi_output),
                               P(i32), i32, P(i32), i32, P(i32), i32, P(i32), i32, i32, vp,
                               P(rsi_tune_entry), i32, P(i32), P(rsi_launch_opts), P(i32)]),
    "rsi_fp32_peak": (C.c_int, [i64, P(C.c_double), vp]),
    "rsi_set_allocator": (C.c_int, [vp, vp, vp]),
    "rsi_selftest_wait": (C.c_int, [i32, vp, P(i32)]),
    "rsi_selftest_stream_wait": (C.c_int, [i32, i64, vp, P(i32), P(C.c_float)]),
}

# every entry point declared in include/rsi.h
EXPORTS = tuple(_PROTOS)

_lock = threading.Lock()
_lib = None


class RSIError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = _status_text(code)
        super().__init__(f"{where}: {msg} (status {code})")


def _status_text(code: int) -> str:
    try:
        return load().rsi_status_string(code).decode()
    except Exception:
        return "status"


def load(path: str | None = None):
    """Load librsi.so (once).  Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(
                f"librsi.so not found at {p}: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'` (nvcc, sm_103a)")
        lib = C.CDLL(p)
        for name, (res, args) in _PROTOS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def check(code: int, where: str) -> None:
    if code != RSI_OK:
        raise RSIError(code, where)
