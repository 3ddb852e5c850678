"""ctypes loader of the in-tree CUDA library ``libbqs.so`` (argument marshalling only).

Every entry point of ``include/bqs.h`` is declared here with its C signature.
There is no fallback: if the library is missing or cannot be loaded, the first
call raises.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libbqs.so")

c_i32, c_i64, c_vp, c_dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_double


class Pivot(ctypes.Structure):
    class _V(ctypes.Union):
        _fields_ = [("i32", ctypes.c_int32), ("i64", ctypes.c_int64), ("f64", ctypes.c_double)]

    _fields_ = [("dtype", ctypes.c_int32), ("reserved", ctypes.c_int32), ("v", _V)]


class Stats(ctypes.Structure):
    _fields_ = [(name, c_i64) for name in (
        "levels", "partition_launches", "active_keys", "moved_keys", "equal_keys",
        "small_segments", "small_keys", "local_segments", "local_keys", "fallback_pivots",
        "kernel_launches")] + [
        ("partition_ms", c_dbl), ("partition_bytes", c_dbl), ("coop_ms", c_dbl)]


# name -> (restype, argtypes); mirrors include/bqs.h
SIGNATURES = {
    "bqs_partition": (ctypes.c_int, [c_vp, c_i64, ctypes.POINTER(Pivot), c_vp, ctypes.POINTER(c_i64), c_vp]),
    "bqs_sort": (ctypes.c_int, [c_vp, c_i64, c_i32, c_vp]),
    "bqs_sort_segmented": (ctypes.c_int, [c_vp, c_vp, c_i64, c_i32, c_vp]),
    "bqs_sort_batched": (ctypes.c_int, [c_vp, c_i64, c_vp, c_i64, c_i32, c_vp]),
    "bqs_sort_pairs": (ctypes.c_int, [c_vp, c_vp, c_i64, c_i32, c_vp]),
    "bqs_sort_noalloc": (ctypes.c_int, [c_vp, c_i64, c_i32, c_vp]),
    "bqs_sort_records": (ctypes.c_int, [c_vp, c_i64, c_i32, c_i32, c_i32, c_i32, c_vp]),
    "bqs_set_option": (ctypes.c_int, [c_i32, c_i64]),
    "bqs_get_option": (ctypes.c_int, [c_i32, ctypes.POINTER(c_i64)]),
    "bqs_workspace_bytes": (ctypes.c_int, [c_i64, c_i32, c_i32, c_i64, ctypes.POINTER(c_i64)]),
    "bqs_set_workspace": (ctypes.c_int, [c_vp, c_i64]),
    "bqs_get_stats": (ctypes.c_int, [ctypes.POINTER(Stats)]),
    "bqs_timing_collect": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(c_i64)]),
    "bqs_status_string": (ctypes.c_char_p, [ctypes.c_int]),
}

_lib = None


def lib():
    """Loads ``libbqs.so`` once (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with paper_1604_06697_gb300.build.build() "
                "(there is no CPU fallback)")
        l = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(l, name)
            f.restype, f.argtypes = res, args
        _lib = l
    return _lib
