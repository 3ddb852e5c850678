"""ctypes wrapper of the BlockQuicksort CPU oracle (``bqs_oracle.cpp``).

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may import this
package.  The CUDA library (``paper_1604_06697_gb300``) never imports it, and
the two share no code.

Every function takes and returns numpy arrays and sorts on the host, single
threaded.  The C++ file states, part by part, which passage of the paper
(arXiv 1604.06697) each routine follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bqs_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle_bqs.so")

DTYPES = {"int32": 0, "int64": 1, "float64": 2}
NP_DTYPES = {0: np.int32, 1: np.int64, 2: np.float64}
PIVOT_RULES = {"mo3": 0, "sqrt": 1}

_lib = None


def build(force: bool = False) -> str:
    """Compiles the oracle into ``oracle/liboracle_bqs.so`` (plain g++, no CUDA)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(
            ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        lib.oracle_sort.argtypes = [vp, i64, i32, i32, i64, i64, vp]
        lib.oracle_sort.restype = ctypes.c_int
        lib.oracle_sort_pairs.argtypes = [vp, vp, i64, i32, i32, vp]
        lib.oracle_sort_pairs.restype = ctypes.c_int
        lib.oracle_sort_segmented.argtypes = [vp, vp, i64, i32, i32]
        lib.oracle_sort_segmented.restype = ctypes.c_int
        lib.oracle_block_partition.argtypes = [vp, i64, i32, i64, vp]
        lib.oracle_block_partition.restype = i64
        lib.oracle_partition_by_value.argtypes = [vp, i64, i32, vp, vp]
        lib.oracle_partition_by_value.restype = i64
        lib.oracle_select.argtypes = [vp, i64, i32, i64, vp]
        lib.oracle_select.restype = ctypes.c_int
        lib.oracle_record_keys.argtypes = [vp, i64, i32, i32, i32, i32, vp]
        lib.oracle_record_keys.restype = ctypes.c_int
        lib.oracle_pivot_value.argtypes = [vp, i64, i32, i32, i64, i64, vp]
        lib.oracle_pivot_value.restype = ctypes.c_int
        _lib = lib
    return _lib


def use_library(path: str) -> None:
    """Points the wrapper at another build of the oracle source (used by the test
    that plants mistakes in a copy of the oracle to show that the pins catch them)."""
    global _lib
    _lib = None
    _load()  # make sure the signatures of the default build are known
    lib = ctypes.CDLL(path)
    for name in ("oracle_sort", "oracle_sort_pairs", "oracle_sort_segmented",
                 "oracle_block_partition", "oracle_partition_by_value", "oracle_select",
                 "oracle_record_keys", "oracle_pivot_value"):
        f, g = getattr(lib, name), getattr(_lib, name)
        f.argtypes, f.restype = g.argtypes, g.restype
    _lib = lib


def reset_library() -> None:
    global _lib
    _lib = None


def _dtype_code(a: np.ndarray) -> int:
    for name, code in DTYPES.items():
        if a.dtype == np.dtype(name):
            return code
    raise TypeError(f"oracle: unsupported dtype {a.dtype}")


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def sort(keys: np.ndarray, pivot: str = "mo3", is_thresh: int = 16,
         depth_limit: int = -1, counters: bool = False):
    """Returns a sorted copy of ``keys`` (int32/int64/float64) by BlockQuicksort.

    ``is_thresh``: Insertionsort for sub-arrays of at most this many elements
    (16 in the paper); ``depth_limit`` < 0 selects 2*floor(log2 n)+3.  With
    ``counters=True`` also returns a dict of comparisons, partitions,
    insertion sorts, heap sorts, the depth limit used and the deepest level.
    """
    a = np.ascontiguousarray(keys).copy()
    c = np.zeros(6, np.uint64)
    rc = _load().oracle_sort(_ptr(a), a.size, _dtype_code(a), PIVOT_RULES[pivot],
                             is_thresh, depth_limit, _ptr(c))
    if rc:
        raise ValueError("oracle_sort: invalid arguments")
    if counters:
        return a, dict(zip(("comparisons", "partitions", "insertion_sorts", "heap_sorts",
                            "depth_limit", "max_depth"), (int(x) for x in c)))
    return a


def sort_inplace(keys: np.ndarray, pivot: str = "mo3") -> None:
    """Sorts a contiguous int32/int64/float64 array in place by BlockQuicksort (the same
    routine as sort(), without the copy; used to time the oracle)."""
    if not keys.flags["C_CONTIGUOUS"]:
        raise ValueError("sort_inplace needs a contiguous array")
    if _load().oracle_sort(_ptr(keys), keys.size, _dtype_code(keys), PIVOT_RULES[pivot], 16, -1,
                           None):
        raise ValueError("oracle_sort: invalid arguments")


def sort_pairs(keys: np.ndarray, vals: np.ndarray, pivot: str = "mo3"):
    """Sorts (key, payload) pairs lexicographically; returns (keys, vals) copies."""
    k = np.ascontiguousarray(keys).copy()
    v = np.ascontiguousarray(vals, dtype=np.uint32).copy()
    if k.size != v.size:
        raise ValueError("keys and vals differ in length")
    rc = _load().oracle_sort_pairs(_ptr(k), _ptr(v), k.size, _dtype_code(k),
                                   PIVOT_RULES[pivot], None)
    if rc:
        raise ValueError("oracle_sort_pairs: invalid arguments")
    return k, v


def sort_segmented(keys: np.ndarray, seg_offsets: np.ndarray, pivot: str = "mo3"):
    """Sorts every segment [off[i], off[i+1]) of a copy of ``keys`` on its own."""
    a = np.ascontiguousarray(keys).copy()
    off = np.ascontiguousarray(seg_offsets, dtype=np.int64)
    nseg = off.size - 1
    if nseg < 0 or (nseg > 0 and off[-1] > a.size):
        raise ValueError("bad seg_offsets")
    rc = _load().oracle_sort_segmented(_ptr(a), _ptr(off), nseg, _dtype_code(a),
                                       PIVOT_RULES[pivot])
    if rc:
        raise ValueError("oracle_sort_segmented: invalid arguments")
    return a


def block_partition(keys: np.ndarray, pivot_pos: int, counters: bool = False):
    """Algorithm 3 on a copy of ``keys`` around keys[pivot_pos].

    Returns (array, p) with array[:p] <= array[p] <= array[p+1:].
    """
    a = np.ascontiguousarray(keys).copy()
    c = np.zeros(6, np.uint64)
    p = _load().oracle_block_partition(_ptr(a), a.size, _dtype_code(a), int(pivot_pos), _ptr(c))
    if p < 0:
        raise ValueError("oracle_block_partition: invalid arguments")
    if counters:
        return a, int(p), int(c[0])
    return a, int(p)


def partition_by_value(keys: np.ndarray, pivot):
    """Plain stable value partition: (out, split) with split = count(< pivot)."""
    a = np.ascontiguousarray(keys)
    out = np.empty_like(a)
    pv = np.array([pivot], dtype=a.dtype)
    s = _load().oracle_partition_by_value(_ptr(a), a.size, _dtype_code(a), _ptr(pv), _ptr(out))
    if s < 0:
        raise ValueError("oracle_partition_by_value: invalid arguments")
    return out, int(s)


def select(keys: np.ndarray, k: int):
    """The key at position k of the sorted keys (k-th order statistic)."""
    a = np.ascontiguousarray(keys)
    out = np.zeros(1, dtype=a.dtype)
    if _load().oracle_select(_ptr(a), a.size, _dtype_code(a), int(k), _ptr(out)):
        raise ValueError("oracle_select: invalid arguments")
    return out[0]


def pivot_value(keys: np.ndarray, b: int, e: int, pivot: str = "sqrt"):
    """The pivot the sort chooses for keys[b:e] under a pivot rule (keys unchanged)."""
    a = np.ascontiguousarray(keys)
    out = np.zeros(1, dtype=a.dtype)
    if _load().oracle_pivot_value(_ptr(a), a.size, _dtype_code(a), PIVOT_RULES[pivot], int(b),
                                  int(e), _ptr(out)):
        raise ValueError("oracle_pivot_value: invalid arguments")
    return out[0]


def ord_f64(x: np.ndarray) -> np.ndarray:
    """The total order key of float64 values used throughout (uint64)."""
    u = np.ascontiguousarray(x, dtype=np.float64).view(np.uint64)
    neg = (u >> np.uint64(63)).astype(bool)
    return np.where(neg, ~u, u | np.uint64(1 << 63))


def record_keys(records: np.ndarray, record_bytes: int, kind: int, offset: int = 0,
                count: int = 1) -> np.ndarray:
    """Keys of fixed-size records (bytes, n * record_bytes): kind 0 = the int32 field at
    ``offset``; kind 1 = the squared norm of ``count`` doubles from ``offset``."""
    rec = np.ascontiguousarray(records).view(np.uint8)
    n = rec.size // record_bytes
    keys = np.empty(n, dtype=np.int32 if kind == 0 else np.float64)
    rc = _load().oracle_record_keys(rec.ctypes.data, n, record_bytes, kind, offset, count,
                                    keys.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_record_keys rejected its arguments")
    return keys


def sort_records(records: np.ndarray, record_bytes: int, kind: int, offset: int = 0,
                 count: int = 1) -> np.ndarray:
    """Records (bytes, n * record_bytes) sorted by their keys, ties by input position:
    the (key, index) pairs are sorted by the paper's algorithm, then the records are
    moved to their places."""
    rec = np.ascontiguousarray(records).view(np.uint8)
    n = rec.size // record_bytes
    keys = record_keys(rec, record_bytes, kind, offset, count)
    _, order = sort_pairs(keys, np.arange(n, dtype=np.uint32))
    return rec.reshape(n, record_bytes)[order.astype(np.int64)].reshape(-1)

