"""ctypes wrapper of the CPU comparison sorts (``cpu_sort_baselines.cpp``).

MEASUREMENT INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only ``tests/``, the CPU
baseline leg of ``bench.py`` and ``__graft_entry__.build()`` use this module.

``sort(a, threads=1)`` is std::sort on one host thread; with more threads it is
__gnu_parallel::sort (OpenMP) or, where the compiler has no OpenMP, a
chunk-sort-and-merge on std::threads.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cpu_sort_baselines.cpp")
_LIB = os.path.join(_HERE, "libcpu_sort_baselines.so")

DTYPES = {"int32": 0, "int64": 1, "float64": 2}
KINDS = {1: "std::sort", 2: "__gnu_parallel::sort", 3: "std::sort chunks + std::merge tree"}

_lib = None


def build(force: bool = False) -> str:
    """Compiles ``libcpu_sort_baselines.so`` with OpenMP if the compiler has it."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        base = ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", _SRC, "-o", tmp, "-pthread"]
        try:
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:],
                                  stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.cpu_sort_keys.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                      ctypes.c_int32]
        lib.cpu_sort_keys.restype = ctypes.c_int
        lib.cpu_sort_has_openmp.restype = ctypes.c_int
        _lib = lib
    return _lib


def sort_inplace(a: np.ndarray, threads: int = 1) -> str:
    """Sorts the contiguous array ``a`` in place; returns the sort's name."""
    assert a.flags["C_CONTIGUOUS"]
    rc = _load().cpu_sort_keys(a.ctypes.data, a.size, DTYPES[str(a.dtype)], int(threads))
    if rc < 0:
        raise ValueError(f"unsupported dtype {a.dtype}")
    return KINDS[rc]


def sort(a: np.ndarray, threads: int = 1) -> np.ndarray:
    out = np.ascontiguousarray(a).copy()
    sort_inplace(out, threads)
    return out


def has_openmp() -> bool:
    return bool(_load().cpu_sort_has_openmp())
