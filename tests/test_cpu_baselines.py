"""The CPU comparison sorts timed by the benchmark (std::sort, parallel sort) give
the oracle's output bit for bit under the same total order."""
import ctypes
import subprocess

import numpy as np
import pytest

import oracle
from oracle import cpu_baselines
from paper_1604_06697_gb300 import inputs

DTYPES = ["int32", "int64", "float64"]


def same_bits(x, y):
    u = np.uint32 if x.itemsize == 4 else np.uint64
    return x.shape == y.shape and np.array_equal(x.view(u), y.view(u))


@pytest.mark.parametrize("threads", [1, 2, 3, 8])
@pytest.mark.parametrize("dtype", DTYPES)
def test_cpu_sorts_match_oracle(dtype, threads):
    for dist in inputs.DISTRIBUTIONS:
        for n in (0, 1, 5000, 100_003):
            a = inputs.make_keys(n, dtype, dist, seed=n + threads)
            assert same_bits(cpu_baselines.sort(a, threads), oracle.sort(a)), (dist, n)


def test_cpu_sorts_float_specials():
    vals = np.array([0.0, -0.0, 1.0, -1.0, np.inf, -np.inf, 5e-324, -5e-324] * 3000)
    a = vals[np.argsort(inputs.splitmix64(4, vals.size))]
    for threads in (1, 4):
        assert same_bits(cpu_baselines.sort(a, threads), oracle.sort(a))


def test_thread_fallback_without_openmp(tmp_path):
    # The chunk-sort-and-merge path used where the compiler has no OpenMP.
    lib_path = str(tmp_path / "libnoomp.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread",
                           cpu_baselines._SRC, "-o", lib_path])
    lib = ctypes.CDLL(lib_path)
    lib.cpu_sort_keys.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32]
    assert lib.cpu_sort_has_openmp() == 0
    for dtype in DTYPES:
        for threads in (2, 3, 5, 8):
            a = inputs.make_keys(123_457, dtype, "mod_sqrt", seed=threads)
            got = a.copy()
            assert lib.cpu_sort_keys(got.ctypes.data, got.size, cpu_baselines.DTYPES[dtype],
                                     threads) == 3
            assert same_bits(got, oracle.sort(a))
