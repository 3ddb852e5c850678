"""bqs_sort_noalloc: the sort entry point for callers that cannot allocate memory.

Such callers (a service that reserves its device memory up front, code inside a
framework whose allocator owns the GPU) get the same sorted result from a fixed
scratch array that the library holds.  These tests call it through the C ABI and
compare it with bqs_sort on the same input, bit for bit, on two calls in a row
(the second call reuses the array the first one left behind).  The file is named
so that pytest collects it last; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_1604_06697_gb300 import inputs

pytestmark = pytest.mark.gpu

DTYPES = {"int32": 0, "int64": 1, "float64": 2}


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_1604_06697_gb300 import _native, build
    build.build()
    torch.cuda.init()
    return _native.lib()


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _sort_with(lib, name, a):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    rc = getattr(lib, name)(t.data_ptr(), t.numel(), DTYPES[str(a.dtype)], _stream())
    torch.cuda.synchronize()
    assert rc == 0, (name, rc, lib.bqs_status_string(rc))
    return t.cpu().numpy()


@pytest.mark.parametrize("dtype", list(DTYPES))
def test_noalloc_matches_bqs_sort_on_two_calls(lib, dtype):
    for call, (n, dist) in enumerate([(1 << 20, "uniform"), (300_001, "mod_sqrt")]):
        a = inputs.make_keys(n, dtype, dist, seed=17 + call)
        want = _sort_with(lib, "bqs_sort", a)
        got = _sort_with(lib, "bqs_sort_noalloc", a)
        assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), (dtype, call)


def test_noalloc_small_and_edge_sizes(lib):
    for n in (0, 1, 2, 17, 2048, 2049, 100_003):
        a = inputs.make_keys(n, "int32", "uniform", seed=n)
        got = _sort_with(lib, "bqs_sort_noalloc", a)
        assert np.array_equal(got, np.sort(a))


def test_noalloc_rejects_sizes_above_its_scratch(lib):
    import torch
    t = torch.zeros((1 << 20) + 1, dtype=torch.int32, device="cuda")
    rc = lib.bqs_sort_noalloc(t.data_ptr(), t.numel(), 0, _stream())
    assert rc == -7
    assert b"2^20" in lib.bqs_status_string(rc)
