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
        if call == 0:   # and the sorted order is the oracle's
            import oracle
            assert np.array_equal(got.view(np.uint8), oracle.sort(a).view(np.uint8))


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


def test_noalloc_refuses_a_capturing_stream_and_leaves_the_capture_valid(lib):
    # The level loop reads counts back between levels, which a capturing stream cannot
    # do: the call must refuse before it enqueues anything, so the caller's capture
    # (here a torch op captured after it) still completes and replays.
    import torch
    a = inputs.make_keys(1 << 16, "int32", "uniform", seed=5)
    t = torch.from_numpy(a).cuda()
    x = torch.arange(1000, device="cuda", dtype=torch.float32)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        rc = lib.bqs_sort_noalloc(t.data_ptr(), t.numel(), 0, ctypes.c_void_p(s.cuda_stream))
        y = x * 2 + 1
    assert rc == -5, lib.bqs_status_string(rc)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(y, x * 2 + 1)
    assert np.array_equal(t.cpu().numpy(), a)     # nothing was sorted or written


def _default_pool_counters():
    """(used high watermark, used, reserved) bytes of the device's default stream-ordered
    memory pool, read through the driver API; the high watermark is reset first by the
    caller through _reset_pool_high."""
    cuda = ctypes.CDLL("libcuda.so.1")
    dev = ctypes.c_int()
    assert cuda.cuCtxGetDevice(ctypes.byref(dev)) == 0
    pool = ctypes.c_void_p()
    assert cuda.cuDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0
    out = []
    for attr in (8, 7, 5):   # CU_MEMPOOL_ATTR_USED_MEM_HIGH, _USED_MEM_CURRENT, _RESERVED_MEM_CURRENT
        v = ctypes.c_uint64()
        assert cuda.cuMemPoolGetAttribute(pool, attr, ctypes.byref(v)) == 0
        out.append(v.value)
    return tuple(out), (cuda, pool)


def test_noalloc_call_allocates_nothing(lib):
    # The entry point's defining property: a call takes no memory from any allocator.
    # After a warm-up call (set-up, including the one symbol-address lookup), the
    # default pool's high watermark is reset; a second call must leave it, the pool's
    # reservation and the device's free memory where they were.
    import torch
    a = inputs.make_keys(1 << 20, "int64", "uniform", seed=23)
    t = torch.from_numpy(a).cuda()
    w = torch.empty_like(t)
    w.copy_(t)
    assert lib.bqs_sort_noalloc(w.data_ptr(), w.numel(), 1, _stream()) == 0
    torch.cuda.synchronize()
    (_, used0, reserved0), (cuda, pool) = _default_pool_counters()
    zero = ctypes.c_uint64(0)
    assert cuda.cuMemPoolSetAttribute(pool, 8, ctypes.byref(zero)) == 0   # reset the high mark
    free0 = torch.cuda.mem_get_info()[0]
    w.copy_(t)
    torch.cuda.synchronize()
    assert lib.bqs_sort_noalloc(w.data_ptr(), w.numel(), 1, _stream()) == 0
    torch.cuda.synchronize()
    (high1, used1, reserved1), _ = _default_pool_counters()
    assert torch.cuda.mem_get_info()[0] == free0
    assert (high1, used1, reserved1) == (used0, used0, reserved0)
    assert np.array_equal(w.cpu().numpy(), np.sort(a))
