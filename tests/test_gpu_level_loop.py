"""The level loop driven by device-side counts (BQS_OPT_LEVEL_LOOP = 1).

The host enqueues levels ahead and reads a per-level flag a few levels behind, so
every kernel takes its work counts from the control block.  Outputs must be the
oracle's, bit for bit.  The level count itself is not reproducible between runs
(tiles reserve their output ranges in whatever order their atomics land, so
position-based pivot samples differ), but the statistics of either loop satisfy the
same conservation laws: every key is finished exactly once (in a pivot class, a
sorting network or a single-block sort), and every partitioned key is either moved
or in its segment's pivot class.
"""
import numpy as np
import pytest

import oracle
from paper_1604_06697_gb300 import inputs

pytestmark = pytest.mark.gpu

DTYPES = ["int32", "int64", "float64"]


@pytest.fixture(scope="module")
def bqs():
    import torch
    from paper_1604_06697_gb300 import build
    build.build()
    import paper_1604_06697_gb300 as m
    torch.cuda.init()
    return m


def assert_same_bits(got, want):
    gu = got.view(np.uint32 if got.itemsize == 4 else np.uint64)
    wu = want.view(np.uint32 if want.itemsize == 4 else np.uint64)
    assert got.shape == want.shape and np.array_equal(gu, wu)


@pytest.fixture(autouse=True)
def host_driven_loops(bqs):
    # Both loops under test are host-driven; arrays up to BQS_OPT_COOP_MAX keys would
    # otherwise take the single-launch path with level_loop 0 (test_gpu_coop.py).
    bqs.set_option("coop_max", 0)
    yield


def sort_with(bqs, a, loop):
    import torch
    bqs.set_option("level_loop", loop)
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    bqs.sort(t)
    torch.cuda.synchronize()
    return t.cpu().numpy(), bqs.stats()


def assert_conservation(st, n):
    if n <= 1:
        return                      # nothing to sort: no device work, zero statistics
    assert st["equal_keys"] + st["small_keys"] + st["local_keys"] == n, st
    assert st["active_keys"] == st["moved_keys"] + st["equal_keys"], st
    assert (st["levels"] > 0) == (st["active_keys"] > 0), st


@pytest.mark.parametrize("dist", inputs.DISTRIBUTIONS)
@pytest.mark.parametrize("dtype", DTYPES)
def test_levels_ahead_matches_oracle_and_host_loop(bqs, dtype, dist):
    for n in (0, 1, 255, 2049, 70_001, 1 << 20):
        a = inputs.make_keys(n, dtype, dist, seed=n + 7)
        want = oracle.sort(a)
        for loop in (1, 0):
            got, st = sort_with(bqs, a, loop)
            assert_same_bits(got, want)
            assert_conservation(st, n)


@pytest.mark.parametrize("cutoff", [2048, 4096])
@pytest.mark.parametrize("tile", [0, 5])
@pytest.mark.parametrize("local", [0, -1])
@pytest.mark.parametrize("dtype", DTYPES)
def test_levels_ahead_options(bqs, dtype, local, tile, cutoff):
    bqs.set_option("tile", tile)
    bqs.set_option("local_cutoff", local)
    bqs.set_option("small_cutoff", cutoff)
    bqs.set_option("pivot", 1)
    for n, dist in [(300_001, "uniform"), (1 << 22, "mod_sqrt"), (100_000, "all_equal")]:
        a = inputs.make_keys(n, dtype, dist, seed=11)
        got, st = sort_with(bqs, a, 1)
        assert_same_bits(got, oracle.sort(a, pivot="sqrt"))
        assert_conservation(st, n)
        if local != 0 and dist == "uniform" and (cutoff < 4096 or dtype == "int32"):
            assert st["local_keys"] > 0     # one block holds 8192 32-bit or 4096 64-bit keys


def test_levels_ahead_depth_fallback_and_timing(bqs):
    bqs.set_option("depth_limit", 1)
    bqs.set_option("small_cutoff", 16)
    bqs.set_option("timing", 1)
    a = inputs.make_keys(1 << 21, "int64", "uniform", seed=5)
    for loop in (1, 0):
        got, st = sort_with(bqs, a, loop)
        assert_same_bits(got, oracle.sort(a))
        assert st["fallback_pivots"] > 0
        assert st["partition_ms"] > 0
        assert_conservation(st, a.size)


@pytest.mark.parametrize("dtype", DTYPES)
def test_levels_ahead_segmented_and_pairs(bqs, dtype):
    import torch
    bqs.set_option("level_loop", 1)
    keys, off = inputs.make_segments(2048, seed=3, lo=1, hi=40_000, dtype=dtype)
    t = torch.from_numpy(keys).cuda()
    bqs.sort_segmented(t, torch.from_numpy(off).cuda())
    assert_same_bits(t.cpu().numpy(), oracle.sort_segmented(keys, off))

    n = 200_003
    k = (inputs.splitmix64(9, n) % np.uint64(5000)).astype(dtype)
    v = np.arange(n, dtype=np.uint32)[np.argsort(inputs.splitmix64(10, n))].astype(np.uint32)
    tk, tv = torch.from_numpy(k).cuda(), torch.from_numpy(v.view(np.int32)).cuda()
    bqs.sort_pairs(tk, tv)
    wk, wv = oracle.sort_pairs(k, v)
    assert_same_bits(tk.cpu().numpy(), wk)
    assert_same_bits(tv.cpu().numpy().view(np.uint32), wv)


def test_levels_ahead_rejects_decreasing_offsets(bqs):
    import torch
    bqs.set_option("level_loop", 1)
    t = torch.zeros(100, dtype=torch.int32, device="cuda")
    off = torch.tensor([0, 50, 40, 100], dtype=torch.int64, device="cuda")
    with pytest.raises(bqs.BqsError):
        bqs.sort_segmented(t, off)
    # the next call is unaffected
    a = inputs.make_keys(5000, "int32", "uniform", seed=1)
    got, _ = sort_with(bqs, a, 1)
    assert_same_bits(got, oracle.sort(a))
