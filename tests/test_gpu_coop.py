"""Parity of the single-launch sort (one cooperative kernel runs every level) with
the CPU oracle, through the C ABI.

Single key-only arrays of more than the small-segment cutoff and at most
BQS_OPT_COOP_MAX keys take this path.  Outputs are compared bit for bit (float64
by bits), over the same sizes, distributions and pivot rules as the host-driven
level loop, plus the limit itself, sample pivots (the pivot step inside the
kernel), depth-limit fallbacks and small cutoffs.
"""
import numpy as np
import pytest

import oracle
from paper_1604_06697_gb300 import inputs

pytestmark = pytest.mark.gpu

DTYPES = ["int32", "int64", "float64"]
SIZES = [2049, 4095, 4097, 8191, 8193, 65535, 65537, 100_003, (1 << 20) + 1]
LIMIT = 1 << 22


@pytest.fixture(scope="module")
def bqs():
    import torch
    from paper_1604_06697_gb300 import build
    build.build()
    import paper_1604_06697_gb300 as m
    torch.cuda.init()
    return m


@pytest.fixture(autouse=True)
def coop_on(bqs):
    saved = {k: bqs.get_option(k) for k in bqs.OPTIONS}
    bqs.set_option("coop_max", LIMIT)
    yield
    for k, v in saved.items():
        bqs.set_option(k, v)


def sort_one(bqs, a):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    bqs.sort(t)
    torch.cuda.synchronize()
    return t.cpu().numpy(), bqs.stats()


def same_bits(got, want):
    return np.array_equal(got.view(np.uint8), want.view(np.uint8))


@pytest.mark.parametrize("pivot", [0, 1])
@pytest.mark.parametrize("dist", inputs.DISTRIBUTIONS)
@pytest.mark.parametrize("dtype", DTYPES)
def test_single_launch_matches_oracle(bqs, dtype, dist, pivot):
    bqs.set_option("pivot", pivot)
    for n in SIZES:
        a = inputs.make_keys(n, dtype, dist, seed=n)
        got, st = sort_one(bqs, a)
        assert same_bits(got, oracle.sort(a)), (dtype, dist, n)
        # one cooperative launch plus the control-block read-back, no partition launch
        assert st["kernel_launches"] == 2 and st["partition_launches"] == 0, st


def test_the_limit_and_one_past_it(bqs):
    bqs.set_option("pivot", 1)
    for n, single in ((LIMIT, True), (LIMIT + 3, False)):
        a = inputs.make_keys(n, "int32", "uniform", seed=5)
        got, st = sort_one(bqs, a)
        assert same_bits(got, oracle.sort(a))
        assert (st["partition_launches"] == 0) == single, (n, st)
    # keys conserved in the statistics of the single launch
    a = inputs.make_keys(LIMIT, "int64", "mod_sqrt", seed=6)
    got, st = sort_one(bqs, a)
    assert same_bits(got, oracle.sort(a))
    assert st["moved_keys"] + st["equal_keys"] == st["active_keys"]
    assert st["small_keys"] + st["equal_keys"] == LIMIT


@pytest.mark.parametrize("rule", [0, 1, 2, 3, 4, 5, 6])
def test_every_pivot_rule(bqs, rule):
    bqs.set_option("pivot", rule)
    for dtype in DTYPES:
        a = inputs.make_keys(300_007, dtype, "uniform", seed=rule)
        got, _ = sort_one(bqs, a)
        assert same_bits(got, oracle.sort(a))


@pytest.mark.parametrize("limit", [0, 1, 3])
@pytest.mark.parametrize("dtype", DTYPES)
def test_depth_limit_fallback_inside_the_launch(bqs, dtype, limit):
    # Past the limit the pivot step inside the kernel takes the key-range midpoint.
    bqs.set_option("depth_limit", limit)
    for dist in ("uniform", "mod_sqrt", "all_equal", "reversed"):
        a = inputs.make_keys(200_001, dtype, dist, seed=limit + 1)
        got, st = sort_one(bqs, a)
        assert same_bits(got, oracle.sort(a)), (dist, limit)
        assert st["partition_launches"] == 0


@pytest.mark.parametrize("cutoff", [2, 16, 256, 1000, 2048, 3000, 4096])
def test_small_cutoffs(bqs, cutoff):
    bqs.set_option("small_cutoff", cutoff)
    bqs.set_option("pivot", 1)
    for dtype in DTYPES:
        a = inputs.make_keys(150_001, dtype, "uniform", seed=cutoff)
        got, st = sort_one(bqs, a)
        assert same_bits(got, oracle.sort(a)), (dtype, cutoff)


def test_structured_inputs(bqs):
    bqs.set_option("pivot", 1)
    for dist in inputs.EXTRA_DISTRIBUTIONS:
        for dtype in DTYPES:
            a = inputs.make_keys(1 << 20, dtype, dist, seed=1)
            got, _ = sort_one(bqs, a)
            assert same_bits(got, oracle.sort(a)), (dtype, dist)


def test_float64_special_values_and_extremes(bqs):
    specials = np.array([0.0, -0.0, np.inf, -np.inf, 5e-324, -5e-324,
                         np.finfo(np.float64).max, -np.finfo(np.float64).max], dtype=np.float64)
    a = np.resize(specials, 50_000).copy()
    got, _ = sort_one(bqs, a)
    assert same_bits(got, oracle.sort(a))
    b = np.resize(np.array([np.iinfo(np.int32).min, np.iinfo(np.int32).max, 0, -1, 1], np.int32),
                  70_001).copy()
    got, _ = sort_one(bqs, b)
    assert same_bits(got, oracle.sort(b))


def test_options_that_keep_the_host_loop(bqs):
    # Local partitioning and the 256-thread block networks stay on the host loop.
    a = inputs.make_keys(1 << 18, "int32", "uniform", seed=3)
    for name, value in (("local_cutoff", -1), ("small_sort", 1), ("level_loop", 1)):
        bqs.set_option(name, value)
        got, st = sort_one(bqs, a)
        assert same_bits(got, oracle.sort(a))
        assert st["partition_launches"] > 0, name
        bqs.set_option(name, 0)
