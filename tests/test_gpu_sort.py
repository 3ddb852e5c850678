"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Sorted outputs are unique, so the comparison is bit-exact (tolerance 0;
float64 compared by bits).  Partitions are compared on what is unique: the
split and the multiset of each side.  Sizes span several tiles and ragged
tails; edge cases cover empty, single-key, all-equal and tile-boundary sizes.
"""
import numpy as np
import pytest

import oracle
from paper_1604_06697_gb300 import inputs

pytestmark = pytest.mark.gpu

DTYPES = ["int32", "int64", "float64"]
EDGE_SIZES = [0, 1, 2, 3, 4, 15, 16, 17, 31, 33, 127, 128, 129, 255, 257, 2047, 2048, 2049,
              4095, 4096, 4097, 8191, 8193, 65535, 65537, (1 << 20) + 1]


@pytest.fixture(scope="module")
def bqs():
    import torch
    from paper_1604_06697_gb300 import build
    build.build()
    import paper_1604_06697_gb300 as m
    torch.cuda.init()
    return m


@pytest.fixture(autouse=True)
def default_options(bqs):
    # These tests check the host-driven level loop at every size; the single-launch
    # path for arrays up to BQS_OPT_COOP_MAX keys has its own (test_gpu_coop.py).
    saved = {k: bqs.get_option(k) for k in bqs.OPTIONS}
    bqs.set_option("coop_max", 0)
    yield
    for k, v in saved.items():
        bqs.set_option(k, v)


def gpu_sort(bqs, a):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    bqs.sort(t)
    torch.cuda.synchronize()
    return t.cpu().numpy()


def assert_same_bits(got, want):
    assert got.dtype == want.dtype and got.shape == want.shape
    gu = got.view(np.uint32 if got.itemsize == 4 else np.uint64)
    wu = want.view(np.uint32 if want.itemsize == 4 else np.uint64)
    if not np.array_equal(gu, wu):
        idx = np.nonzero(gu != wu)[0]
        raise AssertionError(f"{idx.size} mismatches, first at {idx[:5]}: got {got[idx[:5]]} "
                             f"want {want[idx[:5]]}")


@pytest.mark.parametrize("dist", inputs.DISTRIBUTIONS)
@pytest.mark.parametrize("dtype", DTYPES)
def test_sort_matches_oracle_edge_sizes(bqs, dtype, dist):
    for n in EDGE_SIZES:
        a = inputs.make_keys(n, dtype, dist, seed=n + 1)
        assert_same_bits(gpu_sort(bqs, a), oracle.sort(a))


@pytest.mark.parametrize("pivot", [0, 1])
@pytest.mark.parametrize("tile", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("dtype", DTYPES)
def test_sort_pivot_rules_and_tiles(bqs, dtype, tile, pivot):
    bqs.set_option("pivot", pivot)
    bqs.set_option("tile", tile)
    for n, dist in [(100_000, "uniform"), (300_001, "mod_sqrt"), (1 << 18, "swapped_1pct"),
                    (70_001, "reversed")]:
        a = inputs.make_keys(n, dtype, dist, seed=3)
        assert_same_bits(gpu_sort(bqs, a), oracle.sort(a, pivot="sqrt" if pivot else "mo3"))


@pytest.mark.parametrize("cutoff", [2, 3, 16, 64, 1000, 2048, 3000, 4096])
def test_small_cutoffs(bqs, cutoff):
    bqs.set_option("small_cutoff", cutoff)
    for dtype in DTYPES:
        for n in (5, 100, 3000, 50_001):
            a = inputs.make_keys(n, dtype, "uniform", seed=n)
            assert_same_bits(gpu_sort(bqs, a), oracle.sort(a))


@pytest.mark.parametrize("pivot", [0, 1])
@pytest.mark.parametrize("local", [-1, 0, 3000, 16384])
@pytest.mark.parametrize("cutoff", [16, 256, 1000, 2048, 4096])
def test_local_partition_cutoffs(bqs, cutoff, local, pivot):
    # Segments above the small cutoff and up to the local cutoff are partitioned down to
    # the small cutoff by one block in shared memory (for cutoffs of at least 256 keys);
    # 0 turns that off (every such segment is partitioned level by level in HBM).
    bqs.set_option("small_cutoff", cutoff)
    bqs.set_option("local_cutoff", local)
    bqs.set_option("pivot", pivot)
    for dtype in DTYPES:
        for n, dist in [(257, "uniform"), (2049, "reversed"), (16384, "uniform"),
                        (16385, "mod_sqrt"), (300_001, "uniform"), (100_000, "all_equal"),
                        (200_000, "swapped_1pct"), (1 << 20, "uniform")]:
            a = inputs.make_keys(n, dtype, dist, seed=n + cutoff)
            assert_same_bits(gpu_sort(bqs, a), oracle.sort(a, pivot="sqrt" if pivot else "mo3"))
            st = bqs.stats()
            assert st["equal_keys"] + st["small_keys"] + st["local_keys"] == n, (n, dist, st)
            block = 8192 if dtype == "int32" else 4096      # keys one block holds
            reach = block if local in (-1, 16384) else local
            if local != 0 and cutoff >= 256 and reach > cutoff and n == 1 << 20:
                assert st["local_segments"] > 0


@pytest.mark.parametrize("local_sort", [0, 1, 128])
@pytest.mark.parametrize("cutoff", [256, 2048, 3000, 4096])
def test_local_sort_of_the_leaves(bqs, cutoff, local_sort):
    # The single-block local partitioning sorts up to `local_sort` finished
    # sub-segments of its segment in shared memory; the others (all with 0) go back to
    # HBM for the network kernels.  1 sends almost every leaf down the second path
    # while the block sorts one, so both paths share every segment.
    bqs.set_option("small_cutoff", cutoff)
    bqs.set_option("local_cutoff", -1)
    bqs.set_option("local_sort", local_sort)
    bqs.set_option("pivot", 1)
    for dtype in DTYPES:
        for n, dist in [(8192, "uniform"), (8193, "reversed"), (300_001, "mod_sqrt"),
                        (1 << 20, "uniform"), (1 << 20, "swapped_1pct"), (77_777, "all_equal")]:
            a = inputs.make_keys(n, dtype, dist, seed=n + cutoff + local_sort)
            assert_same_bits(gpu_sort(bqs, a), oracle.sort(a, pivot="sqrt"))
            st = bqs.stats()
            assert st["equal_keys"] + st["small_keys"] + st["local_keys"] == n, (n, dist, st)


@pytest.mark.parametrize("dtype", DTYPES)
def test_local_partition_depth_fallback_and_pairs(bqs, dtype):
    import torch
    bqs.set_option("local_cutoff", -1)
    for limit in (0, 2):
        bqs.set_option("depth_limit", limit)
        for dist in ("uniform", "mod_sqrt", "all_equal"):
            a = inputs.make_keys(300_001, dtype, dist, seed=limit)
            assert_same_bits(gpu_sort(bqs, a), oracle.sort(a))
    bqs.set_option("depth_limit", -1)
    n = 1 << 20
    k = (inputs.splitmix64(21, n) % np.uint64(3000)).astype(dtype)
    v = np.arange(n, dtype=np.uint32)[np.argsort(inputs.splitmix64(22, n))].astype(np.uint32)
    tk, tv = torch.from_numpy(k).cuda(), torch.from_numpy(v.view(np.int32)).cuda()
    bqs.sort_pairs(tk, tv)
    wk, wv = oracle.sort_pairs(k, v)
    assert_same_bits(tk.cpu().numpy(), wk)
    assert_same_bits(tv.cpu().numpy().view(np.uint32), wv)
    assert bqs.stats()["local_segments"] > 0


def test_pivot_kernel_with_many_block_pivots(bqs):
    # Depth limit 0 sends every large segment to the pivot kernel's block phase; with
    # cutoff 2 a level holds far more of them than a block's list takes (64 per block),
    # so the blocks fall back to reading their entries again.
    bqs.set_option("depth_limit", 0)
    bqs.set_option("small_cutoff", 2)
    for dtype in DTYPES:
        a = inputs.make_keys(1 << 20, dtype, "uniform", seed=9)
        assert_same_bits(gpu_sort(bqs, a), oracle.sort(a))
        assert bqs.stats()["fallback_pivots"] > 64 * 8 * 152


def test_float64_special_values(bqs):
    vals = np.array([0.0, -0.0, 1.0, -1.0, np.inf, -np.inf, 5e-324, -5e-324, 2.5, -2.5,
                     np.finfo(np.float64).max, -np.finfo(np.float64).max] * 500)
    perm = np.argsort(inputs.splitmix64(1, vals.size))
    a = vals[perm]
    for cutoff in (2, 64, 2048):
        bqs.set_option("small_cutoff", cutoff)
        assert_same_bits(gpu_sort(bqs, a), oracle.sort(a))


@pytest.mark.parametrize("limit", [0, 1, 3])
@pytest.mark.parametrize("dtype", DTYPES)
def test_depth_limit_fallback(bqs, dtype, limit):
    # Past the depth limit every segment is split at the midpoint of its key range.
    bqs.set_option("depth_limit", limit)
    bqs.set_option("small_cutoff", 16)
    for dist in ("uniform", "mod_sqrt", "all_equal", "sorted"):
        a = inputs.make_keys(200_001, dtype, dist, seed=limit)
        got = gpu_sort(bqs, a)
        assert_same_bits(got, oracle.sort(a))
    assert bqs.stats()["fallback_pivots"] > 0 or dist == "all_equal"


def test_extreme_int_values(bqs):
    for dtype in ("int32", "int64"):
        info = np.iinfo(dtype)
        a = np.array([info.max, info.min, 0, -1, 1, info.max, info.min] * 3001, dtype=dtype)
        a = a[np.argsort(inputs.splitmix64(2, a.size))]
        for cutoff in (2, 2048):
            bqs.set_option("small_cutoff", cutoff)
            bqs.set_option("depth_limit", 0 if cutoff == 2 else -1)
            assert_same_bits(gpu_sort(bqs, a), oracle.sort(a))


# ---- key-value pairs --------------------------------------------------------------------

@pytest.mark.parametrize("dtype", DTYPES)
def test_sort_pairs_matches_oracle(bqs, dtype):
    import torch
    for n in (0, 1, 2, 17, 2049, 100_003, 1 << 20):
        keys = (inputs.splitmix64(5, n) % np.uint64(max(1, n // 50 + 1))).astype(dtype)
        vals = np.arange(n, dtype=np.uint32)[np.argsort(inputs.splitmix64(6, n))].astype(np.uint32)
        tk = torch.from_numpy(keys).cuda()
        tv = torch.from_numpy(vals.view(np.int32)).cuda()
        bqs.sort_pairs(tk, tv)
        wk, wv = oracle.sort_pairs(keys, vals)
        assert_same_bits(tk.cpu().numpy(), wk)
        assert_same_bits(tv.cpu().numpy().view(np.uint32), wv)


def test_sort_pairs_workload_shape_with_fallback(bqs):
    import torch
    keys, vals = inputs.make_pairs(1 << 18, seed=1)
    for limit in (-1, 2):
        bqs.set_option("depth_limit", limit)
        tk, tv = torch.from_numpy(keys).cuda(), torch.from_numpy(vals.view(np.int32)).cuda()
        bqs.sort_pairs(tk, tv)
        wk, wv = oracle.sort_pairs(keys, vals)
        assert_same_bits(tk.cpu().numpy(), wk)
        assert_same_bits(tv.cpu().numpy().view(np.uint32), wv)


# ---- partition ------------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", DTYPES)
def test_partition_split_and_sides(bqs, dtype):
    import torch
    for n in (1, 2, 100, 4096, 4097, 100_001, 1 << 20):
        a = (inputs.splitmix64(n, n) % np.uint64(1000)).astype(dtype)
        for pivot in (-5, 0, 500, 999, 1000):
            out, split = bqs.partition(torch.from_numpy(a).cuda(), pivot)
            got = out.cpu().numpy()
            want, wsplit = oracle.partition_by_value(a, pivot)
            assert split == wsplit
            assert_same_bits(np.sort(got[:split]), np.sort(want[:wsplit]))
            assert_same_bits(np.sort(got[split:]), np.sort(want[wsplit:]))
            # keys equal to the pivot come first on the right side
            neq = int(np.count_nonzero(a == pivot))
            assert np.all(got[split:split + neq] == pivot)


def test_partition_rejects_overlap(bqs):
    import torch
    t = torch.arange(1000, dtype=torch.int32, device="cuda")
    with pytest.raises(bqs.BqsError):
        bqs.partition(t, 5, out=t)


# ---- segmented ------------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", DTYPES)
def test_segmented_matches_oracle(bqs, dtype):
    import torch
    lens = [0, 1, 0, 2, 5000, 17, 0, 2048, 2049, 1, 300_000, 3, 65536, 0]
    off = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(lens, out=off[1:])
    a = inputs.make_keys(int(off[-1]), dtype, "uniform", seed=4)
    t = torch.from_numpy(a).cuda()
    bqs.sort_segmented(t, torch.from_numpy(off).cuda())
    assert_same_bits(t.cpu().numpy(), oracle.sort_segmented(a, off))


def test_segmented_log_uniform_batch(bqs):
    import torch
    keys, off = inputs.make_segments(4096, seed=2, lo=16, hi=65536)
    t = torch.from_numpy(keys).cuda()
    bqs.sort_segmented(t, torch.from_numpy(off).cuda())
    assert_same_bits(t.cpu().numpy(), oracle.sort_segmented(keys, off))


def test_segmented_rejects_decreasing_offsets(bqs):
    import torch
    t = torch.zeros(100, dtype=torch.int32, device="cuda")
    off = torch.tensor([0, 50, 40, 100], dtype=torch.int64, device="cuda")
    with pytest.raises(bqs.BqsError):
        bqs.sort_segmented(t, off)


# ---- larger sizes -----------------------------------------------------------------------------

@pytest.mark.parametrize("dist", inputs.DISTRIBUTIONS)
@pytest.mark.parametrize("dtype", DTYPES)
def test_sort_2pow24_matches_oracle(bqs, dtype, dist):
    bqs.set_option("pivot", 1)
    a = inputs.make_keys(1 << 24, dtype, dist, seed=1)
    assert_same_bits(gpu_sort(bqs, a), oracle.sort(a, pivot="sqrt"))


def test_sort_config1_median_of_3(bqs):
    # 2^20 int32 keys uniform over the full range from seed 0, median-of-3 pivots.
    bqs.set_option("pivot", 0)
    a = inputs.make_keys(1 << 20, "int32", "uniform", seed=0)
    assert_same_bits(gpu_sort(bqs, a), oracle.sort(a, pivot="mo3"))


# ---- small-segment networks ------------------------------------------------------------------

@pytest.mark.parametrize("small_sort", [0, 1])
@pytest.mark.parametrize("dtype", DTYPES)
def test_small_networks_every_length(bqs, dtype, small_sort):
    # Segments of every length 1 .. C (and again for 200 random lengths): each one goes
    # straight to a network, warp (<= 256), warp (<= 512 / 1024), group (<= 2048), the
    # larger group (<= 4096, key-only warp-group networks) or block.
    import torch
    bqs.set_option("small_sort", small_sort)
    top = 4096 if small_sort == 0 else 2048
    bqs.set_option("small_cutoff", top)
    rng = inputs.splitmix64(77, 200) % np.uint64(top)
    lens = list(range(1, top + 1)) + [int(v) + 1 for v in rng]
    off = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(lens, out=off[1:])
    for dist in ("uniform", "mod_sqrt", "reversed"):
        a = inputs.make_keys(int(off[-1]), dtype, dist, seed=small_sort + 1)
        t = torch.from_numpy(a).cuda()
        bqs.sort_segmented(t, torch.from_numpy(off).cuda())
        assert_same_bits(t.cpu().numpy(), oracle.sort_segmented(a, off))
        st = bqs.stats()
        assert st["levels"] == 0 and st["small_keys"] == a.size


@pytest.mark.parametrize("small_sort", [0, 1])
@pytest.mark.parametrize("cutoff", [300, 600, 1024, 1500, 2048, 2049, 4096])
def test_small_networks_in_full_sorts(bqs, cutoff, small_sort):
    bqs.set_option("small_sort", small_sort)
    bqs.set_option("small_cutoff", cutoff)
    for dtype in DTYPES:
        a = inputs.make_keys(1_000_003, dtype, "uniform", seed=cutoff)
        assert_same_bits(gpu_sort(bqs, a), oracle.sort(a))


def test_statistics_of_a_sort_without_partition_levels(bqs):
    # A sort that never partitions reads nothing back; its statistics must still be
    # its own, not the previous call's.
    gpu_sort(bqs, inputs.make_keys(1 << 20, "int32", "uniform", seed=1))
    assert bqs.stats()["moved_keys"] > 0
    for n in (100, 1000, 2048):
        a = inputs.make_keys(n, "int64", "uniform", seed=n)
        assert_same_bits(gpu_sort(bqs, a), oracle.sort(a))
        st = bqs.stats()
        assert st["levels"] == 0 and st["moved_keys"] == 0 and st["equal_keys"] == 0
        assert st["small_keys"] == n and st["local_keys"] == 0


def _pairs_case(dtype, n, kind, seed):
    r = inputs.splitmix64(seed, n)
    if kind == "dense":          # key range far below 2^32: every segment packs
        k = (r % np.uint64(5000)).astype(dtype)
    elif kind == "wide":         # full range: 64-bit segments do not pack
        k = r.view(np.int64).astype(dtype) if dtype != "float64" else \
            (r >> np.uint64(11)).astype(np.float64) * 2.0 ** -20 - 2.0 ** 32
    else:                        # half dense cluster, half wide: both paths in one sort
        k = np.where(r & np.uint64(1), r % np.uint64(1000), r >> np.uint64(1)).astype(np.int64)
        k = k.astype(dtype)
    v = np.arange(n, dtype=np.uint32)[np.argsort(inputs.splitmix64(seed + 1, n))].astype(np.uint32)
    return np.ascontiguousarray(k), v


@pytest.mark.parametrize("small_sort", [0, 1])
@pytest.mark.parametrize("kind", ["dense", "wide", "mixed"])
@pytest.mark.parametrize("dtype", DTYPES)
def test_pairs_packed_and_fallback_networks(bqs, dtype, kind, small_sort):
    import torch
    bqs.set_option("small_sort", small_sort)
    # (a cutoff above 2048 is clamped to 2048 for key-value sorts)
    for cutoff, n in ((300, 200_003), (1024, 1 << 20), (2048, 777_777), (4096, 300_007)):
        bqs.set_option("small_cutoff", cutoff)
        keys, vals = _pairs_case(dtype, n, kind, seed=cutoff)
        tk, tv = torch.from_numpy(keys).cuda(), torch.from_numpy(vals.view(np.int32)).cuda()
        bqs.sort_pairs(tk, tv)
        wk, wv = oracle.sort_pairs(keys, vals)
        assert_same_bits(tk.cpu().numpy(), wk)
        assert_same_bits(tv.cpu().numpy().view(np.uint32), wv)


PIVOT_RULES = {0: "median-of-3", 1: "median-of-sqrt(n)", 2: "median-of-5", 3: "median-of-23",
               4: "median-of-3-medians-of-3", 5: "median-of-3-medians-of-5",
               6: "median-of-5-medians-of-5"}


@pytest.mark.parametrize("local", [0, -1])
@pytest.mark.parametrize("rule", sorted(PIVOT_RULES))
def test_every_pivot_rule_sorts(bqs, rule, local):
    # Sec. 4's pivot rules change the recursion, never the sorted output.
    bqs.set_option("pivot", rule)
    bqs.set_option("local_cutoff", local)
    for dtype in DTYPES:
        for n, dist in [(100_000, "uniform"), (300_001, "mod_sqrt"), (1 << 20, "sorted"),
                        (70_001, "reversed"), (50_000, "all_equal"), (1 << 21, "swapped_1pct")]:
            a = inputs.make_keys(n, dtype, dist, seed=rule + 1)
            assert_same_bits(gpu_sort(bqs, a), oracle.sort(a))
            st = bqs.stats()
            assert st["equal_keys"] + st["small_keys"] + st["local_keys"] == n


@pytest.mark.parametrize("pivot", [0, 1])
@pytest.mark.parametrize("dist", inputs.EXTRA_DISTRIBUTIONS)
@pytest.mark.parametrize("dtype", DTYPES)
def test_structured_distributions(bqs, dtype, dist, pivot):
    # The duplicate-heavy and nearly sorted inputs of the paper's further experiments.
    bqs.set_option("pivot", pivot)
    for n in (300_001, 1 << 20):
        a = inputs.make_keys(n, dtype, dist, seed=n)
        assert_same_bits(gpu_sort(bqs, a), oracle.sort(a, pivot="sqrt" if pivot else "mo3"))


@pytest.mark.parametrize("cutoff", [2048, 4096])
@pytest.mark.parametrize("small_sort", [0, 1])
@pytest.mark.parametrize("dtype", DTYPES)
def test_networks_on_a_second_stream(bqs, dtype, small_sort, cutoff):
    # BQS_OPT_OVERLAP: each level's networks run beside the partition levels.
    import torch
    bqs.set_option("overlap", 1)
    bqs.set_option("small_sort", small_sort)
    bqs.set_option("small_cutoff", cutoff)
    bqs.set_option("pivot", 1)
    for n, dist in [(2049, "uniform"), (300_001, "mod_sqrt"), (1 << 22, "uniform"),
                    (1 << 20, "swapped_1pct"), (100_000, "all_equal")]:
        a = inputs.make_keys(n, dtype, dist, seed=n)
        assert_same_bits(gpu_sort(bqs, a), oracle.sort(a, pivot="sqrt"))
        st = bqs.stats()
        assert st["equal_keys"] + st["small_keys"] + st["local_keys"] == n
    keys, vals = _pairs_case(dtype, 1 << 20, "dense", seed=4)
    tk, tv = torch.from_numpy(keys).cuda(), torch.from_numpy(vals.view(np.int32)).cuda()
    bqs.sort_pairs(tk, tv)
    wk, wv = oracle.sort_pairs(keys, vals)
    assert_same_bits(tk.cpu().numpy(), wk)
    assert_same_bits(tv.cpu().numpy().view(np.uint32), wv)
    k2, off = inputs.make_segments(1000, seed=5, lo=1, hi=20_000, dtype=dtype)
    t = torch.from_numpy(k2).cuda()
    bqs.sort_segmented(t, torch.from_numpy(off).cuda())
    assert_same_bits(t.cpu().numpy(), oracle.sort_segmented(k2, off))


def test_deferred_timing_collects_every_partition_launch(bqs):
    # Timing mode 2: no call waits for its events; bqs_timing_collect sums every
    # partition launch that had work, once.
    bqs.set_option("pivot", 1)
    bqs.collect_timing()
    bqs.set_option("timing", 2)
    launches = 0
    for seed in range(3):
        a = inputs.make_keys((1 << 22) + seed, "int32", "uniform", seed=seed)
        got = gpu_sort(bqs, a)
        st = bqs.stats()
        assert st["partition_ms"] == 0 and st["partition_launches"] > 0
        launches += st["partition_launches"]
        assert_same_bits(got, oracle.sort(a))
    ms, n = bqs.collect_timing()
    assert n == launches and ms > 0
    assert bqs.collect_timing() == (0.0, 0)
    bqs.set_option("timing", 1)          # the waiting mode reports the same launches
    a = inputs.make_keys(1 << 22, "int32", "uniform", seed=0)
    gpu_sort(bqs, a)
    assert bqs.stats()["partition_ms"] > 0
