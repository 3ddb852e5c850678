"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself.  Each test checks one part of
the oracle against an independent fact:

* brute force over every input of a tiny domain, whose sorted output has a
  closed form (identity for a permutation, counts for {0,1,2} words);
* a pure-Python Insertionsort and numpy's sort (library routines that compute
  the definition of "sorted") on every size up to 2000;
* the invariants that define a partition (Sec. 2: smaller-or-equal left of the
  returned position, greater-or-equal right of it) for Algorithm 3 at every
  length 1..600, including every branch of its final scan;
* the average comparison count of median-of-three Quicksort, (12/7) n ln n =
  1.188 n log2 n + O(n) (Sec. 3 "Analysis": block partitioning keeps the
  comparisons of median-of-three Quicksort), and of a median-of-sqrt(n) sample,
  whose leading term tends to n log2 n (Sec. 2, Martinez & Roura);
* the Introsort switch to Heapsort at the depth limit (Sec. 2).
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_1604_06697_gb300 import inputs

DTYPES = ["int32", "int64", "float64"]


def _sorted_bits(a):
    """Byte view of an array for bit-exact comparisons."""
    return np.ascontiguousarray(a).view(np.uint8)


def _py_insertion_sort(xs):
    xs = list(xs)
    for i in range(1, len(xs)):
        x = xs[i]
        j = i
        while j > 0 and x < xs[j - 1]:
            xs[j] = xs[j - 1]
            j -= 1
        xs[j] = x
    return xs


# ---- brute force on tiny inputs ------------------------------------------------------

@pytest.mark.parametrize("pivot", ["mo3", "sqrt"])
@pytest.mark.parametrize("is_thresh", [2, 16])
@pytest.mark.parametrize("dtype", DTYPES)
def test_all_permutations_sort_to_identity(dtype, is_thresh, pivot):
    # is_thresh=2 forces block partitions even on 3..7 elements; 16 is the paper's.
    for n in range(0, 8):
        ident = np.arange(n).astype(dtype)
        for perm in itertools.permutations(range(n)):
            got = oracle.sort(np.array(perm).astype(dtype), pivot=pivot, is_thresh=is_thresh)
            assert np.array_equal(got, ident), (n, perm)


def test_all_permutations_n8_with_partitions():
    ident = np.arange(8, dtype=np.int32)
    for perm in itertools.permutations(range(8)):
        got = oracle.sort(np.array(perm, dtype=np.int32), is_thresh=2)
        assert np.array_equal(got, ident), perm


@pytest.mark.parametrize("is_thresh", [2, 16])
def test_all_ternary_words_sort_to_counts(is_thresh):
    # Every word over {0,1,2} of length <= 8: the sorted output is c0 zeros, c1 ones,
    # c2 twos (covers all-equal and two-valued multisets as special cases).
    for n in range(0, 9):
        for word in itertools.product((0, 1, 2), repeat=n):
            a = np.array(word, dtype=np.int32)
            c = [word.count(v) for v in (0, 1, 2)]
            want = np.array([0] * c[0] + [1] * c[1] + [2] * c[2], dtype=np.int32)
            assert np.array_equal(oracle.sort(a, is_thresh=is_thresh), want), word


# ---- agreement with Insertionsort / library sort on every small size -----------------

def test_every_size_up_to_2000_matches_library_sort():
    for n in range(0, 2001):
        a = (inputs.splitmix64(7, n) % np.uint64(max(1, n // 3 + 1))).astype(np.int32)
        assert np.array_equal(oracle.sort(a), np.sort(a, kind="stable")), n


@pytest.mark.parametrize("n", [0, 1, 2, 17, 129, 257, 700, 2000])
def test_matches_pure_python_insertion_sort(n):
    a = (inputs.splitmix64(11, n) % np.uint64(50)).astype(np.int64)
    assert oracle.sort(a, pivot="sqrt").tolist() == _py_insertion_sort(a.tolist())
    assert oracle.sort(a, pivot="mo3").tolist() == _py_insertion_sort(a.tolist())


@pytest.mark.parametrize("dist", inputs.DISTRIBUTIONS)
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("pivot", ["mo3", "sqrt"])
def test_distributions_match_library_sort(dtype, dist, pivot):
    for n in (1000, 50_000, 200_001):
        a = inputs.make_keys(n, dtype, dist, seed=1)
        got = oracle.sort(a, pivot=pivot)
        # numpy orders non-NaN floats by IEEE "<"; the generators emit no -0.0, so the
        # total order used for float64 coincides with it here.
        assert np.array_equal(_sorted_bits(got), _sorted_bits(np.sort(a, kind="stable")))


# ---- float64 total order ---------------------------------------------------------------

def test_float64_total_order_special_values():
    vals = [0.0, -0.0, 1.0, -1.0, np.inf, -np.inf, 5e-324, -5e-324, 2.5, -2.5,
            np.finfo(np.float64).max, -np.finfo(np.float64).max, 0.0, -0.0]
    a = np.array(vals, dtype=np.float64)
    want = np.array([-np.inf, -np.finfo(np.float64).max, -2.5, -1.0, -5e-324, -0.0, -0.0,
                     0.0, 0.0, 5e-324, 1.0, 2.5, np.finfo(np.float64).max, np.inf])
    for pivot in ("mo3", "sqrt"):
        for th in (2, 16):
            got = oracle.sort(a, pivot=pivot, is_thresh=th)
            assert np.array_equal(got.view(np.uint64), want.view(np.uint64))


def test_float64_signed_zero_is_ordered_before_positive_zero_at_scale():
    n = 100_000
    bits = np.where(inputs.splitmix64(5, n) & np.uint64(1), np.float64(-0.0), np.float64(0.0))
    got = oracle.sort(bits)
    nneg = int(np.count_nonzero(np.signbit(bits)))
    assert np.all(np.signbit(got[:nneg])) and not np.any(np.signbit(got[nneg:]))


# ---- key-value pairs ---------------------------------------------------------------------

@pytest.mark.parametrize("dtype", DTYPES)
def test_pairs_match_lexsort(dtype):
    n = 100_000
    keys = (inputs.splitmix64(3, n) % np.uint64(1000)).astype(dtype)
    vals = (inputs.splitmix64(4, n) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    k, v = oracle.sort_pairs(keys, vals)
    order = np.lexsort((vals, keys))       # last key is primary: (key, payload)
    assert np.array_equal(k, keys[order]) and np.array_equal(v, vals[order])


def test_pairs_workload_shape():
    keys, vals = inputs.make_pairs(1 << 16, seed=1)
    k, v = oracle.sort_pairs(keys, vals)
    order = np.lexsort((vals, keys))
    assert np.array_equal(k, keys[order]) and np.array_equal(v, vals[order])


# ---- Algorithm 3: partition invariants -------------------------------------------------

def _check_partition(a, p, before):
    pivot = a[p]
    assert np.all(a[:p] <= pivot) and np.all(a[p + 1:] >= pivot)
    assert np.array_equal(np.sort(a), np.sort(before))


@pytest.mark.parametrize("kind", ["random", "few", "equal", "sorted", "reversed"])
def test_block_partition_invariants_every_length(kind):
    for n in range(1, 601):
        if kind == "random":
            a = inputs.splitmix64(n, n).view(np.int64).copy()
        elif kind == "few":
            a = (inputs.splitmix64(n, n) % np.uint64(3)).astype(np.int64)
        elif kind == "equal":
            a = np.full(n, 9, dtype=np.int64)
        elif kind == "sorted":
            a = np.arange(n, dtype=np.int64)
        else:
            a = np.arange(n, 0, -1, dtype=np.int64)
        for piv in {0, n // 2, n - 1, int(inputs.splitmix64(n + 1000, 1)[0] % np.uint64(n))}:
            out, p = oracle.block_partition(a, piv)
            assert out[p] == a[piv]
            _check_partition(out, p, a)


def test_block_partition_large_and_compares_each_element_once():
    for n in (5000, 65_537, 1_000_003):
        a = inputs.make_keys(n, "int32", "uniform", seed=n)
        out, p, ncmp = oracle.block_partition(a, n // 3, counters=True)
        _check_partition(out, p, a)
        # Sec. 3: every element of the window is compared with the pivot once (the
        # pivot itself is parked outside the scans).
        assert ncmp == n - 1
        pv = a[n // 3]
        assert int(np.count_nonzero(a < pv)) <= p < int(np.count_nonzero(a <= pv))


# ---- comparison counts (Sec. 3 "Analysis") ------------------------------------------------

def _mean_comparisons_per_key(pivot, lg, seeds=3):
    n = 1 << lg
    out = []
    for s in range(seeds):
        perm = np.argsort(inputs.splitmix64(100 + s, n)).astype(np.int32)
        _, c = oracle.sort(perm, pivot=pivot, counters=True)
        out.append(c["comparisons"] / n)
    return float(np.mean(out))


def _golden():
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")) as f:
        return json.load(f)


def test_median_of_3_comparison_slope():
    # Average comparisons of median-of-three Quicksort: 1.18 n log2 n + O(n) as the
    # paper prints it ((12/7) n ln n = 1.188 n log2 n).  A random pivot would give
    # 2 ln 2 = 1.386; a partitioner that compares elements twice would double it.
    g = _golden()["mo3_comparisons_per_n_log2n"]
    lgs = list(range(14, 22))
    ys = [_mean_comparisons_per_key("mo3", lg) for lg in lgs]
    slope = np.polyfit(lgs, ys, 1)[0]
    assert abs(slope - g["value"]) < g["tolerance"], slope
    assert abs(12 / 7 * math.log(2) - g["value"]) < 0.01


def test_insertion_sort_threshold_is_the_papers():
    m = _golden()["insertion_sort_max_len"]["value"]
    for n in (m, m + 1):
        a = inputs.make_keys(n, "int64", "uniform", seed=n)
        got, c = oracle.sort(a, counters=True)
        assert np.array_equal(got, np.sort(a))
        # at most m keys: Insertionsort directly; one more: one partition first
        assert c["partitions"] == (0 if n == m else 1), (n, c)


def test_depth_limit_golden_cases():
    for n, want in _golden()["depth_limit"]["cases"].items():
        a = inputs.make_keys(int(n), "int32", "uniform", seed=1)
        _, c = oracle.sort(a, counters=True)
        assert c["depth_limit"] == want, (n, c["depth_limit"])


def test_median_of_sqrt_comparison_slope():
    # With a sample of growing size the leading term tends to n log2 n.
    lgs = list(range(14, 22))
    ys = [_mean_comparisons_per_key("sqrt", lg) for lg in lgs]
    slope = np.polyfit(lgs, ys, 1)[0]
    assert 0.95 < slope < 1.07, slope


# ---- Introsort depth limit ------------------------------------------------------------------

def test_depth_limit_zero_is_pure_heapsort():
    a = inputs.make_keys(30_000, "int64", "uniform", seed=9)
    got, c = oracle.sort(a, depth_limit=0, counters=True)
    assert np.array_equal(got, np.sort(a))
    assert c["heap_sorts"] == 1 and c["partitions"] == 0


def test_shallow_depth_limit_switches_subarrays_to_heapsort():
    a = inputs.make_keys(200_000, "float64", "mod_sqrt", seed=9)
    got, c = oracle.sort(a, depth_limit=3, counters=True)
    assert np.array_equal(got, np.sort(a))
    assert c["heap_sorts"] > 0 and c["partitions"] > 0


@pytest.mark.parametrize("n", [17, 100, 1 << 10, (1 << 14) + 5, 1 << 18])
def test_default_depth_limit_is_the_papers(n):
    # Sec. 2 states the limit 2 log n + 3 (log = log2, floored as in Appendix B's ilogb).
    a = inputs.make_keys(n, "int32", "uniform", seed=n)
    _, c = oracle.sort(a, counters=True)
    assert c["depth_limit"] == 2 * (n.bit_length() - 1) + 3


@pytest.mark.parametrize("limit", [1, 2, 4, 6])
def test_heapsort_starts_exactly_at_the_limit(limit):
    # Without a limit, record how deep partitioning goes; with a smaller limit no
    # partition may run deeper, and Heapsort must take over the unfinished parts.
    a = inputs.make_keys(5000, "int64", "uniform", seed=limit)
    _, free = oracle.sort(a, counters=True)
    got, c = oracle.sort(a, depth_limit=limit, counters=True)
    assert np.array_equal(got, np.sort(a))
    assert c["max_depth"] == min(limit, free["max_depth"])
    assert (c["heap_sorts"] > 0) == (free["max_depth"] > limit)


def test_default_depth_limit_not_reached_on_random_input():
    a = inputs.make_keys(1 << 18, "int32", "uniform", seed=9)
    _, c = oracle.sort(a, counters=True)
    assert c["heap_sorts"] == 0


# ---- value partition (the definition behind bqs_partition) ----------------------------------

@pytest.mark.parametrize("dtype", DTYPES)
def test_partition_by_value_definition(dtype):
    for n in (0, 1, 5, 1000, 4097):
        a = (inputs.splitmix64(n, n) % np.uint64(17)).astype(dtype)
        for pv in (-1, 0, 8, 16, 17):
            out, s = oracle.partition_by_value(a, pv)
            assert s == int(np.count_nonzero(a < pv))
            assert np.array_equal(out[:s], a[a < pv]) and np.array_equal(out[s:], a[a >= pv])


@pytest.mark.parametrize("dtype", DTYPES)
def test_select_is_the_order_statistic(dtype):
    # v is the k-th order statistic iff count(x < v) <= k < count(x <= v) (under the
    # total order; for float64 ord() makes -0.0 < +0.0).
    for n in (1, 2, 7, 100, 1001):
        a = (inputs.splitmix64(n, n) % np.uint64(13)).astype(dtype)
        if dtype == "float64":
            a = np.where(a == 0, np.float64(-0.0), a)
            a[: n // 3] = 0.0
        key = oracle.ord_f64(a) if dtype == "float64" else a
        for k in range(n):
            v = oracle.select(a, k)
            kv = oracle.ord_f64(np.array([v]))[0] if dtype == "float64" else v
            assert int(np.count_nonzero(key < kv)) <= k < int(np.count_nonzero(key <= kv))


def test_segmented_is_per_segment_sort():
    keys, off = inputs.make_segments(64, seed=2, lo=16, hi=4096)
    got = oracle.sort_segmented(keys, off)
    for i in range(64):
        assert np.array_equal(got[off[i]:off[i + 1]], np.sort(keys[off[i]:off[i + 1]]))


# ---- wide element types (Sec. 4, "Different Element Types") ------------------------------

def _records(n, rb, seed, kind):
    r = inputs.splitmix64(seed, n * rb // 4)
    rec = (r & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.uint8).copy()
    if kind == 0:       # Record: first field with many ties
        f = rec.view(np.int32).reshape(n, rb // 4)
        f[:, 0] = (inputs.splitmix64(seed + 1, n) % np.uint64(max(1, n // 4))).astype(np.int32)
    else:               # Vector: doubles in [-1, 1), some vectors repeated (equal norms)
        v = rec.view(np.float64).reshape(n, rb // 8)
        v[:] = 2.0 * inputs.unit_double(inputs.splitmix64(seed + 2, v.size)).reshape(v.shape) - 1.0
        v[1::7] = v[0::7][: v[1::7].shape[0]]
    return rec


def test_record_keys_follow_their_definition():
    rb = 84
    rec = _records(500, rb, 1, 0)
    keys = oracle.record_keys(rec, rb, 0)
    assert np.array_equal(keys, rec.view(np.int32).reshape(500, 21)[:, 0])
    rb = 80
    rec = _records(300, rb, 2, 1)
    keys = oracle.record_keys(rec, rb, 1, 0, 10)
    v = rec.view(np.float64).reshape(300, 10)
    for i in range(300):
        s = 0.0
        for c in range(10):      # Python floats: every product and sum rounded on its own
            s = s + v[i, c] * v[i, c]
        assert keys[i] == s
    assert oracle.record_keys(rec, rb, 1, 16, 3)[5] == sum(x * x for x in v[5, 2:5])


@pytest.mark.parametrize("kind,rb,count", [(0, 84, 1), (1, 80, 10)])
def test_sorted_records_are_ordered_by_key_then_position(kind, rb, count):
    n = 2000
    rec = _records(n, rb, 7, kind)
    got = oracle.sort_records(rec, rb, kind, 0, count).reshape(n, rb)
    keys = oracle.record_keys(rec, rb, kind, 0, count)
    order = sorted(range(n), key=lambda i: (keys[i], i))
    assert np.array_equal(got, rec.reshape(n, rb)[order])


# ---- pivot rules on hand-worked samples (Sec. 2; Sec. 4 "Different Pivot Selection Methods") ----
#
# tests/golden/pivot_samples.json lists, for a few lengths, the positions the rules
# sample (derived by hand there) and values to plant at them in an otherwise all-zero
# array.  A rule that samples other positions, groups them otherwise, sizes its sample
# otherwise or switches at another length sees mostly zeros or other groups, and
# returns another pivot.

def _pivot_golden():
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "pivot_samples.json")) as f:
        return json.load(f)


def _planted(length, b, positions, values, dtype="int32", total_pad=37):
    a = np.zeros(b + length + total_pad, dtype=dtype)
    for p, v in zip(positions, values):
        assert 0 <= p < length
        a[b + p] = v
    return a


@pytest.mark.parametrize("b", [0, 1000])
@pytest.mark.parametrize("case", [0, 1])
def test_sqrt_sample_size_and_positions(case, b):
    g = _pivot_golden()["sqrt_sample"][case]
    k, stride = g["k"], g["stride"]
    positions = [stride * (2 * i + 1) for i in range(k)]
    values = [1 + (37 * i) % k for i in range(k)]
    for dtype in DTYPES:
        a = _planted(g["len"], b, positions, values, dtype)
        got = oracle.pivot_value(a, b, b + g["len"], "sqrt")
        assert got == g["pivot"], (g["len"], b, dtype, got)


@pytest.mark.parametrize("b", [0, 333])
@pytest.mark.parametrize("case", [0, 1, 2, 3])
def test_median_of_5_medians_of_5_below_20000(case, b):
    g = _pivot_golden()["mo5_of_mo5"]
    c = g["cases"][case]
    if "stride" in c:
        positions = [c["stride"] * (2 * i + 1) + c["shift"] for i in range(25)]
    else:
        positions = c["positions"]
    a = _planted(c["len"], b, positions, g["values"])
    got = oracle.pivot_value(a, b, b + c["len"], c["rule"])
    assert got == g["pivot"], (c["len"], b, got)


def test_sqrt_rule_takes_over_at_20000():
    g, s = _pivot_golden()["mo5_of_mo5"], _pivot_golden()["switch_at_20000"]
    positions = [s["stride"] * (2 * i + 1) + s["shift"] for i in range(25)]
    a = _planted(s["len"], 0, positions, g["values"])
    assert oracle.pivot_value(a, 0, s["len"], "sqrt") == s["pivot"]
    # the same planted values one element shorter are read as median-of-5-medians-of-5
    # (19999: positions 400 (2i+1) - 1)
    c = g["cases"][2]
    positions = [c["stride"] * (2 * i + 1) + c["shift"] for i in range(25)]
    a = _planted(c["len"], 0, positions, g["values"])
    assert oracle.pivot_value(a, 0, c["len"], "sqrt") == g["pivot"]


@pytest.mark.parametrize("case", [0, 1])
def test_median_of_3_sample(case):
    c = _pivot_golden()["mo3"][case]
    for b in (0, 70):
        a = _planted(c["len"], b, c["positions"], c["values"])
        assert oracle.pivot_value(a, b, b + c["len"], c["rule"]) == c["pivot"]
