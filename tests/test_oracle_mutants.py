"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of the oracle source (on the CPU, in a
temporary directory), builds it, and runs the fast pins of
``test_oracle_pins.py`` against that build in a child process.  A pin must
fail (an assertion, a crash, or a run that does not end in time all count as
"caught").  The committed oracle is never modified.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "bqs_oracle.cpp")

# (name, original text, planted mistake)
MUTANTS = [
    ("left scan direction", "s.pending += step > 0 ? !lt(A[at], pivot) : !lt(pivot, A[at]);",
     "s.pending += step > 0 ? lt(A[at], pivot) : !lt(pivot, A[at]);"),
    ("right scan direction", "s.pending += step > 0 ? !lt(A[at], pivot) : !lt(pivot, A[at]);",
     "s.pending += step > 0 ? !lt(A[at], pivot) : lt(pivot, A[at]);"),
    ("left block advance", "if (left.pending == 0) begin += kB;", "if (left.pending == 0) begin += kB - 1;"),
    ("final split of the rest", "right_len = rest - left_len;\n      scan(A, pivot, begin, left_len",
     "right_len = rest - left_len - (rest > 3);\n      scan(A, pivot, begin, left_len"),
    ("compaction pivot slot", "std::swap(A[--slot], A[left.misplaced[j]]);\n      std::swap(A[home], A[slot]);",
     "std::swap(A[--slot], A[left.misplaced[j]]);\n      std::swap(A[home], A[slot - 1]);"),
    ("right compaction start", "int64_t slot = begin;", "int64_t slot = begin + 1;"),
    ("median-of-3 sample", "return median_of_3(A, b, b + len / 2, e - 1);",
     "return median_of_3(A, b, b + len / 2, e - 2);"),
    ("pivot = first element", "return median_of_3(A, b, b + len / 2, e - 1);",
     "return b;"),
    ("pivot not excluded", "stack.push_back({b, p, depth});\n          b = p + 1;",
     "stack.push_back({b, p, depth});\n          b = p;"),
    ("heap child choice", "if (child + 1 < n && lt(H[child], H[child + 1])) ++child;",
     "if (child + 1 < n && lt(H[child + 1], H[child])) ++child;"),
    ("insertion sort bound", "while (j > b && lt(x, A[j - 1]))",
     "while (j > b + 1 && lt(x, A[j - 1]))"),
    ("float64 order of negatives", "return (u >> 63) ? ~u : (u | (uint64_t(1) << 63));",
     "return (u >> 63) ? (u ^ (uint64_t(1) << 63)) : (u | (uint64_t(1) << 63));"),
    ("payload tie-break", "return a.val < b.val;", "return a.val > b.val;"),
    ("sample median rank", "size_t mid = (pos.size() - 1) / 2;",
     "size_t mid = (pos.size() - 1) / 4;"),
    ("depth limit", "2 * floor_log2(n) + 3", "2 * floor_log2(n) + 300"),
    ("value partition", "else out[hi++] = keys[i];", "else out[hi++] = pivot;"),
    ("order statistic index", "*(int32_t*)out = a[k];", "*(int32_t*)out = a[k > 0 ? k - 1 : k];"),
    ("record norm components", "for (int32_t c = 0; c < count; ++c) {\n        double x;",
     "for (int32_t c = 1; c < count; ++c) {\n        double x;"),
    ("record key field", "std::memcpy(&v, r, 4);", "std::memcpy(&v, r + 4, 4);"),
    # the pivot rules of Sec. 4: group size, sample positions, the 20000 switch, sample size
    ("mo5-of-mo5 groups of three", "p.begin() + 5 * g, p.begin() + 5 * g + 5)",
     "p.begin() + 5 * g, p.begin() + 5 * g + 3)"),
    ("sample positions i*len/k", "p[i] = b + ((2 * i + 1) * len) / (2 * k);",
     "p[i] = b + (i * len) / k;"),
    ("sqrt switch at 2000", "if (len < 20000) return median_of_5_medians_of_5(A, b, len);",
     "if (len < 2000) return median_of_5_medians_of_5(A, b, len);"),
    ("sqrt switch at or above 20000", "if (len < 20000) return median_of_5_medians_of_5(A, b, len);",
     "if (len <= 20000) return median_of_5_medians_of_5(A, b, len);"),
    ("half-size sqrt sample", "spaced(b, len, isqrt(len) | 1)", "spaced(b, len, (isqrt(len) / 2) | 1)"),
    ("sample offset dropped", "p[i] = b + ((2 * i + 1) * len) / (2 * k);",
     "p[i] = ((2 * i + 1) * len) / (2 * k);"),
    ("mo3 switch below 64", "if (pivot_rule == kMedianOf3 || len < 64) {",
     "if (pivot_rule == kMedianOf3 || len < 32) {"),
]

_RUNNER = r"""
import sys
sys.path.insert(0, {root!r})
sys.path.insert(0, {tests!r})
import oracle
oracle.use_library({so!r})
import test_oracle_pins as P
pins = [
    lambda: P.test_all_permutations_sort_to_identity("int32", 2, "mo3"),
    lambda: P.test_all_permutations_sort_to_identity("int64", 2, "sqrt"),
    lambda: P.test_all_ternary_words_sort_to_counts(16),
    lambda: P.test_float64_total_order_special_values(),
    lambda: P.test_pairs_match_lexsort("int64"),
    lambda: P.test_block_partition_invariants_every_length("few"),
    lambda: P.test_block_partition_invariants_every_length("random"),
    lambda: P.test_distributions_match_library_sort("int32", "uniform", "sqrt"),
    lambda: P.test_median_of_3_comparison_slope(),
    lambda: P.test_median_of_sqrt_comparison_slope(),
    lambda: P.test_shallow_depth_limit_switches_subarrays_to_heapsort(),
    lambda: P.test_default_depth_limit_not_reached_on_random_input(),
    lambda: P.test_partition_by_value_definition("int32"),
    lambda: P.test_block_partition_large_and_compares_each_element_once(),
    lambda: P.test_default_depth_limit_is_the_papers(1 << 10),
    lambda: P.test_select_is_the_order_statistic("int32"),
    lambda: P.test_record_keys_follow_their_definition(),
    lambda: P.test_sqrt_sample_size_and_positions(0, 1000),
    lambda: P.test_sqrt_sample_size_and_positions(1, 0),
    lambda: P.test_median_of_5_medians_of_5_below_20000(0, 333),
    lambda: P.test_median_of_5_medians_of_5_below_20000(1, 0),
    lambda: P.test_median_of_5_medians_of_5_below_20000(3, 0),
    lambda: P.test_sqrt_rule_takes_over_at_20000(),
    lambda: P.test_median_of_3_sample(0),
]
for i, pin in enumerate(pins):
    try:
        pin()
    except AssertionError:
        print("caught by pin", i)
        sys.exit(3)
print("not caught")
sys.exit(0)
"""


@pytest.mark.parametrize("name,orig,bad", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(name, orig, bad, tmp_path):
    src = open(SRC).read()
    assert src.count(orig) == 1, f"mutation site for {name!r} not found exactly once"
    mutant = tmp_path / "mutant.cpp"
    mutant.write_text(src.replace(orig, bad))
    so = tmp_path / "mutant.so"
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", str(mutant), "-o", str(so)])
    code = _RUNNER.format(root=ROOT, tests=os.path.join(ROOT, "tests"), so=str(so))
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=240)
    except subprocess.TimeoutExpired:
        return  # a planted mistake that makes the oracle loop forever is caught too
    assert r.returncode != 0, f"planted mistake {name!r} passed every pin:\n{r.stdout}{r.stderr}"
