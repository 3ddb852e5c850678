"""The seeded input generators: SplitMix64 against its published outputs, and every
distribution against its definition written out directly on small n."""
import math

import numpy as np
import pytest

from paper_1604_06697_gb300 import inputs


def test_splitmix64_matches_the_published_sequence():
    # SplitMix64 from state 0 (Steele, Lea and Flood; Vigna's reference code): its
    # first outputs.
    got = [int(x) for x in inputs.splitmix64(0, 3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    # counter-based: any window equals the same outputs of the full stream
    full = inputs.splitmix64(7, 1000, stream=3)
    assert np.array_equal(inputs.splitmix64(7, 100, stream=3, start=450), full[450:550])


@pytest.mark.parametrize("n", [1, 2, 17, 1000, 4096])
def test_structured_distributions_follow_their_definitions(n):
    i = list(range(n))
    want = {
        "i_mod_sqrt": [x % max(1, math.isqrt(n)) for x in i],
        "i2_half_mod": [(x ** 2 + n // 2) % n for x in i],
        "i8_half_mod": [(x ** 8 + n // 2) % n for x in i],
        "half_01": [0 if x < n // 2 else 1 for x in i],
    }
    for dist, w in want.items():
        for dtype in inputs.DTYPES:
            a = inputs.make_keys(n, dtype, dist, seed=3)
            assert a.dtype == np.dtype(dtype) and a.tolist() == [np.dtype(dtype).type(v) for v in w], dist
    r = inputs.make_keys(n, "int64", "random_01", seed=3)
    assert set(np.unique(r).tolist()) <= {0, 1}


@pytest.mark.parametrize("dist,k", [("adj_swaps_sqrt", lambda n: math.isqrt(n)),
                                    ("adj_swaps_n", lambda n: n)])
def test_neighbour_swaps_are_a_permutation_with_few_inversions(dist, k):
    for n in (2, 50, 3000):
        a = inputs.make_keys(n, "int64", dist, seed=5)
        assert sorted(a.tolist()) == list(range(n))
        # every swap of neighbours changes the inversion count by one
        inv = sum(1 for x in range(n) for y in range(x + 1, n) if a[x] > a[y]) if n <= 50 else \
            int(np.sum([np.sum(a[x + 1:] < a[x]) for x in range(n)]))
        assert inv <= k(n) and (inv - k(n)) % 2 == 0


def test_unknown_distribution_is_rejected():
    with pytest.raises(ValueError):
        inputs.make_keys(10, "int32", "no_such")
