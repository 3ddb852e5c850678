"""Index arithmetic of the pivot kernel's work split, checked on the host.

k_pivot's warps visit the entries i = b + w*G + k*G*nw of the pivot list (block b of
G, warp w of nw, k = 0, 1, ...); the segments that need the whole block go on block
b's list, and when that list overflows the block reads the entries i = b + r*G
(r = 0, 1, ...) again.  Both must be the same set for every block, and the blocks'
sets must split the list exactly once.
"""
import pytest


def warp_phase(b, G, nw, count):
    out = []
    for w in range(nw):
        i = b + w * G
        while i < count:
            out.append(i)
            i += G * nw
    return out


def fallback_pass(b, G, count):
    rounds = (count + G - 1) // G
    return [b + r * G for r in range(rounds) if b + r * G < count]


@pytest.mark.parametrize("G,nw", [(1, 8), (3, 8), (1216, 8), (7, 4)])
@pytest.mark.parametrize("count", [0, 1, 5, 8, 1215, 1216, 1217, 9728, 9729, 20001])
def test_pivot_kernel_entries_split_exactly_once(G, nw, count):
    seen = []
    for b in range(G):
        mine = warp_phase(b, G, nw, count)
        assert sorted(mine) == fallback_pass(b, G, count)
        seen += mine
    assert sorted(seen) == list(range(count))
