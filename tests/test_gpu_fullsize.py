"""Parity at the configurations' own sizes, in the launch configuration bench.py times
(sqrt(n) pivot, autotuned launch shape), against the oracle.

* The headline input (2^28 int32 uniform, seed 1): byte for byte against the
  oracle's sort of it, in this process.
* The other 17 dtype x distribution cases at 2^28 (seed 1), 2^26 key-value pairs
  (int64 keys mod 2^20, payload = index, seed 1) and the batch of 65,536 segments
  (log-uniform lengths in [16, 65536], seed 2, sorted by one replay of a captured
  bqs_sort_batched): the BLAKE2b-256 digest of the GPU's output bytes against the
  digest of the oracle's output for the same seeded input.  The oracle runs for
  these are started at once in a pool of spawned worker processes (see
  tests/_oracle_jobs.py), so they proceed on the host cores while the GPU sorts.
  Equal digests mean equal bytes (collision probability 2^-256).
* Cheap properties on every case as well: non-decreasing order on the device.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1604_06697_gb300 import inputs

import _oracle_jobs as jobs

pytestmark = pytest.mark.gpu

N = 1 << 28
HEADLINE = ("int32", "uniform")
CASES = [(d, s) for d in ("int32", "int64", "float64") for s in inputs.DISTRIBUTIONS]
PAIRS_N = 1 << 26
NSEG = 65536


def _workers() -> int:
    """Oracle workers: each holds up to two copies of a 2 GiB input."""
    try:
        with open("/proc/meminfo") as f:
            avail = next(int(l.split()[1]) for l in f if l.startswith("MemAvailable")) << 10
    except Exception:
        avail = 16 << 30
    by_mem = int(avail // (7 << 30))
    return max(1, min(6, (os.cpu_count() or 2) - 2, by_mem))


@pytest.fixture(scope="module")
def digests():
    """Starts every oracle run of this module in spawned workers; maps case -> result."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(_workers())
    out = {}
    # longest jobs first
    out["segments"] = pool.apply_async(jobs.segmented_job, (NSEG, 2, "sqrt"))
    out["pairs"] = pool.apply_async(jobs.pairs_job, (PAIRS_N, 1, "sqrt"))
    for dtype, dist in CASES:
        if (dtype, dist) != HEADLINE:
            out[(dtype, dist)] = pool.apply_async(jobs.sort_job, (N, dtype, dist, 1, "sqrt"))
    pool.close()
    yield out
    pool.terminate()
    pool.join()


@pytest.fixture(scope="module")
def bqs():
    import torch
    from paper_1604_06697_gb300 import build
    build.build()
    import paper_1604_06697_gb300 as m
    torch.cuda.init()
    return m


def _gpu_sorted(bqs, dtype, a):
    """Sorts a in the bench's launch configuration; returns the device result."""
    import torch
    from paper_1604_06697_gb300 import autotune
    bqs.set_option("pivot", 1)
    autotune.tune(dtype, a.size, kind="sort")
    t = torch.from_numpy(a).cuda()
    bqs.sort(t)
    torch.cuda.synchronize()
    if dtype == "float64":
        o = t.view(torch.int64)
        # signed image of ord(): non-negative floats keep their bits, negative ones get
        # their complemented bits with the sign bit set (so -0.0 -> -1 < +0.0 -> 0)
        o = torch.where(o < 0, ~o | torch.iinfo(torch.int64).min, o)
        assert bool((o[1:] >= o[:-1]).all())
    else:
        assert bool((t[1:] >= t[:-1]).all())
    return t


def test_headline_input_byte_for_byte(bqs, digests):
    dtype, dist = HEADLINE
    a = inputs.make_keys(N, dtype, dist, seed=1)
    got = _gpu_sorted(bqs, dtype, a).cpu().numpy()
    oracle.sort_inplace(a, pivot="sqrt")
    assert np.array_equal(got.view(np.uint8), a.view(np.uint8))


@pytest.mark.parametrize("dtype,dist", [c for c in CASES if c != HEADLINE])
def test_full_size_sort_matches_oracle(bqs, digests, dtype, dist):
    a = inputs.make_keys(N, dtype, dist, seed=1)
    t = _gpu_sorted(bqs, dtype, a)
    del a
    got = t.cpu().numpy()
    del t
    assert jobs.digest(got) == digests[(dtype, dist)].get(timeout=3000), (dtype, dist)


def test_pairs_at_2p26_match_oracle(bqs, digests):
    import torch
    from paper_1604_06697_gb300 import autotune
    k, v = inputs.make_pairs(PAIRS_N, seed=1)
    bqs.set_option("pivot", 1)
    autotune.tune("int64", PAIRS_N, kind="pairs")
    tk = torch.from_numpy(k).cuda()
    tv = torch.from_numpy(v.view(np.int32)).cuda()
    bqs.sort_pairs(tk, tv)
    torch.cuda.synchronize()
    gk, gv = tk.cpu().numpy(), tv.cpu().numpy().view(np.uint32)
    assert jobs.digest(gk, gv) == digests["pairs"].get(timeout=3000)


def test_65536_segments_in_one_graph_replay_match_oracle(bqs, digests):
    import torch
    from paper_1604_06697_gb300 import autotune
    keys, off = inputs.make_segments(NSEG, seed=2)
    n = int(off[-1])
    bqs.set_option("pivot", 1)
    autotune.tune("int32", n, kind="batched", nseg=NSEG)
    src = torch.from_numpy(keys).cuda()
    toff = torch.from_numpy(off).cuda()
    work = src.clone()
    bqs.sort_batched(work, toff)           # one-time set-up outside capture
    torch.cuda.synchronize()
    work.copy_(src)
    g = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream()
    with torch.cuda.graph(g, stream=cap):
        bqs.sort_batched(work, toff)
    work.copy_(src)
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    got = work.cpu().numpy()
    assert jobs.digest(got) == digests["segments"].get(timeout=3000)
    # and a second replay on a fresh copy gives the same bytes
    work.copy_(src)
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(work.cpu().numpy(), got)
