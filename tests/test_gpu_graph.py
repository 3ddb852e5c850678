"""Sorts captured into a CUDA graph: the level loop becomes a device-side loop.

A capture records the whole sort (scratch allocation, first work lists, the
conditional while loop over levels, scratch release); replaying the graph must
give the oracle's result, replay after replay.
"""
import numpy as np
import pytest

import oracle
from paper_1604_06697_gb300 import inputs

pytestmark = pytest.mark.gpu


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
    saved = {k: bqs.get_option(k) for k in bqs.OPTIONS}
    yield
    for k, v in saved.items():
        bqs.set_option(k, v)


def _bits(a):
    return a.view(np.uint32 if a.itemsize == 4 else np.uint64)


def _capture(fn):
    import torch
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fn()                      # ordinary call first: one-time set-up outside capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        fn()
    return g


@pytest.mark.parametrize("local", [0, -1])
@pytest.mark.parametrize("dtype", ["int32", "int64", "float64"])
def test_captured_sort_replays(bqs, dtype, local):
    import torch
    bqs.set_option("pivot", 1)
    bqs.set_option("local_cutoff", local)
    for n, dist in [(1 << 20, "uniform"), (100_003, "mod_sqrt"), (3000, "reversed")]:
        a = inputs.make_keys(n, dtype, dist, seed=n)
        src = torch.from_numpy(a).cuda()
        work = torch.empty_like(src)
        g = _capture(lambda: (work.copy_(src), bqs.sort(work)))
        want = oracle.sort(a)
        for _ in range(3):
            work.zero_()
            g.replay()
            torch.cuda.synchronize()
            assert np.array_equal(_bits(work.cpu().numpy()), _bits(want))


def test_captured_pairs_replay(bqs):
    import torch
    keys, vals = inputs.make_pairs(1 << 18, seed=1)
    sk, sv = torch.from_numpy(keys).cuda(), torch.from_numpy(vals.view(np.int32)).cuda()
    wk, wv = torch.empty_like(sk), torch.empty_like(sv)
    g = _capture(lambda: (wk.copy_(sk), wv.copy_(sv), bqs.sort_pairs(wk, wv)))
    ok, ov = oracle.sort_pairs(keys, vals)
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(wk.cpu().numpy(), ok)
        assert np.array_equal(wv.cpu().numpy().view(np.uint32), ov)


@pytest.mark.parametrize("dtype", ["int32", "float64"])
def test_captured_batched_segments(bqs, dtype):
    import torch
    keys, off = inputs.make_segments(2000, seed=2, lo=16, hi=65536, dtype=dtype)
    src = torch.from_numpy(keys).cuda()
    toff = torch.from_numpy(off).cuda()
    work = torch.empty_like(src)
    g = _capture(lambda: (work.copy_(src), bqs.sort_batched(work, toff)))
    want = oracle.sort_segmented(keys, off)
    for _ in range(2):
        work.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(_bits(work.cpu().numpy()), _bits(want))


def test_batched_outside_capture_matches_segmented(bqs):
    import torch
    keys, off = inputs.make_segments(500, seed=5, lo=1, hi=40000)
    t1 = torch.from_numpy(keys).cuda()
    t2 = t1.clone()
    toff = torch.from_numpy(off).cuda()
    bqs.sort_batched(t1, toff)
    bqs.sort_segmented(t2, toff)
    torch.cuda.synchronize()
    assert torch.equal(t1, t2)
    assert np.array_equal(t1.cpu().numpy(), oracle.sort_segmented(keys, off))
