"""Serving loop: admission, batching and latency accounting (CPU), and on the GPU the
check that every request's result is the same alone and in the mix."""
import collections

import numpy as np
import pytest

from paper_1604_06697_gb300 import serving


def test_admission_respects_budget_and_tracks_peak():
    a = serving.Admission(1000)
    assert a.try_admit(600)
    assert not a.try_admit(500)       # would exceed the budget: waits
    assert a.try_admit(400)
    assert a.used == 1000 and a.peak == 1000
    a.release(600)
    assert a.try_admit(500)
    with pytest.raises(ValueError):
        a.try_admit(2000)             # can never fit


def test_form_batch_takes_oldest_dtype_in_order_within_cap():
    R = serving.Request
    q = collections.deque([R(0, 0.0, 100, "int32"), R(1, 0.1, 50, "int64"),
                           R(2, 0.2, 300, "int32"), R(3, 0.3, 10, "int32"),
                           R(4, 0.4, 20, "int64")])
    b = serving.form_batch(q, max_batch_keys=420)
    assert [r.rid for r in b] == [0, 2, 3]
    assert [r.rid for r in q] == [1, 4]            # others keep their order
    b = serving.form_batch(q, max_batch_keys=10)   # the oldest is always taken
    assert [r.rid for r in b] == [1] and [r.rid for r in q] == [4]


def test_percentile_and_request_stream():
    assert serving.percentile([1, 2, 3, 4, 5], 50) == 3
    assert abs(serving.percentile(list(range(101)), 99) - 99) < 1e-9
    a = serving.make_requests(500, 1000.0, seed=3)
    b = serving.make_requests(500, 1000.0, seed=3)
    assert [(r.arrival, r.size, r.dtype) for r in a] == [(r.arrival, r.size, r.dtype) for r in b]
    sizes = np.array([r.size for r in a])
    assert sizes.min() >= 1 << 10 and sizes.max() < 1 << 26
    gaps = np.diff([r.arrival for r in a])
    assert np.all(gaps >= 0) and 0.0005 < gaps.mean() < 0.002    # Poisson, rate 1000/s
    assert {r.dtype for r in a} == {"int32", "int64", "float64"}


def test_request_bytes_counts_keys_and_scratch():
    assert serving.request_bytes(1000, "int32") >= 2 * 4000
    assert serving.request_bytes(1000, "float64") >= 2 * 8000


@pytest.mark.gpu
def test_each_result_is_the_same_alone_and_in_the_mix():
    import torch

    import oracle
    import paper_1604_06697_gb300 as bqs
    from paper_1604_06697_gb300 import build
    build.build()
    pool = serving.KeyPool(max_size=1 << 20, seed=3)
    reqs = serving.make_requests(60, rate_hz=50_000.0, seed=3, log2_lo=4.0, log2_hi=20.0)
    loop = serving.ServingLoop(pool, mode="batched", slots=3, hbm_budget=8 << 30,
                               max_batch_keys=1 << 22, keep_results=True)
    rep = loop.run(reqs)
    assert rep["requests"] == 60 and rep["batches"] < 60     # requests were batched
    for r in reqs:
        alone = pool.keys(r).clone()
        bqs.sort(alone)
        torch.cuda.synchronize()
        assert torch.equal(r.result.view(torch.int64 if r.dtype != "int32" else torch.int32),
                           alone.view(torch.int64 if r.dtype != "int32" else torch.int32)), r.rid
    for r in reqs:   # and every result is the oracle's sort of the request's keys
        want = oracle.sort(pool.keys(r).cpu().numpy())
        got = r.result.cpu().numpy()
        assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), r.rid
    assert all(r.latency >= 0 and r.queue_delay >= 0 for r in reqs)


@pytest.mark.gpu
def test_plain_mode_serves_every_request():
    from paper_1604_06697_gb300 import build
    build.build()
    pool = serving.KeyPool(max_size=1 << 18, seed=4)
    reqs = serving.make_requests(20, rate_hz=5_000.0, seed=4, log2_lo=4.0, log2_hi=18.0)
    loop = serving.ServingLoop(pool, mode="plain", keep_results=True)
    rep = loop.run(reqs)
    assert rep["requests"] == 20 and rep["batches"] == 20 and rep["slots"] == 3
    assert rep["p99_ms"] >= rep["p50_ms"] > 0
    import oracle
    for r in reqs:
        want = oracle.sort(pool.keys(r).cpu().numpy())
        assert np.array_equal(r.result.cpu().numpy().view(np.uint8), want.view(np.uint8)), r.rid
