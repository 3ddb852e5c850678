"""Failure detection without a GPU fault.

The partition kernel's waits on its shared-memory pipeline and the grid-wide barriers
of the single-launch sort are bounded.  A test-only
option leaves one tile unrequested, so that wait runs out: the kernel records a
timeout in the device status word, waits (again bounded) for the copies it did
issue, and returns.  The call reports BQS_ERR_TIMEOUT and the device stays usable:
the next sort is correct.  Host-side failures (bad arguments, decreasing offsets)
are covered in test_gpu_sort.py and test_abi.py.
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


@pytest.mark.parametrize("log2n,level_loop,overlap", [(24, 0, 0), (24, 1, 0), (24, 0, 1), (20, 0, 1)])
def test_bounded_wait_times_out_and_device_stays_usable(bqs, log2n, level_loop, overlap):
    # level_loop 1: the levels enqueued after the failing one find no work; overlap 1:
    # the call's stream still waits for the networks on the second stream.  2^20 keys:
    # the first level is small enough for the partition kernel with the bookkeeping
    # fused in, whose failing block copies the control block out itself (the level's
    # last segment never completes).
    import torch
    a = inputs.make_keys(1 << log2n, "int32", "uniform", seed=8)   # every block owns tiles
    t = torch.from_numpy(a).cuda()
    bqs.set_option("level_loop", level_loop)
    bqs.set_option("overlap", overlap)
    old_limit = bqs.get_option("wait_limit")
    bqs.set_option("wait_limit", 1 << 16)      # give up after ~10 ms instead of seconds
    bqs.set_option("test_stall", 1)
    try:
        with pytest.raises(bqs.BqsError) as e:
            bqs.sort(t)
        assert e.value.status == -4                  # BQS_ERR_TIMEOUT
    finally:
        bqs.set_option("test_stall", 0)
        bqs.set_option("wait_limit", old_limit)
    torch.cuda.synchronize()                         # no sticky CUDA error
    t2 = torch.from_numpy(a).cuda()
    bqs.sort(t2)
    torch.cuda.synchronize()
    assert np.array_equal(t2.cpu().numpy(), oracle.sort(a))


def test_single_launch_barrier_times_out_and_device_stays_usable(bqs):
    # The single-launch sort meets at grid-wide barriers; the test option keeps block 0
    # from arriving at the first one, so every other block's bounded wait runs out and
    # records the timeout.  The call reports BQS_ERR_TIMEOUT and the next sort (the
    # same path) is correct.
    import torch
    a = inputs.make_keys(1 << 20, "int32", "uniform", seed=9)
    t = torch.from_numpy(a).cuda()
    old = {k: bqs.get_option(k) for k in ("coop_max", "wait_limit")}
    bqs.set_option("coop_max", 1 << 22)
    bqs.set_option("wait_limit", 1 << 16)
    bqs.set_option("test_stall", 1)
    try:
        with pytest.raises(bqs.BqsError) as e:
            bqs.sort(t)
        assert e.value.status == -4
    finally:
        bqs.set_option("test_stall", 0)
        bqs.set_option("wait_limit", old["wait_limit"])
    torch.cuda.synchronize()
    t2 = torch.from_numpy(a).cuda()
    bqs.sort(t2)
    torch.cuda.synchronize()
    assert bqs.stats()["partition_launches"] == 0          # the single launch ran again
    assert np.array_equal(t2.cpu().numpy(), oracle.sort(a))
    bqs.set_option("coop_max", old["coop_max"])
