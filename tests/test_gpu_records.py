"""Wide elements (Sec. 4's Record and Vector types) sorted through the C ABI: the
output records must equal the oracle's byte for byte (key order, ties by input
position)."""
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


def _records(n, rb, seed, kind):
    r = inputs.splitmix64(seed, n * rb // 4)
    rec = (r & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.uint8).copy()
    if kind == 0:
        f = rec.view(np.int32).reshape(n, rb // 4)
        f[:, 0] = (inputs.splitmix64(seed + 1, n) % np.uint64(max(1, n // 4))).astype(np.int32)
    else:
        v = rec.view(np.float64).reshape(n, rb // 8)
        v[:] = 2.0 * inputs.unit_double(inputs.splitmix64(seed + 2, v.size)).reshape(v.shape) - 1.0
        v[1::7] = v[0::7][: v[1::7].shape[0]]
    return rec


def _gpu_sort_records(bqs, rec, rb, kind, off, count):
    import torch
    t = torch.from_numpy(rec.copy()).cuda()
    bqs.sort_records(t, rb, kind, off, count)
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("small_sort", [0, 1])
@pytest.mark.parametrize("kind,rb,off,count", [(0, 84, 0, 1),      # Record: 21 ints, first one
                                               (0, 84, 40, 1),     # another field
                                               (1, 80, 0, 10),     # Vector: 10 doubles, norm
                                               (1, 96, 16, 6)])    # norm of a sub-range
def test_records_match_oracle(bqs, kind, rb, off, count, small_sort):
    bqs.set_option("small_sort", small_sort)
    for n in (0, 1, 2, 1000, 100_003, 1 << 20):
        rec = _records(n, rb, n + 3, kind)
        got = _gpu_sort_records(bqs, rec, rb, kind, off, count)
        want = oracle.sort_records(rec, rb, kind, off, count)
        assert np.array_equal(got, want), (n, kind)


def test_record_arguments_are_checked(bqs):
    import torch
    t = torch.zeros(84 * 10, dtype=torch.uint8, device="cuda")
    with pytest.raises(bqs.BqsError):
        bqs.sort_records(t, 84, bqs.KEY_I32_FIELD, 2, 1)     # misaligned key
    with pytest.raises(bqs.BqsError):
        bqs.sort_records(t, 84, bqs.KEY_F64_SQNORM, 0, 10)   # 84-byte records, doubles
    with pytest.raises(bqs.BqsError):
        bqs.sort_records(t, 84, 7, 0, 1)                       # unknown key kind
