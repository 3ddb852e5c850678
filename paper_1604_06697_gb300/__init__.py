"""GB300-native (sm_103a) data-parallel BlockQuicksort.

A thin binding over the C ABI of ``libbqs.so`` (see ``include/bqs.h``).  The
functions take CUDA tensors and only marshal arguments: every step of every
sort runs in the library's CUDA kernels.  PyTorch supplies device memory and
streams.
"""
from __future__ import annotations

import ctypes

from . import _native

BQS_OK = 0
DTYPE_CODES = {"int32": 0, "int64": 1, "float64": 2}
OPTIONS = {"pivot": 0, "small_cutoff": 1, "depth_limit": 2, "timing": 3, "tile": 4,
           "local_cutoff": 5, "wait_limit": 6, "test_stall": 7, "level_loop": 8,
           "small_sort": 9, "overlap": 10,
           "local_sort": 11, "coop_max": 12}


class BqsError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = _native.lib().bqs_status_string(status).decode()
        super().__init__(f"{where}: status {status} ({msg})")
        self.status = status


def _check(status: int, where: str) -> None:
    if status != BQS_OK:
        raise BqsError(status, where)


_CODE_BY_DTYPE = {}   # torch dtype -> code, filled on first use


def _dtype_code(t) -> int:
    code = _CODE_BY_DTYPE.get(t.dtype)
    if code is None:
        name = str(t.dtype).replace("torch.", "")
        if name not in DTYPE_CODES:
            raise TypeError(f"unsupported key dtype {t.dtype}")
        code = _CODE_BY_DTYPE[t.dtype] = DTYPE_CODES[name]
    return code


_raw_stream = None   # torch's accessor of the current stream's handle, when it has one


def _stream_ptr(t, stream):
    global _raw_stream
    if stream is not None:
        return ctypes.c_void_p(stream.cuda_stream)
    if _raw_stream is None:
        import torch
        _raw_stream = getattr(torch._C, "_cuda_getCurrentRawStream", False)
    if _raw_stream:
        return ctypes.c_void_p(_raw_stream(t.device.index))
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


def _require_cuda(*ts):
    for t in ts:
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError("expected contiguous CUDA tensors")


def sort(keys, stream=None):
    """Sorts a contiguous CUDA tensor of int32/int64/float64 keys in place."""
    _require_cuda(keys)
    _check(_native.lib().bqs_sort(keys.data_ptr(), keys.numel(), _dtype_code(keys),
                                  _stream_ptr(keys, stream)), "bqs_sort")
    return keys


NOALLOC_MAX_KEYS = 1 << 20


def sort_noalloc(keys, stream=None):
    """Sorts like sort() without allocating any memory during the call.

    For callers that cannot allocate device memory while they sort (memory
    reserved up front, or owned by another framework's allocator).  Uses a fixed
    scratch array held by the library; n is limited to NOALLOC_MAX_KEYS.  Calls
    that run on the GPU at the same time share that array and must be serialised.
    """
    _require_cuda(keys)
    _check(_native.lib().bqs_sort_noalloc(keys.data_ptr(), keys.numel(), _dtype_code(keys),
                                          _stream_ptr(keys, stream)), "bqs_sort_noalloc")
    return keys


KEY_I32_FIELD, KEY_F64_SQNORM = 0, 1


def sort_records(records, record_bytes, key_kind, key_offset=0, key_count=1, stream=None):
    """Sorts fixed-size records in place by a key taken from each record.

    ``records`` is a contiguous CUDA tensor holding n * record_bytes bytes (any dtype).
    key_kind KEY_I32_FIELD: the int32 at byte ``key_offset``; KEY_F64_SQNORM: the squared
    norm of ``key_count`` doubles from ``key_offset``.  Equal keys keep their order.
    """
    _require_cuda(records)
    nbytes = records.numel() * records.element_size()
    if record_bytes <= 0 or nbytes % record_bytes:
        raise ValueError("records must hold a whole number of records")
    _check(_native.lib().bqs_sort_records(records.data_ptr(), nbytes // record_bytes, record_bytes,
                                          key_kind, key_offset, key_count,
                                          _stream_ptr(records, stream)), "bqs_sort_records")
    return records


def sort_pairs(keys, vals, stream=None):
    """Sorts (key, uint32 payload) pairs in place by (key, payload).

    ``vals`` is an int32 or uint32 tensor whose bits are the payloads.
    """
    _require_cuda(keys, vals)
    if vals.numel() != keys.numel() or vals.element_size() != 4:
        raise ValueError("vals must hold one 32-bit payload per key")
    _check(_native.lib().bqs_sort_pairs(keys.data_ptr(), vals.data_ptr(), keys.numel(),
                                        _dtype_code(keys), _stream_ptr(keys, stream)),
           "bqs_sort_pairs")
    return keys, vals


def sort_segmented(keys, seg_offsets, stream=None):
    """Sorts every segment [off[i], off[i+1]) of ``keys`` in place (int64 offsets)."""
    import torch
    _require_cuda(keys, seg_offsets)
    if seg_offsets.dtype != torch.int64:
        raise TypeError("seg_offsets must be int64")
    _check(_native.lib().bqs_sort_segmented(keys.data_ptr(), seg_offsets.data_ptr(),
                                            seg_offsets.numel() - 1, _dtype_code(keys),
                                            _stream_ptr(keys, stream)), "bqs_sort_segmented")
    return keys


def sort_batched(keys, seg_offsets, stream=None):
    """Segmented sort that never reads device memory back during the call.

    Inside ``torch.cuda.graph(...)`` capture the whole level loop is recorded as a
    device-side loop, so replaying the graph sorts the batch in one launch.
    """
    import torch
    _require_cuda(keys, seg_offsets)
    if seg_offsets.dtype != torch.int64:
        raise TypeError("seg_offsets must be int64")
    _check(_native.lib().bqs_sort_batched(keys.data_ptr(), keys.numel(), seg_offsets.data_ptr(),
                                          seg_offsets.numel() - 1, _dtype_code(keys),
                                          _stream_ptr(keys, stream)), "bqs_sort_batched")
    return keys


def partition(keys, pivot, out=None, stream=None):
    """Partitions ``keys`` around ``pivot`` into ``out``; returns (out, split).

    out[:split] holds exactly the keys < pivot, out[split:] the keys >= pivot.
    """
    import torch
    _require_cuda(keys)
    if out is None:
        out = torch.empty_like(keys)
    _require_cuda(out)
    code = _dtype_code(keys)
    pv = _native.Pivot()
    pv.dtype = code
    pv.reserved = 0
    if code == 0:
        pv.v.i32 = int(pivot)
    elif code == 1:
        pv.v.i64 = int(pivot)
    else:
        pv.v.f64 = float(pivot)
    split = ctypes.c_int64(0)
    _check(_native.lib().bqs_partition(keys.data_ptr(), keys.numel(), ctypes.byref(pv),
                                       out.data_ptr(), ctypes.byref(split),
                                       _stream_ptr(keys, stream)), "bqs_partition")
    return out, int(split.value)


def set_option(name: str, value: int) -> None:
    _check(_native.lib().bqs_set_option(OPTIONS[name], int(value)), f"bqs_set_option({name})")


def get_option(name: str) -> int:
    v = ctypes.c_int64(0)
    _check(_native.lib().bqs_get_option(OPTIONS[name], ctypes.byref(v)), f"bqs_get_option({name})")
    return int(v.value)


def workspace_bytes(n: int, dtype: str, with_payload: bool = False, nseg: int = 0) -> int:
    v = ctypes.c_int64(0)
    _check(_native.lib().bqs_workspace_bytes(n, DTYPE_CODES[dtype], int(with_payload), nseg,
                                             ctypes.byref(v)), "bqs_workspace_bytes")
    return int(v.value)


def set_workspace(buf) -> None:
    """Uses a caller-owned CUDA buffer (uint8 tensor) as scratch; None clears it."""
    if buf is None:
        _check(_native.lib().bqs_set_workspace(None, 0), "bqs_set_workspace")
    else:
        _check(_native.lib().bqs_set_workspace(buf.data_ptr(), buf.numel() * buf.element_size()),
               "bqs_set_workspace")


def stats() -> dict:
    """Counters of this thread's last sort call."""
    s = _native.Stats()
    _check(_native.lib().bqs_get_stats(ctypes.byref(s)), "bqs_get_stats")
    return {name: getattr(s, name) for name, _ in _native.Stats._fields_}


def collect_timing():
    """With the "timing" option at 2: (ms, launches) summed over the partition launches
    that had work in this thread's sorts since the last collect (waits for them)."""
    ms, n = ctypes.c_double(0), ctypes.c_int64(0)
    _check(_native.lib().bqs_timing_collect(ctypes.byref(ms), ctypes.byref(n)), "bqs_timing_collect")
    return float(ms.value), int(n.value)
