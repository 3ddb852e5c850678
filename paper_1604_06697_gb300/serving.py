"""Sort-request serving loop with continuous batching on one GPU.

Requests (size, dtype) arrive over time.  Each arrival is admitted when the keys it
brings, plus the scratch its sort needs, fit in a stated HBM budget; its keys then
live in device memory until the request completes.  Worker slots (one CUDA stream
and one host thread each; the sort's level loop is driven from the host) take work
as they become free:

* ``mode="batched"`` (continuous batching): a free slot takes every admitted,
  waiting request of the oldest request's dtype (up to ``max_batch_keys``), packs
  them into one buffer and sorts them with a single ``bqs_sort_batched`` call, one
  segment per request.  Requests that arrive while batches are on the GPU are
  picked up by the next free slot, so work from different batches overlaps on the
  device.
* ``mode="plain"``: the baseline -- one ``bqs_sort`` call per request, first come
  first served, on the same number of slots, so the two modes differ only in batching.

Admission copies a request's keys into HBM on a copy stream of its own and records an
event; the slot that later sorts the request waits for that event on the device, so
an arrival never waits behind a running sort.  Latency of a request = time its sort
finished on the GPU (a CUDA event, placed on the host clock through a reference
event) minus its arrival time; it includes the time spent waiting for admission and
for a slot (reported on its own as the queue delay: arrival to the moment a slot
takes the request).  Every sort runs in the library's kernels; this module only
schedules.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import threading
import time

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the run
    size: int
    dtype: str
    # filled in by the loop
    admitted: float = math.nan
    started: float = math.nan
    done: float = math.nan
    batch: int = -1
    result: object = None   # the sorted keys (a device tensor view) when kept

    @property
    def latency(self) -> float:
        return self.done - self.arrival

    @property
    def queue_delay(self) -> float:
        return self.started - self.arrival


ITEM = {"int32": 4, "int64": 8, "float64": 8}


def request_bytes(size: int, dtype: str) -> int:
    """HBM a request holds while admitted: its keys, their copy in a batch buffer, and
    the sort's scratch (a second key buffer plus work lists, at most one more copy)."""
    return 3 * size * ITEM[dtype] + (1 << 20)


class Admission:
    """HBM budget accounting (host side, thread safe)."""

    def __init__(self, budget_bytes: int):
        self.budget = int(budget_bytes)
        self.used = 0
        self.peak = 0
        self._lock = threading.Lock()

    def try_admit(self, nbytes: int) -> bool:
        with self._lock:
            if nbytes > self.budget:
                raise ValueError(f"request of {nbytes} B exceeds the whole budget")
            if self.used + nbytes > self.budget:
                return False
            self.used += nbytes
            self.peak = max(self.peak, self.used)
            return True

    def release(self, nbytes: int) -> None:
        with self._lock:
            self.used -= nbytes
            assert self.used >= 0


def form_batch(waiting: collections.deque, max_batch_keys: int):
    """Takes the oldest waiting request and every other waiting request of its dtype,
    in arrival order, while the batch stays within max_batch_keys keys (the oldest
    request is always taken)."""
    if not waiting:
        return []
    dtype = waiting[0].dtype
    batch, keys, keep = [], 0, collections.deque()
    while waiting:
        r = waiting.popleft()
        if r.dtype == dtype and (not batch or keys + r.size <= max_batch_keys):
            batch.append(r)
            keys += r.size
        else:
            keep.append(r)
    waiting.extendleft(reversed(keep))
    return batch


def percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return math.nan
    k = (len(xs) - 1) * q / 100.0
    f, c = math.floor(k), math.ceil(k)
    return xs[f] if f == c else xs[f] + (xs[c] - xs[f]) * (k - f)


class KeyPool:
    """Device-resident random keys per dtype; request i's keys are a slice at a
    seeded offset.  Placing a request in HBM is then one device copy."""

    def __init__(self, max_size: int, seed: int = 3, dtypes=("int32", "int64", "float64")):
        import torch
        from . import inputs
        self.max_size = max_size
        self.seed = seed
        self.pool = {}
        for i, dt in enumerate(dtypes):
            self.pool[dt] = torch.from_numpy(inputs.make_keys(2 * max_size, dt, "uniform",
                                                              seed * 1000 + i)).cuda()

    def offset(self, rid: int, size: int) -> int:
        from . import inputs
        r = int(inputs.splitmix64(self.seed, 1, stream=4, start=rid)[0])
        return r % (self.max_size + 1)

    def keys(self, r: Request):
        off = self.offset(r.rid, r.size)
        return self.pool[r.dtype][off:off + r.size]


class ServingLoop:
    def __init__(self, pool: KeyPool, mode: str = "batched", slots: int = 3,
                 hbm_budget: int = 64 << 30, max_batch_keys: int = 1 << 27,
                 keep_results: bool = False):
        if mode not in ("batched", "plain"):
            raise ValueError("mode must be 'batched' or 'plain'")
        self.pool = pool
        self.mode = mode
        self.slots = slots
        self.admission = Admission(hbm_budget)
        self.max_batch_keys = max_batch_keys
        self.keep_results = keep_results

    def run(self, requests):
        import torch

        import paper_1604_06697_gb300 as bqs

        reqs = sorted(requests, key=lambda r: r.arrival)
        dev = torch.device("cuda")
        streams = [torch.cuda.Stream(dev) for _ in range(self.slots)]
        copy_stream = torch.cuda.Stream(dev)     # admission copies only
        waiting = collections.deque()       # admitted, not yet started
        pending = collections.deque(reqs)   # not yet arrived or not yet admitted
        cv = threading.Condition()
        finished = []
        stop = [False]
        batch_id = [0]
        errors = []

        torch.cuda.synchronize()
        ref = torch.cuda.Event(enable_timing=True)
        ref.record()
        torch.cuda.synchronize()
        t0 = time.perf_counter()

        def now():
            return time.perf_counter() - t0

        def gpu_time(ev):
            return ref.elapsed_time(ev) / 1e3

        def worker(slot):
            stream = streams[slot]
            try:
                while True:
                    with cv:
                        while not waiting and not stop[0]:
                            cv.wait(0.01)
                        if not waiting and stop[0]:
                            return
                        if self.mode == "plain":
                            batch = [waiting.popleft()]
                        else:
                            batch = form_batch(waiting, self.max_batch_keys)
                        bid = batch_id[0]
                        batch_id[0] += 1
                    start = now()
                    with torch.cuda.stream(stream):
                        for r in batch:   # its keys have landed in HBM
                            stream.wait_event(r._ready)
                            r._buf.record_stream(stream)
                        if self.mode == "plain":
                            r = batch[0]
                            buf = r._buf
                            bqs.sort(buf, stream=stream)
                            views = [buf]
                        else:
                            sizes = [r.size for r in batch]
                            off = np.zeros(len(batch) + 1, np.int64)
                            np.cumsum(sizes, out=off[1:])
                            buf = torch.empty(int(off[-1]), dtype=batch[0]._buf.dtype, device=dev)
                            for r, a, b in zip(batch, off[:-1], off[1:]):
                                buf[a:b].copy_(r._buf)
                            toff = torch.from_numpy(off).to(dev, non_blocking=True)
                            bqs.sort_batched(buf, toff, stream=stream)
                            views = [buf[a:b] for a, b in zip(off[:-1], off[1:])]
                        ev = torch.cuda.Event(enable_timing=True)
                        ev.record(stream)
                    ev.synchronize()
                    t_done = gpu_time(ev)
                    with cv:
                        for r, v in zip(batch, views):
                            r.started = start
                            r.done = t_done
                            r.batch = bid
                            r.result = v if self.keep_results else None
                            r._buf = None
                            r._ready = None
                            self.admission.release(request_bytes(r.size, r.dtype))
                            finished.append(r)
                        cv.notify_all()
            except Exception as e:  # surfaced after the run
                errors.append(e)
                with cv:
                    stop[0] = True
                    cv.notify_all()

        threads = [threading.Thread(target=worker, args=(i,), daemon=True) for i in range(self.slots)]
        for t in threads:
            t.start()
        try:
            while pending and not errors:
                r = pending[0]
                wait = r.arrival - now()
                if wait > 0:
                    time.sleep(min(wait, 0.002))
                    continue
                if not self.admission.try_admit(request_bytes(r.size, r.dtype)):
                    with cv:
                        cv.wait(0.001)   # a completion frees memory
                    continue
                pending.popleft()
                r.admitted = now()
                with torch.cuda.stream(copy_stream):
                    r._buf = self.pool.keys(r).clone()   # the request's keys, now in HBM
                    r._ready = torch.cuda.Event()
                    r._ready.record(copy_stream)
                with cv:
                    waiting.append(r)
                    cv.notify_all()
        finally:
            with cv:
                stop[0] = True
                cv.notify_all()
            for t in threads:
                t.join()
        if errors:
            raise errors[0]
        return self.report(finished, now())

    def report(self, finished, wall):
        lat = [r.latency for r in finished]
        queue = [r.queue_delay for r in finished]
        keys = sum(r.size for r in finished)
        span = max(r.done for r in finished) - min(r.arrival for r in finished) if finished else math.nan
        arrivals = max(r.arrival for r in finished) - min(r.arrival for r in finished) if finished else math.nan
        batches = len({r.batch for r in finished})
        return {
            "mode": self.mode, "slots": self.slots, "requests": len(finished), "batches": batches,
            "p50_ms": 1e3 * percentile(lat, 50), "p99_ms": 1e3 * percentile(lat, 99),
            "mean_ms": 1e3 * (sum(lat) / len(lat)) if lat else math.nan,
            "queue_p50_ms": 1e3 * percentile(queue, 50), "queue_p99_ms": 1e3 * percentile(queue, 99),
            "offered_keys_per_s": keys / arrivals if arrivals and arrivals > 0 else math.nan,
            "served_keys_per_s": keys / span if span and span > 0 else math.nan,
            "keys": keys, "span_s": span, "wall_s": wall,
            "hbm_peak_bytes": self.admission.peak, "hbm_budget_bytes": self.admission.budget,
        }


def make_requests(count: int, rate_hz: float, seed: int = 3, log2_lo: float = 10.0,
                  log2_hi: float = 26.0):
    from . import inputs
    return [Request(i, a, s, d) for i, (a, s, d) in
            enumerate(inputs.request_stream(count, rate_hz, seed, log2_lo, log2_hi))]
