"""Autotuner for the sort's launch shape.

Chooses, for one workload class (dtype, size bucket, single array or batch), the
partition tile variant (threads x keys per thread), the small-segment cutoff, the
small-segment network shape (one warp / warp group per segment, or one 256-thread
block), whether the networks run on a second stream beside the partitions, and the
single-block local-partitioning cutoff by timing every candidate on a synthetic input
of that class with CUDA events.  Results are cached in a JSON file keyed by GPU
name, dtype, workload kind and log2 size bucket, so a later process applies the
choice without re-timing.  The tuner only sets the library's options; every
candidate runs the same kernels through the C ABI.
"""
from __future__ import annotations

import itertools
import json
import math
import os

from . import inputs

TILES = (0, 1, 2, 3, 4, 5)     # TMA partition variants (see bqs_set_option(BQS_OPT_TILE))
SMALL_CUTOFFS = (256, 1024, 2048, 4096)   # above 2048: key-only sorts, warp-group networks
LOCAL_CUTOFFS = (0, -1)        # off, or as large as one thread block holds
SMALL_SORTS = (0, 1)           # warp / warp-group networks, or 256-thread block networks
OVERLAPS = (0, 1)              # networks on the call's stream, or beside the partitions
COOP_MAX = 1 << 22             # single arrays up to this size may run as one cooperative launch
KNOBS = ("tile", "small_cutoff", "local_cutoff", "small_sort", "overlap", "coop_max")


def default_cache_path() -> str:
    base = os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache"))
    return os.path.join(base, "paper_1604_06697_gb300", "autotune.json")


def cache_key(dtype: str, n: int, kind: str) -> str:
    import torch
    gpu = torch.cuda.get_device_name()
    return f"{gpu}|{dtype}|{kind}|2^{max(0, int(math.log2(max(1, n))))}|v2"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(path, table):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def apply(config: dict) -> None:
    import paper_1604_06697_gb300 as bqs
    for k in KNOBS:
        if k in config:
            bqs.set_option(k, int(config[k]))


def _time(run, reps: int) -> float:
    import torch
    ms = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        run()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    return min(ms)


def candidate_configs(kind: str = "sort", n: int | None = None) -> list:
    """Every launch shape the tuner times for a workload kind.  Cutoffs above 2048 keys
    exist only for key-only sorts with the warp-group networks (the library clamps the
    others to 2048), so they are not timed twice."""
    host = [dict(tile=t, small_cutoff=s, local_cutoff=l, small_sort=w, overlap=o, coop_max=0)
            for t, s, l, w, o in itertools.product(TILES, SMALL_CUTOFFS, LOCAL_CUTOFFS,
                                                   SMALL_SORTS, OVERLAPS)
            if s <= 2048 or (kind != "pairs" and w == 0)]
    # Single arrays that fit the cooperative launch: every level in one kernel (tile,
    # local partitioning and overlap do not apply there), one candidate per cutoff.
    coop = [dict(tile=0, small_cutoff=s, local_cutoff=0, small_sort=0, overlap=0, coop_max=COOP_MAX)
            for s in SMALL_CUTOFFS] if kind == "sort" and (n is None or n <= COOP_MAX) else []
    return host + coop


def tune(dtype: str, n: int, kind: str = "sort", nseg: int = 0, reps: int | None = None,
         cache_path: str | None = None, force: bool = False, candidates=None) -> dict:
    """Returns (and caches) the fastest configuration for this workload class.

    kind: "sort" (one array of n keys, uniform values), "pairs" (n key-value pairs:
    keys uniform in [0, 2^20), payload = index, sorted by bqs_sort_pairs) or
    "batched" (nseg arrays with log-uniform lengths in [16, 65536] totalling about n
    keys, sorted by bqs_sort_batched).  reps: timed sorts per candidate, the best one
    kept (default 5 up to 2^22 keys, where one sort takes well under a millisecond
    and launch jitter decides between close candidates; 2 above).
    """
    import torch

    import paper_1604_06697_gb300 as bqs

    if reps is None:
        reps = 5 if n <= (1 << 22) else 2
    path = cache_path or default_cache_path()
    table = _load(path)
    key = cache_key(dtype, n, kind)
    if key in table and not force:
        apply(table[key]["config"])
        return table[key]

    if kind == "pairs":
        import numpy as np
        pk, pv = inputs.make_pairs(n, seed=1)
        src_k = torch.from_numpy(pk.astype(dtype)).cuda()
        src_v = torch.from_numpy(pv.view(np.int32)).cuda()
        work_k, work_v = torch.empty_like(src_k), torch.empty_like(src_v)

        def run():
            bqs.sort_pairs(work_k, work_v)

        def prep():
            work_k.copy_(src_k)
            work_v.copy_(src_v)
    elif kind == "batched":
        keys, off = inputs.make_segments(nseg, seed=2, dtype=dtype)
        src = torch.from_numpy(keys).cuda()
        toff = torch.from_numpy(off).cuda()
        work = torch.empty_like(src)

        def run():
            bqs.sort_batched(work, toff)

        def prep():
            work.copy_(src)
    else:
        src = torch.from_numpy(inputs.make_keys(n, dtype, "uniform", 1)).cuda()
        work = torch.empty_like(src)

        def run():
            bqs.sort(work)

        def prep():
            work.copy_(src)

    saved = {k: bqs.get_option(k) for k in KNOBS}
    results = []
    cands = candidates or candidate_configs(kind, n)
    try:
        for cfg in cands:
            apply(cfg)
            best = float("inf")
            for _ in range(reps):
                prep()
                torch.cuda.synchronize()
                best = min(best, _time(run, 1))
            results.append((best, cfg))
    finally:
        apply(saved)
    results.sort(key=lambda r: r[0])
    entry = {"config": results[0][1], "ms": results[0][0],
             "timed": [{"config": c, "ms": t} for t, c in results]}
    table[key] = entry
    _store(path, table)
    apply(entry["config"])
    return entry
