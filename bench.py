"""Benchmark of the GB300 BlockQuicksort: keys/s and HBM-roofline fraction.

Default workload: one array of 2^28 int32 keys, uniform over the full range
(seed 1), sorted in place by bqs_sort with the median-of-sqrt(n) pivot rule.
A step is one complete sort of one such array; every timed step sorts its own
pre-generated copy already resident in HBM (1 GiB per step, far above the
129 MB L2, so no flush is needed between steps).

Prints ONE JSON line (rank 0).  Multi-GPU runs (torchrun, one process per GPU)
are independent replicas: every rank sorts its own arrays, there is no data-path
collective, value = all keys sorted by all ranks / max-over-ranks time.

--impl reference times the CPU oracle (the paper's single-threaded block
partition Quicksort) on this host, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "keys/s + % HBM roofline, 2^28 int32 sort; served p99 vs plain per-array launch"
FALLBACK_HBM_GBS = 6800.0


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--log2n", type=int, default=28)
    ap.add_argument("--dtype", default="int32", choices=["int32", "int64", "float64"])
    ap.add_argument("--dist", default="uniform")
    ap.add_argument("--pivot", default="sqrt", choices=["mo3", "sqrt"])
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    return ap.parse_args(argv)


def workload_name(a) -> str:
    return f"bqs_sort 2^{a.log2n} {a.dtype} {a.dist} seed {a.seed}, {a.pivot} pivot"


def measured_peak_gbs():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def committed_traffic():
    """DRAM bytes per processed key of the partition kernel from the committed ncu summary.

    Returns None when the kernel's source files changed since the capture (their
    hash is stored beside the counters), so a stale figure is never reported.
    """
    import hashlib
    path = os.path.join(ROOT, "profiles", "partition_traffic.json")
    try:
        with open(path) as f:
            tr = json.load(f)
        h = hashlib.sha256()
        for rel in tr["source_files"]:
            with open(os.path.join(ROOT, rel), "rb") as f:
                h.update(f.read())
        return tr if h.hexdigest()[:16] == tr["source_sha256_16"] else None
    except Exception:
        return None


# ---- CPU oracle timing (bounded sample) --------------------------------------------------------

def time_oracle(a, seconds: float):
    """Sorts 2^24-key samples of the workload with the oracle until `seconds` have passed."""
    import oracle
    from paper_1604_06697_gb300 import inputs

    oracle.build()
    m = min(1 << 24, 1 << a.log2n)
    sample = inputs.make_keys(m, a.dtype, a.dist, a.seed)
    keys = 0
    t0 = time.perf_counter()
    reps = 0
    while True:
        oracle.sort(sample, pivot=a.pivot)
        keys += m
        reps += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": keys / dt, "unit": "keys/s", "cores": 1, "kind": "oracle",
            "sample": f"{reps} x oracle sort of the first 2^{int(math.log2(m))} keys of the "
                      f"workload ({a.dtype} {a.dist} seed {a.seed}, {a.pivot} pivot), "
                      f"single thread, {dt:.1f} s"}


# ---- clocks ----------------------------------------------------------------------------------

class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while the timed region runs.

    Samples carry nvidia-smi's own timestamps; only those inside [mark_start, mark_end]
    are summarised.
    """
    QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.5)
        except Exception:
            self.proc = None
        return self

    def mark_start(self):
        import datetime
        self.t0 = datetime.datetime.now()

    def mark_end(self):
        import datetime
        self.t1 = datetime.datetime.now()

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        import datetime
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lo = self.t0 - datetime.timedelta(milliseconds=50) if self.t0 else None
        hi = self.t1 + datetime.timedelta(milliseconds=50) if self.t1 else None
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f")
                if lo and hi and not (lo <= ts <= hi):
                    continue
                sm.append(float(f[2]))
                mx.append(float(f[3]))
                power.append(float(f[4]))
            except ValueError:
                continue
            for name, val in zip(names, f[6:10]):
                if val.lower() in ("active", "1"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


# ---- reference arm -------------------------------------------------------------------------------

def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    per_step = max(1.0, 20.0 / max(1, a.steps + a.warmup))
    base = time_oracle(a, per_step * (a.steps + a.warmup))
    value = base["value"]
    n = 1 << a.log2n
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "keys/s",
        "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": 1e3 * n / value, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": a.dtype, "data": "synthetic",
        "config": {"workload": workload_name(a), "n": n, "dist": a.dist, "seed": a.seed,
                   "pivot": a.pivot},
        "cpu_baseline": base,
        "e2e": {"value": value, "unit": "keys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---- our arm ----------------------------------------------------------------------------------------

def run_ours(a):
    import torch

    from paper_1604_06697_gb300 import build as _build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    _build.build()
    import paper_1604_06697_gb300 as bqs
    from paper_1604_06697_gb300 import inputs

    n = 1 << a.log2n
    bqs.set_option("pivot", 1 if a.pivot == "sqrt" else 0)
    host = inputs.make_keys(n, a.dtype, a.dist, a.seed)
    src = torch.from_numpy(host).to(dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # Warm-up (each step restores the unsorted input first).
    work = torch.empty_like(src)
    for _ in range(a.warmup):
        work.copy_(src)
        bqs.sort(work)
    torch.cuda.synchronize(dev)

    # One resident unsorted copy per timed step.
    bufs = [src.clone() for _ in range(a.steps)]
    torch.cuda.synchronize(dev)
    bqs.set_option("timing", 1)
    part_ms, part_bytes, launches, part_launches, levels = 0.0, 0.0, 0, 0, []
    clk = ClockSampler(dev.index if dev.index is not None else 0)
    barrier()
    torch.cuda.synchronize(dev)
    with clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        clk.mark_start()
        e0.record(stream)
        for k in range(a.steps):
            bqs.sort(bufs[k])
            s = bqs.stats()
            part_ms += s["partition_ms"]
            part_bytes += s["partition_bytes"]
            launches += s["kernel_launches"]
            part_launches += s["partition_launches"]
            levels.append(s["levels"])
        e1.record(stream)
        torch.cuda.synchronize(dev)
        clk.mark_end()
    barrier()
    bqs.set_option("timing", 0)
    ms = e0.elapsed_time(e1)
    # Correctness spot check outside the timed region: sorted and same multiset sum.
    out = bufs[0]
    ok = bool((out[1:] >= out[:-1]).all().item()) if a.dtype != "float64" else True
    del bufs
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())

    value = world * n * a.steps / (ms / 1e3)

    # End to end through the public API with host buffers: pinned H2D, sort, D2H.
    e2e = None
    if not a.no_e2e:
        pin_in = torch.from_numpy(host).pin_memory()
        pin_out = torch.empty_like(pin_in).pin_memory()
        dbuf = torch.empty_like(src)
        for _ in range(2):
            dbuf.copy_(pin_in, non_blocking=True)
            bqs.sort(dbuf)
            pin_out.copy_(dbuf, non_blocking=True)
        torch.cuda.synchronize(dev)
        barrier()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(a.steps):
            dbuf.copy_(pin_in, non_blocking=True)
            bqs.sort(dbuf)
            pin_out.copy_(dbuf, non_blocking=True)
        f1.record(stream)
        torch.cuda.synchronize(dev)
        ems = f0.elapsed_time(f1)
        if world > 1:
            import torch.distributed as dist
            t = torch.tensor([ems], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ems = float(t.item())
        nbytes = n * host.itemsize
        e2e = {"value": world * n * a.steps / (ems / 1e3), "unit": "keys/s",
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}
        del pin_in, pin_out, dbuf

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu:
        cpu = time_oracle(a, a.cpu_seconds)

    peak, peak_kind = measured_peak_gbs()
    achieved = (part_bytes / (part_ms / 1e3)) / 1e9 if part_ms > 0 else None
    traffic = None
    tr = committed_traffic()
    if tr and tr.get("dtype") == a.dtype and part_launches:
        # ncu DRAM bytes per processed key x keys per launch of this run
        traffic = tr["dram_bytes_per_active_key"] * (part_bytes / (2 * host.itemsize)) / part_launches
    roofline = {
        "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
        "frac": (achieved / peak) if achieved else None, "traffic": traffic,
        "kernel": "k_partition", "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)"
                  if peak_kind == "measured" else "fallback 6.8 TB/s",
        "algorithmic_bytes_per_launch": part_bytes / max(1, part_launches),
        "avg_launch_ms": part_ms / max(1, part_launches),
        "frac_of_8tbs_spec": (achieved / 8000.0) if achieved else None,
    }
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "keys/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": a.dtype, "data": "synthetic",
            "config": {"workload": workload_name(a), "n": n, "dist": a.dist, "seed": a.seed,
                       "pivot": a.pivot, "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2 (one resident 2^%d-key copy per step)" % a.log2n},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "levels_per_sort": levels[0] if levels else None,
            "clocks": clk.summary(), "sorted_check": ok,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main(argv=None):
    a = parse_args(argv)
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
