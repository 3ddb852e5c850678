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
    ap.add_argument("--workload", default="sort",
                    choices=["sort", "pairs", "batched", "serving", "matrix", "pivots",
                             "structured", "records"],
                    help="sort (the default headline line), pairs, batched, serving, matrix, "
                         "pivots, structured or records")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the autotuner and use --tile/--small/--local instead")
    ap.add_argument("--tile", type=int, default=None)
    ap.add_argument("--small", type=int, default=None)
    ap.add_argument("--local", type=int, default=None)
    ap.add_argument("--small-sort", type=int, default=None, choices=[0, 1])
    ap.add_argument("--overlap", type=int, default=None, choices=[0, 1])
    ap.add_argument("--coop-max", type=int, default=None,
                    help="with --no-tune: largest single array sorted in one launch (0: never)")
    return ap.parse_args(argv)


def workload_name(a) -> str:
    return f"bqs_sort 2^{a.log2n} {a.dtype} {a.dist} seed {a.seed}, {a.pivot} pivot"


def workload_config(a) -> dict:
    """The workload both arms run, identical in both JSON lines."""
    n = 1 << a.log2n
    nbytes = n * (4 if a.dtype == "int32" else 8)
    size = "2^%d-key (%.1f MiB) array" % (a.log2n, nbytes / 2**20)
    l2 = ("inputs larger than L2: every step sorts its own unsorted copy of the " + size
          if nbytes > (129 << 20) else
          "input smaller than L2: every step sorts its own unsorted copy of the " + size)
    return {"workload": workload_name(a), "n": n, "dtype": a.dtype, "dist": a.dist,
            "seed": a.seed, "pivot": a.pivot, "l2": l2}


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


# ---- replicas (one process per GPU, no data-path collective) -----------------------------------

def max_over_ranks(value: float, device=None) -> float:
    """The largest of every rank's value (the slowest rank's time); the value itself when
    there is one process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank: float, ms_max: float, world: int) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return world * units_per_rank / (ms_max / 1e3)


# ---- CPU oracle timing (bounded sample) --------------------------------------------------------

def gpu_local_cpus(dev):
    """CPUs of the NUMA node the GPU is attached to (sysfs), or None if unknown."""
    import torch
    try:
        pr = torch.cuda.get_device_properties(dev)
        bus = "%04x:%02x:%02x.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
        with open("/sys/bus/pci/devices/%s/local_cpulist" % bus) as f:
            text = f.read().strip()
    except Exception:
        return None
    cpus = set()
    for part in text.split(","):
        if "-" in part:
            lo, hi = part.split("-")
            cpus.update(range(int(lo), int(hi) + 1))
        elif part:
            cpus.add(int(part))
    return cpus or None


def pinned_near_gpu(dev, make):
    """Allocates pinned host buffers (make()) from a thread bound to the GPU's own NUMA
    node, so that their pages sit next to the GPU's host link; the affinity is restored
    afterwards.  Returns (buffers, node CPUs used or None)."""
    cpus = gpu_local_cpus(dev)
    saved = os.sched_getaffinity(0) if hasattr(os, "sched_getaffinity") else None
    use = (cpus & saved) if (cpus and saved) else None
    if use:
        os.sched_setaffinity(0, use)
    try:
        return make(), (sorted(use) if use else None)
    finally:
        if use:
            os.sched_setaffinity(0, saved)


def time_oracle(a, host_keys, min_seconds: float = 0.0):
    """Sorts the whole workload with the oracle, single threaded, on a fresh copy each
    time, at least once and until min_seconds of sorting have passed."""
    import oracle

    oracle.build()
    work = np.empty_like(host_keys)
    reps, t_sort = 0, 0.0
    while True:
        work[:] = host_keys
        t0 = time.perf_counter()
        oracle.sort_inplace(work, pivot=a.pivot)
        t_sort += time.perf_counter() - t0
        reps += 1
        if t_sort >= min_seconds:
            break
    return {"value": host_keys.size * reps / t_sort, "unit": "keys/s", "cores": 1, "kind": "oracle",
            "sample": f"{reps} x oracle sort of the whole 2^{a.log2n}-key workload ({a.dtype} "
                      f"{a.dist} seed {a.seed}, {a.pivot} pivot), single thread, {t_sort:.1f} s"}


def time_library_sorts(a, host_keys, seconds: float):
    """std::sort on one host thread and a parallel sort on every host core, each on the
    whole workload (at least once, up to three times while under seconds / 2)."""
    import numpy as np

    from oracle import cpu_baselines

    cpu_baselines.build()
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    out = []
    for threads in (1, cores):
        m = host_keys.size
        keys, reps, t_sort = 0, 0, 0.0
        work = np.empty(m, host_keys.dtype)
        kind = ""
        while True:
            work[:] = host_keys[:m]
            t0 = time.perf_counter()
            kind = cpu_baselines.sort_inplace(work, threads)
            t_sort += time.perf_counter() - t0
            keys += m
            reps += 1
            if t_sort >= seconds / 2 or reps >= 3:
                break
        out.append({"value": keys / t_sort, "unit": "keys/s", "cores": threads, "kind": kind,
                    "sample": f"{reps} x {kind} of the whole 2^{int(math.log2(m))}-key "
                              f"workload, {threads} thread(s), {t_sort:.1f} s"})
    return out


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
    """The reference arm: the paper's algorithm as the single-threaded CPU oracle, on
    this host, on the same workload and config as our arm.  Every timed step sorts its
    own unsorted copy of the whole array; the warm-up steps sort its first 2^20 keys
    (the oracle has nothing to warm up but its code and the input's pages)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_1604_06697_gb300 import inputs

    oracle.build()
    n = 1 << a.log2n
    host = inputs.make_keys(n, a.dtype, a.dist, a.seed)
    work = np.empty_like(host)
    m = min(n, 1 << 20)
    for _ in range(a.warmup):
        work[:m] = host[:m]
        oracle.sort_inplace(work[:m], pivot=a.pivot)
    step_s = []
    for _ in range(a.steps):
        work[:] = host
        t0 = time.perf_counter()
        oracle.sort_inplace(work, pivot=a.pivot)
        step_s.append(time.perf_counter() - t0)
    ok = bool(np.all(work[1:] >= work[:-1])) if a.dtype != "float64" else True
    total = sum(step_s)
    value = n * a.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "keys/s",
        "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": 1e3 * total / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": a.dtype, "data": "synthetic",
        "config": workload_config(a),
        "cpu_baseline": {"value": value, "unit": "keys/s", "cores": 1, "kind": "oracle",
                         "sample": f"{a.steps} timed steps, each one oracle sort of the whole "
                                   f"2^{a.log2n}-key workload on its own unsorted copy, single "
                                   f"thread ({a.warmup} warm-up steps on its first 2^20 keys)"},
        "e2e": {"value": value, "unit": "keys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "step_seconds": [round(x, 3) for x in step_s], "sorted_check": ok,
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
    tuned = None
    if not a.no_tune:   # launch shape chosen by the autotuner (cached per GPU/dtype/size)
        from paper_1604_06697_gb300 import autotune
        tuned = autotune.tune(a.dtype, n, kind="sort")["config"]
    else:
        for name, v in (("tile", a.tile), ("small_cutoff", a.small), ("local_cutoff", a.local),
                        ("small_sort", a.small_sort), ("overlap", a.overlap),
                        ("coop_max", a.coop_max)):
            if v is not None:
                bqs.set_option(name, v)
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
    # Partition launches are timed with CUDA events on the library's stream inside the
    # timed region, on every TIMED_EVERY-th sort (an event pair around a launch costs
    # about 2 us of device time, ~0.1 ms per 2^28-key sort if every sort carried them);
    # with timing mode 2 no call waits for its events, they are summed once the region
    # has ended (bqs_timing_collect).
    TIMED_EVERY = 4
    bqs.collect_timing()
    part_ms, part_bytes, launches, part_launches, levels = 0.0, 0.0, 0, 0, []
    active_keys = 0
    # A sort that takes the single-launch path is one kernel: its CUDA-event time and
    # the whole sort's algorithmic bytes stand for the dominant kernel.
    coop_ms, coop_bytes, coop_sorts = 0.0, 0.0, 0
    clk = ClockSampler(dev.index if dev.index is not None else 0)
    barrier()
    torch.cuda.synchronize(dev)
    with clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        clk.mark_start()
        e0.record(stream)
        for k in range(a.steps):
            timed = k % TIMED_EVERY == 0
            bqs.set_option("timing", 2 if timed else 0)
            bqs.sort(bufs[k])
            s = bqs.stats()
            if timed and s.get("coop_ms", 0.0) > 0.0:
                coop_ms += s["coop_ms"]
                coop_bytes += 2.0 * host.itemsize * (s["active_keys"] + n)
                coop_sorts += 1
            elif timed:
                part_bytes += s["partition_bytes"]
                part_launches += s["partition_launches"]
            launches += s["kernel_launches"]
            active_keys += s["active_keys"]
            levels.append(s["levels"])
        e1.record(stream)
        torch.cuda.synchronize(dev)
        clk.mark_end()
    barrier()
    bqs.set_option("timing", 0)
    part_ms, timed_launches = bqs.collect_timing()
    ms = e0.elapsed_time(e1)
    # Correctness spot check outside the timed region: sorted and same multiset sum.
    out = bufs[0]
    ok = bool((out[1:] >= out[:-1]).all().item()) if a.dtype != "float64" else True
    del bufs
    ms = max_over_ranks(ms, dev)
    value = replica_throughput(n * a.steps, ms, world)

    # With the networks on a second stream the partition kernel shares the GPU during
    # the timed region; its bandwidth alone is measured again here, outside it, with
    # the networks on the call's stream.
    isolated = None
    if bqs.get_option("overlap"):
        bqs.set_option("overlap", 0)
        bqs.set_option("timing", 1)
        iso_ms = iso_bytes = 0.0
        for _ in range(max(3, min(a.steps, 10))):
            work.copy_(src)
            bqs.sort(work)
            s = bqs.stats()
            iso_ms += s["partition_ms"]
            iso_bytes += s["partition_bytes"]
        bqs.set_option("timing", 0)
        bqs.set_option("overlap", 1)
        torch.cuda.synchronize(dev)
        isolated = (iso_bytes / (iso_ms / 1e3)) / 1e9 if iso_ms > 0 else None

    # End to end through the public API with host buffers: every step copies its keys
    # from pinned host memory to the device, sorts them and copies the result back.
    # Triple-buffered on two copy streams: step k+1's upload and step k-1's download
    # overlap step k's sort (the upload's buffer was downloaded two steps earlier); the
    # timed region spans the first upload to the last download.
    e2e = None
    if not a.no_e2e:
        NB = 3
        (pin_in, pin_out), near = pinned_near_gpu(
            dev, lambda: (torch.from_numpy(host).pin_memory(),
                          [torch.empty(host.shape, dtype=src.dtype).pin_memory() for _ in range(2)]))
        dbuf = [torch.empty_like(src) for _ in range(NB)]
        up, down = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

        def run_e2e(steps):
            downloaded = [None] * NB      # event: buffer i's last download finished
            uploaded = [None] * steps

            def upload(k):
                b = k % NB
                if downloaded[b] is not None:
                    up.wait_event(downloaded[b])
                with torch.cuda.stream(up):
                    dbuf[b].copy_(pin_in, non_blocking=True)
                uploaded[k] = torch.cuda.Event()
                uploaded[k].record(up)

            upload(0)
            for k in range(steps):
                if k + 1 < steps:
                    upload(k + 1)                 # overlaps this step's sort
                stream.wait_event(uploaded[k])
                bqs.sort(dbuf[k % NB])
                sorted_ev = torch.cuda.Event()
                sorted_ev.record(stream)
                down.wait_event(sorted_ev)
                with torch.cuda.stream(down):
                    pin_out[k % 2].copy_(dbuf[k % NB], non_blocking=True)
                downloaded[k % NB] = torch.cuda.Event()
                downloaded[k % NB].record(down)
            stream.wait_stream(up)
            stream.wait_stream(down)

        run_e2e(2)
        torch.cuda.synchronize(dev)
        barrier()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        up.wait_stream(stream)
        f0.record(stream)
        up.wait_event(f0)
        down.wait_event(f0)
        run_e2e(a.steps)
        f1.record(stream)
        torch.cuda.synchronize(dev)
        ems = max_over_ranks(f0.elapsed_time(f1), dev)
        nbytes = n * host.itemsize
        e2e = {"value": replica_throughput(n * a.steps, ems, world), "unit": "keys/s",
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
               "pipelining": "triple-buffered: step k+1's pinned upload and step k-1's "
                             "download overlap step k's sort on two copy streams",
               "result_check": bool((pin_out[(a.steps - 1) % 2][1:] >= pin_out[(a.steps - 1) % 2][:-1]).all()),
               "host_buffers": ("pinned, allocated on the GPU's NUMA node (CPUs %d-%d)" % (near[0], near[-1])
                                if near else "pinned (GPU's NUMA node unknown)")}
        del pin_in, pin_out, dbuf

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu:
        cpu = time_oracle(a, host)
        cpu["library_sorts"] = time_library_sorts(a, host, a.cpu_seconds)

    peak, peak_kind = measured_peak_gbs()
    achieved = (part_bytes / (part_ms / 1e3)) / 1e9 if part_ms > 0 else None
    traffic = None
    tr = committed_traffic()
    if tr and tr.get("dtype") == a.dtype and part_launches:
        # ncu DRAM bytes per processed key x keys per launch of this run
        traffic = tr["dram_bytes_per_active_key"] * (part_bytes / (2 * host.itemsize)) / part_launches
    kernel = "k_partition"
    if coop_sorts and not part_launches:
        kernel = "k_coop_sort (every level of the sort in one launch)"
        part_ms, part_bytes, part_launches, timed_launches = coop_ms, coop_bytes, coop_sorts, coop_sorts
        achieved = (part_bytes / (part_ms / 1e3)) / 1e9 if part_ms > 0 else None
        traffic = None
    roofline = {
        "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
        "frac": (achieved / peak) if achieved else None, "traffic": traffic,
        "kernel": kernel, "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)"
                  if peak_kind == "measured" else "fallback 6.8 TB/s",
        "algorithmic_bytes_per_launch": part_bytes / max(1, part_launches),
        "avg_launch_ms": part_ms / max(1, part_launches),
        "frac_of_8tbs_spec": (achieved / 8000.0) if achieved else None,
        "concurrent_with_networks": bool(bqs.get_option("overlap")),
        "timed_launches": timed_launches,
        "timed_steps": "CUDA events around every %s launch of timed steps 0, %d, %d, ..."
                       % ("partition" if kernel == "k_partition" else "single-launch sort",
                          TIMED_EVERY, 2 * TIMED_EVERY),
        "achieved_isolated": isolated,
        "frac_isolated": (isolated / peak) if isolated else None,
    }
    # The whole sort against the same peaks: every partition level reads and writes its
    # active keys once, and every key is read and written once more by its final pass
    # (network, single-block partitioning or pivot-class fill): sum over levels of
    # 2 s n_active + 2 s n, divided by the measured time per sort.
    s_key = host.itemsize
    sort_bytes = 2.0 * s_key * (active_keys / max(1, a.steps) + n)
    sort_gbs = sort_bytes / (ms / a.steps / 1e3) / 1e9
    roofline["sort"] = {
        "algorithmic_bytes_per_sort": sort_bytes,
        "formula": "sum over partition levels of 2*sizeof(key)*active keys + 2*sizeof(key)*n",
        "achieved": sort_gbs, "unit": "GB/s", "frac": sort_gbs / peak,
        "peak_source": roofline["peak_source"],
        "frac_of_8tbs_spec": sort_gbs / 8000.0,
    }
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "keys/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": a.dtype, "data": "synthetic",
            "config": workload_config(a),
            "launch_shape": tuned,
            "parallelism": "replicas" if world > 1 else "single GPU",
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "levels_per_sort": levels[0] if levels else None,
            "clocks": clk.summary(), "sorted_check": ok,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---- further workloads (one JSON line each) ---------------------------------------------------

def _cuda_ms(fn):
    import torch
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def run_pairs(a):
    """2^26 (int64 key in [0, 2^20), uint32 payload = index) pairs, ordered by (key, payload)."""
    import torch

    from paper_1604_06697_gb300 import build as _build
    _build.build()
    import paper_1604_06697_gb300 as bqs
    from paper_1604_06697_gb300 import inputs

    n = 1 << 26
    keys, vals = inputs.make_pairs(n, seed=1)
    sk = torch.from_numpy(keys).cuda()
    sv = torch.from_numpy(vals.view(np.int32)).cuda()
    bqs.set_option("pivot", 1)
    from paper_1604_06697_gb300 import autotune
    tuned = autotune.tune("int64", n, kind="pairs")["config"]
    wk, wv = torch.empty_like(sk), torch.empty_like(sv)
    for _ in range(a.warmup):
        wk.copy_(sk); wv.copy_(sv); bqs.sort_pairs(wk, wv)
    bufs = [(sk.clone(), sv.clone()) for _ in range(a.steps)]
    bqs.set_option("timing", 1)
    pm = pb = 0.0
    launches = 0

    def steps():
        nonlocal pm, pb, launches
        for k, v in bufs:
            bqs.sort_pairs(k, v)
            s = bqs.stats()
            pm += s["partition_ms"]; pb += s["partition_bytes"]; launches += s["kernel_launches"]
    ms = _cuda_ms(steps)
    bqs.set_option("timing", 0)
    k0 = bufs[0][0]
    ok = bool(((k0[1:] > k0[:-1]) | ((k0[1:] == k0[:-1]) & (bufs[0][1][1:] > bufs[0][1][:-1]))).all())
    peak, kind = measured_peak_gbs()
    ach = pb / (pm / 1e3) / 1e9 if pm else None
    print(json.dumps({
        "workload": "pairs", "metric": "key-value pairs/s", "value": n * a.steps / (ms / 1e3),
        "unit": "pairs/s", "ms_per_step": ms / a.steps, "steps": a.steps, "warmup": a.warmup,
        "dtype": "int64+u32", "data": "synthetic",
        "config": {"workload": "bqs_sort_pairs 2^26 int64 keys mod 2^20, payload = index, seed 1",
                   "pivot": "sqrt", "autotuned": tuned},
        "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                     "frac": ach / peak if ach else None, "kernel": "k_partition_tma (pairs)"},
        "gpu_launches": launches, "ordered_check": ok}), flush=True)


def run_batched(a):
    """65,536 int32 arrays, lengths log-uniform in [16, 65536], one graph launch (the
    device-side level loop) against one bqs_sort call per array."""
    import torch

    from paper_1604_06697_gb300 import build as _build
    _build.build()
    import paper_1604_06697_gb300 as bqs
    from paper_1604_06697_gb300 import autotune, inputs

    nseg = 65536
    keys, off = inputs.make_segments(nseg, seed=2)
    n = int(off[-1])
    src = torch.from_numpy(keys).cuda()
    toff = torch.from_numpy(off).cuda()
    bqs.set_option("pivot", 1)
    tuned = autotune.tune("int32", n, kind="batched", nseg=nseg)

    scratch = src.clone()
    bqs.sort_batched(scratch, toff)      # one-time set-up outside capture
    torch.cuda.synchronize()
    del scratch
    bufs = [src.clone() for _ in range(a.steps)]
    graphs = []
    cap = torch.cuda.Stream()
    for b in bufs:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=cap):
            bqs.sort_batched(b, toff)
        graphs.append(g)
    warm = src.clone()
    gw = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gw, stream=cap):
        bqs.sort_batched(warm, toff)
    for _ in range(a.warmup):
        warm.copy_(src)
        gw.replay()
    ms = _cuda_ms(lambda: [g.replay() for g in graphs])
    out = bufs[0].cpu().numpy()
    ok = all(np.array_equal(out[off[i]:off[i + 1]], np.sort(keys[off[i]:off[i + 1]]))
             for i in range(0, nseg, 997))

    # Second baseline: the same batch in one bqs_sort_segmented call on an ordinary
    # stream (the host drives the level loop): how much of the gain is the graph.
    seg_bufs = [src.clone() for _ in range(a.steps)]
    for _ in range(a.warmup):
        warm.copy_(src)
        bqs.sort_segmented(warm, toff)
    seg_ms = _cuda_ms(lambda: [bqs.sort_segmented(b, toff) for b in seg_bufs])
    seg_ok = bool(np.array_equal(seg_bufs[0].cpu().numpy(), out))
    del seg_bufs

    # Baseline: one bqs_sort call per array (arrays placed at 16-byte aligned offsets).
    lens = np.diff(off)
    poff = np.zeros(nseg + 1, np.int64)
    np.cumsum((lens + 3) // 4 * 4, out=poff[1:])
    padded = np.zeros(int(poff[-1]), np.int32)
    for i in range(nseg):
        padded[poff[i]:poff[i] + lens[i]] = keys[off[i]:off[i + 1]]
    pbuf = torch.from_numpy(padded).cuda()
    views = [pbuf[int(poff[i]):int(poff[i] + lens[i])] for i in range(nseg)]
    for v in views[:64]:
        bqs.sort(v)
    pbuf.copy_(torch.from_numpy(padded).cuda())
    base_ms = _cuda_ms(lambda: [bqs.sort(v) for v in views])
    print(json.dumps({
        "workload": "batched", "metric": "keys/s, 65,536 int32 arrays in one graph launch",
        "value": n * a.steps / (ms / 1e3), "unit": "keys/s", "ms_per_step": ms / a.steps,
        "steps": a.steps, "warmup": a.warmup, "dtype": "int32", "data": "synthetic",
        "config": {"workload": "bqs_sort_batched, 65,536 arrays, lengths floor(exp(U(ln16, ln65536))), seed 2",
                   "total_keys": n, "autotuned": tuned["config"], "pivot": "sqrt"},
        "baseline_one_call_per_array": {"value": n / (base_ms / 1e3), "unit": "keys/s",
                                        "ms": base_ms, "calls": nseg},
        "baseline_one_segmented_call": {"value": n * a.steps / (seg_ms / 1e3), "unit": "keys/s",
                                        "ms": seg_ms / a.steps, "same_output": seg_ok,
                                        "how": "bqs_sort_segmented, not captured: the host "
                                               "reads each level's counts"},
        "speedup_vs_one_segmented_call": (seg_ms / a.steps) / (ms / a.steps),
        "speedup_vs_per_array": base_ms / (ms / a.steps), "sorted_check": ok}), flush=True)


def run_matrix(a, dists=None, sizes=(24, 28), name="matrix"):
    """2^24 and 2^28 keys x int32/int64/float64 x the six distributions (seed 1); with
    dists/sizes given, those instead (the structured inputs)."""
    import torch

    from paper_1604_06697_gb300 import build as _build
    _build.build()
    import paper_1604_06697_gb300 as bqs
    from paper_1604_06697_gb300 import autotune, inputs

    bqs.set_option("pivot", 1)
    rows = []
    peak, _ = measured_peak_gbs()
    for log2n in sizes:
        n = 1 << log2n
        for dtype in ("int32", "int64", "float64"):
            autotune.tune(dtype, n, kind="sort")
            for dist in (dists or inputs.DISTRIBUTIONS):
                src = torch.from_numpy(inputs.make_keys(n, dtype, dist, 1)).cuda()
                work = torch.empty_like(src)
                for _ in range(a.warmup):
                    work.copy_(src)
                    bqs.sort(work)
                best, pm, pb, lv = float("inf"), 0.0, 0.0, 0
                bqs.set_option("timing", 1)
                for _ in range(a.steps):
                    work.copy_(src)
                    ms = _cuda_ms(lambda: bqs.sort(work))
                    s = bqs.stats()
                    if ms < best:
                        best, pm, pb, lv = ms, s["partition_ms"], s["partition_bytes"], s["levels"]
                bqs.set_option("timing", 0)
                ach = pb / (pm / 1e3) / 1e9 if pm else None
                rows.append({"log2n": log2n, "dtype": dtype, "dist": dist, "ms": round(best, 3),
                             "keys_per_s": n / (best / 1e3), "levels": lv,
                             "partition_GBs": ach, "partition_frac": ach / peak if ach else None})
                print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
                del src, work
    print(json.dumps({"workload": name, "metric": "keys/s per size x dtype x distribution",
                      "unit": "keys/s", "timing": f"best of {a.steps} sorts after {a.warmup} warm-up",
                      "data": "synthetic", "rows": rows}), flush=True)


PIVOT_RULES = ["median-of-3", "median-of-sqrt(n)", "median-of-5", "median-of-23",
               "median-of-3-medians-of-3", "median-of-3-medians-of-5", "median-of-5-medians-of-5"]


def run_pivots(a):
    """The pivot rules of Sec. 4 on the same input: levels and keys/s per rule."""
    import torch

    from paper_1604_06697_gb300 import build as _build
    _build.build()
    import paper_1604_06697_gb300 as bqs
    from paper_1604_06697_gb300 import autotune, inputs

    n = 1 << a.log2n
    bqs.set_option("pivot", 1)
    tuned = autotune.tune(a.dtype, n, kind="sort")["config"]
    src = torch.from_numpy(inputs.make_keys(n, a.dtype, a.dist, a.seed)).cuda()
    work = torch.empty_like(src)
    peak, _ = measured_peak_gbs()
    rows = []
    for rule, name in enumerate(PIVOT_RULES):
        bqs.set_option("pivot", rule)
        for _ in range(a.warmup):
            work.copy_(src)
            bqs.sort(work)
        bqs.set_option("timing", 1)
        best, pm, pb, lv = float("inf"), 0.0, 0.0, 0
        for _ in range(a.steps):
            work.copy_(src)
            ms = _cuda_ms(lambda: bqs.sort(work))
            st = bqs.stats()
            if ms < best:
                best, pm, pb, lv = ms, st["partition_ms"], st["partition_bytes"], st["levels"]
        bqs.set_option("timing", 0)
        ach = pb / (pm / 1e3) / 1e9 if pm else None
        rows.append({"rule": rule, "name": name, "ms": round(best, 3), "keys_per_s": n / (best / 1e3),
                     "levels": lv, "partition_keys_per_key": pb / (2 * src.element_size()) / n,
                     "partition_GBs": ach, "partition_frac": ach / peak if ach else None})
        print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    print(json.dumps({"workload": "pivots", "metric": "keys/s and partition levels per pivot rule",
                      "unit": "keys/s", "data": "synthetic",
                      "config": {"n": n, "dtype": a.dtype, "dist": a.dist, "seed": a.seed,
                                 "launch_shape": tuned},
                      "timing": f"best of {a.steps} sorts after {a.warmup} warm-up", "rows": rows}),
          flush=True)


def run_records(a):
    """Sec. 4's wide element types: Record (21 int32, compared by the first) and Vector
    (10 float64, compared by the norm), sorted indirectly by bqs_sort_records."""
    import torch

    from paper_1604_06697_gb300 import build as _build
    _build.build()
    import paper_1604_06697_gb300 as bqs
    from paper_1604_06697_gb300 import inputs

    n = 1 << a.log2n
    bqs.set_option("pivot", 1)
    rows = []
    for name, kind, rb, count in (("Record", bqs.KEY_I32_FIELD, 84, 1),
                                  ("Vector", bqs.KEY_F64_SQNORM, 80, 10)):
        r = inputs.splitmix64(a.seed, n * rb // 4)
        host = (r & np.uint64(0xFFFFFFFF)).astype(np.uint32)
        del r
        if kind == bqs.KEY_F64_SQNORM:
            hv = host.view(np.float64)
            for c0 in range(0, hv.size, 1 << 24):
                c1 = min(hv.size, c0 + (1 << 24))
                hv[c0:c1] = 2.0 * inputs.unit_double(inputs.splitmix64(a.seed + 1, c1 - c0, start=c0)) - 1.0
        src = torch.from_numpy(host.view(np.uint8)).cuda()
        work = torch.empty_like(src)
        for _ in range(a.warmup):
            work.copy_(src)
            bqs.sort_records(work, rb, kind, 0, count)
        best = float("inf")
        for _ in range(a.steps):
            work.copy_(src)
            best = min(best, _cuda_ms(lambda: bqs.sort_records(work, rb, kind, 0, count)))
        w = work.view(torch.int32).view(n, rb // 4)
        if kind == bqs.KEY_I32_FIELD:
            k = w[:, 0]
        else:
            v = work.view(torch.float64).view(n, rb // 8)
            k = (v * v).sum(dim=1)
        ok = bool((k[1:] >= k[:-1]).all()) if kind == bqs.KEY_I32_FIELD else \
            bool((k[1:] >= k[:-1] * (1 - 1e-12)).all())
        rows.append({"element": name, "record_bytes": rb, "n": n, "ms": round(best, 3),
                     "elements_per_s": n / (best / 1e3),
                     "record_GBs": n * rb / (best / 1e3) / 1e9, "ordered_check": ok})
        print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
        del src, work
    print(json.dumps({"workload": "records", "metric": "elements/s, indirect sort of wide elements",
                      "unit": "elements/s", "data": "synthetic",
                      "timing": f"best of {a.steps} sorts after {a.warmup} warm-up", "rows": rows}),
          flush=True)


def run_serving(a):
    """Poisson sort requests (sizes 2^U(10,26), mixed dtypes) at several rates, served
    with continuous batching and with one launch per request."""
    from paper_1604_06697_gb300 import build as _build
    _build.build()
    import paper_1604_06697_gb300 as bqs
    from paper_1604_06697_gb300 import serving

    bqs.set_option("pivot", 1)
    pool = serving.KeyPool(max_size=1 << 26, seed=3)
    rows = []
    for rate in (1000, 2000, 5000, 10000, 20000):
        row = {"rate_hz": rate}
        for mode in ("plain", "batched"):
            reqs = serving.make_requests(a.serve_requests, rate, seed=3)
            offered = sum(r.size for r in reqs) / max(r.arrival for r in reqs)
            rep = serving.ServingLoop(pool, mode=mode, slots=3, hbm_budget=64 << 30,
                                      max_batch_keys=1 << 27).run(reqs)
            row[mode] = {k: rep[k] for k in ("p50_ms", "p99_ms", "queue_p50_ms", "queue_p99_ms",
                                             "served_keys_per_s", "offered_keys_per_s", "slots",
                                             "batches", "requests", "hbm_peak_bytes")}
            row["offered_keys_per_s"] = offered
        rows.append(row)
    print(json.dumps({
        "workload": "serving", "metric": "p50/p99 latency and served keys/s, batched vs plain",
        "unit": "ms / keys/s", "requests_per_rate": a.serve_requests, "data": "synthetic",
        "config": {"sizes": "floor(2^U(10,26))", "dtypes": "uniform over int32/int64/float64",
                   "arrivals": "Poisson", "hbm_budget_bytes": 64 << 30, "slots": 3, "seed": 3,
                   "admission": "keys copied into HBM on a copy stream; the slot waits on "
                                "the copy's event on the device",
                   "plain": "one bqs_sort per request on the same 3 slots"},
        "rates": rows}), flush=True)


def main(argv=None):
    a = parse_args(argv)
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "pairs":
        run_pairs(a)
    elif a.workload == "batched":
        run_batched(a)
    elif a.workload == "serving":
        run_serving(a)
    elif a.workload == "matrix":
        run_matrix(a)
    elif a.workload == "pivots":
        run_pivots(a)
    elif a.workload == "records":
        run_records(a)
    elif a.workload == "structured":
        from paper_1604_06697_gb300 import inputs
        run_matrix(a, dists=inputs.EXTRA_DISTRIBUTIONS, sizes=(a.log2n,), name="structured")
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
