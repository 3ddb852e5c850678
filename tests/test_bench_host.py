"""Host-side helpers of bench.py that need no GPU."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


@pytest.mark.skipif(not hasattr(os, "sched_getaffinity"), reason="no CPU affinity API")
def test_pinned_buffers_bind_to_the_gpu_node_and_restore_affinity(monkeypatch):
    before = os.sched_getaffinity(0)
    node = {min(before)}                      # pretend the GPU's node holds one CPU
    monkeypatch.setattr(bench, "gpu_local_cpus", lambda dev: node)
    seen = []
    out, used = bench.pinned_near_gpu(0, lambda: seen.append(os.sched_getaffinity(0)) or "buf")
    assert out == "buf" and seen == [node] and used == sorted(node)
    assert os.sched_getaffinity(0) == before
    # unknown node: nothing changes
    monkeypatch.setattr(bench, "gpu_local_cpus", lambda dev: None)
    seen.clear()
    out, used = bench.pinned_near_gpu(0, lambda: seen.append(os.sched_getaffinity(0)) or "buf")
    assert used is None and seen == [before] and os.sched_getaffinity(0) == before


def test_autotune_candidates_cover_every_knob_once():
    from paper_1604_06697_gb300 import autotune
    for kind in ("sort", "pairs", "batched"):
        cands = autotune.candidate_configs(kind)
        keys = [tuple(sorted(c.items())) for c in cands]
        assert len(keys) == len(set(keys))                       # no duplicates
        assert all(set(c) == set(autotune.KNOBS) for c in cands)
        coop = [c for c in cands if c["coop_max"]]
        # the single-launch path: single arrays only, one candidate per cutoff, with
        # the settings it needs (no local partitioning, warp-group networks)
        assert len(coop) == (len(autotune.SMALL_CUTOFFS) if kind == "sort" else 0)
        assert all(c["small_sort"] == 0 and c["local_cutoff"] == 0 for c in coop)
        assert autotune.candidate_configs(kind, n=autotune.COOP_MAX + 1) == \
            [c for c in cands if not c["coop_max"]]
        cands = [c for c in cands if not c["coop_max"]]
        for c in cands:                                          # 4096 only where it applies
            if c["small_cutoff"] > 2048:
                assert kind != "pairs" and c["small_sort"] == 0
        big = [c for c in cands if c["small_cutoff"] > 2048]
        per_cutoff = len(autotune.TILES) * len(autotune.LOCAL_CUTOFFS) * len(autotune.OVERLAPS)
        assert len(big) == (0 if kind == "pairs" else per_cutoff)
        assert len(cands) - len(big) == per_cutoff * len(autotune.SMALL_SORTS) * 3


def test_reference_arm_runs_the_same_config(capsys):
    import json
    bench.main(["--impl", "reference", "--log2n", "14", "--steps", "2", "--warmup", "1"])
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    a = bench.parse_args(["--log2n", "14"])
    assert line["impl"] == "reference" and line["config"] == bench.workload_config(a)
    assert line["steps"] == 2 and len(line["step_seconds"]) == 2 and line["sorted_check"]
    assert abs(line["ms_per_step"] - 1e3 * sum(line["step_seconds"]) / 2) < 1.0
    assert line["value"] == line["cpu_baseline"]["value"] == line["e2e"]["value"]
    assert line["cpu_baseline"]["cores"] == 1 and line["cpu_baseline"]["kind"] == "oracle"
