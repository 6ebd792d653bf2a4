"""The benchmark's reference arm (the FP64 oracle timed on the host cores, no
GPU needed) prints exactly one JSON line carrying the benchmark's keys, its own
CPU-baseline description and an end-to-end entry without device copies."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    run = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], cwd=ROOT, capture_output=True, text=True,
                         timeout=900, check=True)
    lines = [ln for ln in run.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, run.stdout
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert (d["n_gpus"], d["steps"], d["warmup"]) == (1, 1, 3)
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["higher_is_better"] is True
    assert d["vs_baseline"] is None and d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"]
    assert cb["value"] == d["value"] and cb["unit"] == d["unit"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_stage_stamps_skips_repeats_and_counts_clustered(monkeypatch):
    """The stamp reader takes a replan once (by its start stamp), its DBSCAN
    phases only when the replan clustered (phase stamps after the prune's end),
    and restarts the episodes on schedule."""
    import numpy as np
    import torch
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)

    def stamps(t0, clustered):
        c = np.zeros(16, np.int64)
        c[9] = t0                       # kernel start
        c[10] = t0 + 100                # end of prune
        if clustered:
            c[0:9] = t0 + 100 + 10 * np.arange(1, 10)   # DBSCAN phases
            c[11] = t0 + 100 + 95       # end of DBSCAN
        else:
            c[0:9] = t0 - 50            # left from an earlier replan
            c[11] = t0 + 100
        c[12] = c[11] + 40              # statistics, selection, weights
        c[13] = c[12] + 7               # (dense update sums)
        c[14] = c[13] + 30              # update and shift
        return c

    class Fake:
        def __init__(self, seq):
            self.seq, self.i = seq, -1

        def step(self):
            self.i += 1

        def peek(self, name):
            assert name == "DBCYC"
            return self.seq[self.i]

    a = Fake([stamps(1000, True), stamps(2000, True), stamps(3000, True), stamps(4000, True)])
    b = Fake([stamps(500, False), stamps(500, False), stamps(900, True), stamps(900, True)])
    restarts = []

    def replay():
        a.step()
        b.step()

    out = bench.stage_stamps([a, b], replay, lambda: restarts.append(1), n_steps=4, episode=3)
    assert restarts == [1]
    assert out["replans"] == 4 + 2 and out["clustered"] == 4 + 1
    assert out["prune"] == [100, 100] and out["dbscan"] == [95, 95]
    assert out["dbscan_phases"]["cell unions"] == [10, 10]
    assert out["select_weights"] == [40, 40] and out["update_shift"] == [30, 30]
    assert out["kernel"][1] == 100 + 95 + 77
