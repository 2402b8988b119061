"""The benchmark's JSON contract on the host side: metric names, bin counts and the oracle
(reference) arm on a small workload, which runs without a GPU."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bin_counts_and_metric_names():
    w = bench.WORKLOADS["survey512"]
    # B000 and B112 over k1 <= k2 (325 each), B202 over all 625 pairs, twice with the window
    assert bench.n_bins_output(w) == 2 * (325 + 625 + 325)
    assert bench.n_bins_output(bench.WORKLOADS["box1024"]) == 820 + 1600 + 820 + 820
    assert bench.n_bins_output(bench.WORKLOADS["batch64"]) == 120 + 225
    assert bench.metric_name(w).startswith("B_l1l2L(k1,k2) bins/s at 512^3")
    assert bench.metric_name(bench.WORKLOADS["survey512_zeta"]).startswith("zeta_l1l2L(r1,r2) bins/s")
    cfg = bench.config_of("survey512", w, 1)
    assert cfg["workload"] == "survey512" and cfg["bins_per_step"] == 2550


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "box64",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "higher_is_better", "config",
              "cpu_baseline", "e2e"):
        assert k in out, k
    assert out["impl"] == "reference" and out["value"] > 0 and out["cpu_baseline"]["kind"] == "oracle"
