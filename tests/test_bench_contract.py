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


def test_sampled_parity_reads_the_stored_oracle_values():
    """bench.sampled_parity against a result that holds the stored FP64 oracle values at the
    sampled pairs: zero error; scaled by 1 + 3e-5: that relative error; another workload: None."""
    import numpy as np

    w = bench.WORKLOADS["survey512"]
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "survey512_sampled_pairs.json")))
    nb = len(w["edges"]) - 1
    res = {k: np.zeros((len(w["ells"]), nb, nb)) for k in ("B", "shot", "window", "window_shot")}
    for rec in gold["values"]:
        im = [tuple(e) for e in w["ells"]].index(tuple(rec["ells"]))
        for k in res:
            res[k][im, rec["b1"], rec["b2"]] = rec[k]
    out = bench.sampled_parity(w, gold["workload"]["seed"], res)
    assert out["pairs"] == len(gold["values"]) and max(out["max_rel_err"].values()) == 0.0 and out["pass"]
    scaled = {k: v * (1 + 3e-5) for k, v in res.items()}
    out = bench.sampled_parity(w, gold["workload"]["seed"], scaled)
    assert all(abs(e - 3e-5) < 1e-9 for e in out["max_rel_err"].values()) and out["pass"]
    out = bench.sampled_parity(w, gold["workload"]["seed"], {k: v * (1 + 3e-4) for k, v in res.items()})
    assert not out["pass"]
    assert bench.sampled_parity(bench.WORKLOADS["box256"], 1002, res) is None
    assert bench.sampled_parity(w, 7, res) is None
