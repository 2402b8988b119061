"""Benchmark: bispectrum multipoles B_{l1 l2 L}(k1, k2) per second.

Default workload (the 512^3 configuration the metric is quoted on): a survey-like
catalogue with a local line of sight - 3000 Mpc/h box, 512^3 mesh, observer at
(1500, 1500, -300) Mpc/h, 1e6 galaxies in a 1000-1700 Mpc/h shell inside a 60x60 degree
cap with a Gaussian n(r) (mean 1350, sigma 200 Mpc/h), 5e7 randoms with the same n(r),
FKP weights with P0 = 1e4, TSC with interlacing; B000, B202 and B112 on 25 bins of width
0.01 h/Mpc from 0.01 h/Mpc, plus the window bispectrum from the randoms.  A step is one
pass of the whole path: assign galaxies, assign randoms, measure (data, shot noise,
window).  Inputs are synthetic (synthcat, seeded) and far larger than L2.

`--impl reference` times the FP64 oracle (the CPU reference of this project) on a
bounded sample on the host cores.  For N > 1 (torchrun) every rank measures its own
independent realisation (replicas; no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "survey512": dict(kind="survey", N=512, L=3000.0, n_gen=256, observer=(1500.0, 1500.0, -300.0),
                      n_gal=1_000_000, n_ran=50_000_000, edges=list(np.round(np.linspace(0.01, 0.26, 26), 6)),
                      ells=[(0, 0, 0), (2, 0, 2), (1, 1, 2)], mas="TSC", interlace=True, P0=1e4, window=True),
    "survey128": dict(kind="survey", N=128, L=3000.0, n_gen=128, observer=(1500.0, 1500.0, -300.0),
                      n_gal=1_000_000 // 64, n_ran=50_000_000 // 64,
                      edges=list(np.round(np.linspace(0.005, 0.13, 26), 6)),
                      ells=[(0, 0, 0), (2, 0, 2), (1, 1, 2)], mas="TSC", interlace=True, P0=1e4, window=True),
    # profiling case: the 512^3 survey mesh geometry (3000 Mpc/h, shells up to 0.26 h/Mpc) with two
    # bins and B000 only, a few GB on the device
    "box512_2bins": dict(kind="box", N=512, L=3000.0, n_gen=256, n_p=1_000_000, edges=[0.24, 0.25, 0.26],
                         ells=[(0, 0, 0)], mas="TSC", interlace=True, P0=0.0, window=False),
    # profiling case: shell batches of nine components with the 512^3 survey's prune ratio
    # (shells up to 0.26 h/Mpc at half the mesh and half the box), about 3 GB on the device
    "box256_l2_2bins": dict(kind="box", N=256, L=1500.0, n_gen=256, n_p=1_000_000, edges=[0.24, 0.25, 0.26],
                            ells=[(0, 0, 0), (2, 0, 2), (1, 1, 2)], mas="TSC", interlace=True, P0=0.0,
                            window=False),
    "box256": dict(kind="box", N=256, L=1000.0, n_gen=256, n_p=4_000_000,
                   edges=list(np.round(np.linspace(0.01, 0.21, 21), 6)),
                   ells=[(0, 0, 0), (1, 1, 0), (2, 2, 0), (2, 0, 2), (1, 1, 2), (2, 2, 2)], mas="TSC",
                   interlace=True, P0=0.0, window=False),
    "box128": dict(kind="box", N=128, L=1000.0, n_gen=128, n_p=500_000,
                   edges=list(np.round(np.linspace(0.01, 0.21, 21), 6)),
                   ells=[(0, 0, 0), (1, 1, 0), (2, 2, 0), (2, 0, 2), (1, 1, 2), (2, 2, 2)], mas="TSC",
                   interlace=True, P0=0.0, window=False),
    # large periodic box: fields of the 40 bins (1.5 TB) do not fit; the shell fields are held in
    # blocks of bins sized from the free device memory
    "box1024": dict(kind="box", N=1024, L=2000.0, n_gen=256, n_p=120_000_000,
                    edges=list(np.round(np.linspace(0.005, 0.405, 41), 6)),
                    ells=[(0, 0, 0), (2, 0, 2), (1, 1, 2), (2, 2, 2)], mas="TSC", interlace=True, P0=0.0,
                    window=False),
    # three-point-function multipoles and window Q on the 512^3 survey: 25 r-bins of 8 Mpc/h
    "survey512_zeta": dict(kind="survey", N=512, L=3000.0, n_gen=256, observer=(1500.0, 1500.0, -300.0),
                           n_gal=1_000_000, n_ran=50_000_000, edges=list(np.round(np.linspace(10.0, 210.0, 26), 6)),
                           ells=[(0, 0, 0), (2, 0, 2), (1, 1, 2)], mas="TSC", interlace=True, P0=1e4, window=True,
                           estimator="threept"),
    # 64 independent periodic realisations on meshes of two sizes (32 at 128^3, 32 at 256^3,
    # 1e6-4e6 particles each), 15 bins, B000 + B202, measured one after another
    "batch64": dict(kind="batch", N=256, L=1000.0, n_real=64, sizes=(128, 256), n_p_range=(1_000_000, 4_000_000),
                    edges=list(np.round(np.linspace(0.01, 0.16, 16), 6)), ells=[(0, 0, 0), (2, 0, 2)], mas="TSC",
                    interlace=True, P0=0.0, window=False),
    "box64": dict(kind="box", N=64, L=1000.0, n_gen=64, n_p=200_000, edges=list(np.round(np.linspace(0.01, 0.21, 11), 6)),
                  ells=[(0, 0, 0), (2, 0, 2)], mas="CIC", interlace=False, P0=0.0, window=False),
}


def n_bins_output(w):
    """Distinct outputs: k1 <= k2 when l1 = l2, all pairs otherwise; twice with the window."""
    nb = len(w["edges"]) - 1
    n = sum(nb * (nb + 1) // 2 if l1 == l2 else nb * nb for (l1, l2, _) in w["ells"])
    return n * (2 if w["window"] else 1)


def make_inputs(w, seed):
    import synthcat

    if w["kind"] == "survey":
        gal, ran = synthcat.survey_catalogs(w["n_gen"], w["L"], w["observer"], w["n_gal"], w["n_ran"], seed)
        return gal, ran
    return {"xyz": synthcat.periodic_catalog(w["n_gen"], w["L"], w["n_p"], seed)}, None


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([s.strip() for s in line.split(",")])

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = [r for r in self.rows if len(r) >= 7]
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[0]) for r in rows if num(r[0])]
        mx = [num(r[1]) for r in rows if num(r[1])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def run_gpu(args, w, rank, world):
    import torch

    import paper_1803_02132_gb300 as bisp
    from paper_1803_02132_gb300 import replicas

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", dev))
    gal, ran = make_inputs(w, seed=1002 + rank)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    g_dev = {k: t(v) for k, v in gal.items()}
    r_dev = {k: t(v) for k, v in ran.items()} if ran is not None else None
    # end-to-end inputs live in pinned host memory (copied in by the library every step)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).pin_memory()
    gal = {k: pin(v) for k, v in gal.items()}
    ran = {k: pin(v) for k, v in ran.items()} if ran is not None else None
    stream = torch.cuda.Stream()
    plan = bisp.Plan(w["N"], w["L"], w["edges"], w["ells"], los="local" if w["kind"] == "survey" else "global",
                     observer=w.get("observer", (0, 0, 0)), mas=w["mas"], interlace=w["interlace"],
                     fkp_P0=w["P0"], want_window=w["window"], stream=stream, precision=args.precision,
                     estimator=w.get("estimator", "bispectrum"))
    f64 = args.precision == "fp64"

    def step(dev_inputs=True):
        if dev_inputs:
            plan.assign(bisp.DATA, g_dev["xyz"], None, g_dev.get("nbar"))
            if r_dev is not None:
                plan.assign(bisp.RANDOMS, r_dev["xyz"], None, r_dev.get("nbar"))
        else:
            plan.assign(bisp.DATA, gal["xyz"], None, gal.get("nbar"))
            if ran is not None:
                plan.assign(bisp.RANDOMS, ran["xyz"], None, ran.get("nbar"))
        return plan.measure()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(dev)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    ms_pair = []
    pair_launches = 0
    pair_bytes = 0.0
    launches = 0
    last = None
    for _ in range(args.steps):
        last = step()
        inf = plan.info()
        ms_pair.append(inf["ms_pair"])
        pair_launches += inf["pair_launches"]
        pair_bytes += inf["pair_bytes"]
        launches += inf["kernel_launches"]
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    info = plan.info()  # stage times of the last device-input step
    # end to end through the public API with host buffers (H2D and D2H inside); the plain
    # FP64 comparison line leaves it out (its device time already runs to tens of seconds)
    ms_e2e = 0.0
    if not f64 and not args.no_e2e:
        # one untimed step with host buffers first: the plan grows its arena once for the staged
        # host inputs, as the device leg's warm-up steps did for theirs
        step(dev_inputs=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step(dev_inputs=False)
        torch.cuda.synchronize()
        ms_e2e = (time.perf_counter() - t0) * 1e3
    ms, ms_e2e = replicas.max_over_ranks([ms, ms_e2e], dist, device="cuda")
    plan.close()
    nbins = n_bins_output(w)
    fp64 = None
    if not f64 and world == 1 and not args.no_fp64_baseline and w.get("estimator", "bispectrum") == "bispectrum":
        try:
            fp64 = fp64_step(bisp, w, g_dev, r_dev, nbins)
            fp64["speedup"] = (nbins / (ms / args.steps / 1e3)) / fp64["value"]
        except Exception as e:  # the comparison must not cost the main line
            fp64 = {"error": str(e)[:300]}
    ms_step = ms / args.steps
    value = replicas.weak_scaling_rate(nbins, ms_step, world)
    h2d = sum(v.numel() * v.element_size() for v in gal.values()) + (
        sum(v.numel() * v.element_size() for v in ran.values()) if ran else 0)
    d2h = (4 if w["window"] else 2) * len(w["ells"]) * (len(w["edges"]) - 1) ** 2 * 8 + (len(w["edges"]) - 1) * 8
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    pair_ms_avg = sum(ms_pair) / max(pair_launches, 1)
    pair_gbs = (pair_bytes / max(pair_launches, 1)) / (pair_ms_avg / 1e3) / 1e9 if pair_ms_avg > 0 else None
    out = {
        "metric": metric_name(w),
        "value": value, "unit": "bins/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if f64 else "f32 (FP64 accumulation)", "data": "synthetic",
        "config": config_of(args.workload, w, world),
        "e2e": None if (f64 or args.no_e2e) else {"value": replicas.weak_scaling_rate(nbins, ms_e2e / args.steps, world),
                                 "unit": "bins/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "kernel": "k_f64_dot3 (plain FP64 mesh sum, one per bin pair and 3j term)"
                     if f64 else "k_pair_tma (mesh sum of F F G, Eq. bi_estimator_FFTs)",
                     "achieved": pair_gbs, "peak": hbm, "unit": "GB/s",
                     "frac": (pair_gbs / hbm) if pair_gbs else None,
                     "traffic": None if f64 else pair_traffic(pair_bytes / max(pair_launches, 1)),
                     "peak_source": "of measured (MEASURED_PEAKS.json hbm_gbs, burst copy)" if "hbm_gbs" in peaks
                     else "of fallback 6800 GB/s"},
        "parity": None if f64 else sampled_parity(w, 1002 + rank, last),
        "stages_ms": {"assign_data": info["ms_assign_data"], "assign_randoms": info["ms_assign_randoms"],
                      "measure": info["ms_measure"], "pair": info["ms_pair"]},
        "clocks": clk,
    }
    if fp64:
        out["fp64_gpu_baseline"] = fp64
    return out


def run_batch(args, w):
    """A campaign of independent realisations (mixed mesh sizes).  Groups of up to 8
    realisations go to 8 plans (4 per mesh size, each on its own stream): the group's catalogues
    are assigned from 8 host threads at once, then bisp_measure_batch measures the group's plans
    concurrently; device-resident inputs."""
    import concurrent.futures as cf

    import torch

    import paper_1803_02132_gb300 as bisp
    import synthcat

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    rng = np.random.default_rng(2004)
    cats = []
    for i in range(w["n_real"]):
        N = w["sizes"][i % len(w["sizes"])]
        n_p = int(rng.integers(w["n_p_range"][0], w["n_p_range"][1] + 1))
        xyz = synthcat.periodic_catalog(N // 2, w["L"], n_p, 3000 + i)
        cats.append((N, torch.from_numpy(np.ascontiguousarray(xyz, np.float32)).cuda()))
    per_size = 4
    plans = {N: [bisp.Plan(N, w["L"], w["edges"], w["ells"], los="global", mas=w["mas"], interlace=w["interlace"])
                 for _ in range(per_size)] for N in w["sizes"]}
    pool = cf.ThreadPoolExecutor(max_workers=per_size * len(w["sizes"]))

    def step():
        st = {"launches": 0, "pair_ms": 0.0, "pair_bytes": 0.0, "pair_launches": 0}
        group = per_size * len(w["sizes"])
        for g0 in range(0, len(cats), group):
            used = {N: 0 for N in w["sizes"]}
            jobs = []
            for N, xyz in cats[g0:g0 + group]:
                jobs.append((plans[N][used[N]], xyz))
                used[N] += 1
            list(pool.map(lambda j: j[0].assign(bisp.DATA, j[1]), jobs))
            bisp.measure_batch([pl for pl, _ in jobs])
            for pl, _ in jobs:
                inf = pl.info()
                st["launches"] += inf["kernel_launches"]
                st["pair_ms"] += inf["ms_pair"]
                st["pair_bytes"] += inf["pair_bytes"]
                st["pair_launches"] += inf["pair_launches"]
        return st

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", 0)))
    clocks.start()
    # the plans run on their own streams: the whole campaign is timed by the host clock between
    # device-wide synchronisations (every call returns after its work has completed)
    t0 = time.perf_counter()
    tot = {"launches": 0, "pair_ms": 0.0, "pair_bytes": 0.0, "pair_launches": 0}
    for _ in range(args.steps):
        st = step()
        for k in tot:
            tot[k] += st[k]
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / args.steps
    clk = clocks.stop()
    pool.shutdown()
    for pls in plans.values():
        for pl in pls:
            pl.close()
    nbins = n_bins_output(w) * w["n_real"]
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    gbs = tot["pair_bytes"] / (tot["pair_ms"] / 1e3) / 1e9 if tot["pair_ms"] > 0 else None
    return {
        "metric": f"B_l1l2L(k1,k2) bins/s, {w['n_real']} realisations at 128^3 and 256^3 (global LOS, B000+B202)",
        "value": nbins / (ms / 1e3), "unit": "bins/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (FP64 accumulation)", "data": "synthetic",
        "config": {"workload": args.workload, "realisations": w["n_real"], "meshes": list(w["sizes"]),
                   "particles": list(w["n_p_range"]), "nbins": len(w["edges"]) - 1, "ells": w["ells"],
                   "bins_per_step": nbins, "schedule": "8 plans (4 per mesh size): groups of 8 realisations "
                                                       "assigned from 8 host threads, measured by one "
                                                       "bisp_measure_batch call (concurrent plans)",
                   "l2": "inputs of 12-48 MB per realisation, fields of 8-64 MB (no flush between measures)"},
        "e2e": None, "gpu_launches": tot["launches"] // args.steps,
        "roofline": {"bound": "hbm", "kernel": "k_pair_tma (mesh sum of F F G, Eq. bi_estimator_FFTs)",
                     "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm if gbs else None, "traffic": None,
                     "peak_source": "of measured (MEASURED_PEAKS.json hbm_gbs, burst copy)" if "hbm_gbs" in peaks
                     else "of fallback 6800 GB/s"},
        "clocks": clk,
    }


def fp64_step(bisp, w, g, r, nbins):
    """One step of the plain FP64 form (cuFFT Z2D fields, one FP64 mesh sum per bin pair and
    3j term) on the same device-resident inputs, timed with CUDA events on its stream."""
    import torch

    stream = torch.cuda.Stream()
    plan = bisp.Plan(w["N"], w["L"], w["edges"], w["ells"], los="local" if w["kind"] == "survey" else "global",
                     observer=w.get("observer", (0, 0, 0)), mas=w["mas"], interlace=w["interlace"],
                     fkp_P0=w["P0"], want_window=w["window"], stream=stream, precision="fp64")
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    plan.assign(bisp.DATA, g["xyz"], None, g.get("nbar"))
    if r is not None:
        plan.assign(bisp.RANDOMS, r["xyz"], None, r.get("nbar"))
    plan.measure()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    inf = plan.info()
    plan.close()
    gbs = inf["pair_bytes"] / (inf["ms_pair"] / 1e3) / 1e9 if inf["ms_pair"] > 0 else None
    return {"value": nbins / (ms / 1e3), "unit": "bins/s", "ms_per_step": ms, "steps": 1, "warmup": 0,
            "dtype": "f64", "form": "plain FP64: cuFFT Z2D fields, one FP64 mesh sum per bin pair and 3j term",
            "ms_measure": inf["ms_measure"], "mesh_sum_kernel": "k_f64_dot3", "mesh_sum_gbs": gbs}


def metric_name(w):
    los = "local LOS" if w["kind"] == "survey" else "global LOS"
    if w.get("estimator") == "threept":
        mult = "+".join("zeta%d%d%d" % tuple(e) for e in w["ells"]) + (" + window Q" if w["window"] else "")
        return f"zeta_l1l2L(r1,r2) bins/s at {w['N']}^3 ({los}, {mult})"
    mult = "+".join("B%d%d%d" % tuple(e) for e in w["ells"]) + (" + window" if w["window"] else "")
    return f"B_l1l2L(k1,k2) bins/s at {w['N']}^3 ({los}, {mult})"


def config_of(name, w, world):
    nb = len(w["edges"]) - 1
    return {"workload": name, "nmesh": w["N"], "box_len": w["L"], "nbins": nb,
            "ells": w["ells"], "n_gal": w.get("n_gal", w.get("n_p")), "n_ran": w.get("n_ran", 0),
            "bins_per_step": n_bins_output(w), "los": "local" if w["kind"] == "survey" else "global",
            "mas": w["mas"], "interlace": w["interlace"], "window": w["window"],
            "l2": "inputs larger than L2 (meshes and fields of 0.5 GB each)" if w["N"] >= 256
            else "working set of a few hundred MB (no flush)",
            "parallelism": f"replicas x{world}"}


def sampled_parity(w, seed, res):
    """Errors of one measurement `res` against the stored FP64 oracle values at the sampled bin
    pairs of tests/golden/survey512_sampled_pairs.json (written by the oracle alone, read here as
    data), when the workload and its seed are the ones stored: per output the max error relative
    to the value and relative to its multipole's largest |value|, and whether every value is within
    the bound of the 512^3 parity test.  None for any other workload."""
    path = os.path.join(ROOT, "tests", "golden", "survey512_sampled_pairs.json")
    try:
        gold = json.load(open(path))
    except (OSError, ValueError):
        return None
    gw = gold["workload"]
    same = (gw.get("seed") == seed and gw["N"] == w["N"] and gw["L"] == w["L"] and gw["n_gal"] == w.get("n_gal")
            and gw["n_ran"] == w.get("n_ran") and gw["P0"] == w["P0"] and np.allclose(gw["edges"], w["edges"])
            and [tuple(e) for e in gw["ells"]] == [tuple(e) for e in w["ells"]])
    if not same:
        return None
    rel, rel_scale, ok = {}, {}, True
    for key in ("B", "shot", "window", "window_shot"):
        r = s = 0.0
        for rec in gold["values"]:
            im = [tuple(e) for e in w["ells"]].index(tuple(rec["ells"]))
            ref, got = rec[key], float(res[key][im, rec["b1"], rec["b2"]])
            scale = float(np.abs(res[key][im]).max())
            r = max(r, abs(got - ref) / abs(ref) if ref else 0.0)
            s = max(s, abs(got - ref) / scale if scale else 0.0)
            ok = ok and abs(got - ref) <= max(1e-4 * abs(ref), 1e-6 * scale)
        rel[key], rel_scale[key] = r, s
    return {"pairs": len(gold["values"]), "max_rel_err": rel, "max_err_over_multipole_max": rel_scale,
            "pass": ok, "bound": "1e-4 of the value or 1e-6 of its multipole's largest |value|",
            "against": "FP64 oracle at sampled bin pairs (tests/golden/survey512_sampled_pairs.json)"}


def pair_traffic(alg_bytes_per_launch):
    """DRAM bytes per k_pair_tma launch: the measured DRAM/algorithmic ratio of a small-case
    ncu capture of the same kernel, times this launch's algorithmic bytes (traffic grows with
    the number of mesh cells).  None when the kernel source changed since the capture."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "k_pair_tma_traffic.json")))
        src = open(os.path.join(ROOT, "paper_1803_02132_gb300", "csrc", "pair.cu"), "rb").read()
        if hashlib.sha256(src).hexdigest() != rec["source_sha256"]:
            return None
        return rec["dram_bytes_per_algorithmic_byte"] * alg_bytes_per_launch
    except Exception:
        return None


def _oracle_sample(w, N, nb, seed=7):
    """The workload's recipe on an N^3 mesh in the same box (particles in proportion to the
    cells) with its first nb bins (k-bins of the workload's width from its first edge; r-bins of
    at least one cell of that mesh for the three-point function)."""
    from oracle import estimator as E

    import synthcat

    L = w["L"]
    three = w.get("estimator") == "threept"
    if three:
        width = w["edges"][1] - w["edges"][0]
        e0 = max(w["edges"][0], 0.9 * L / N)
        edges = [e0 + i * width for i in range(nb + 1)]
    else:
        edges = list(w["edges"][:nb + 1])
    frac = (N / w["N"]) ** 3
    mas = {"NGP": 1, "CIC": 2, "TSC": 3}[w["mas"]]
    if w["kind"] == "survey":
        gal, ran = synthcat.survey_catalogs(N, L, w["observer"], int(w["n_gal"] * frac), int(w["n_ran"] * frac), seed)
        p = E.Params(N=N, L=L, edges=edges, ells=w["ells"], los="local", observer=w["observer"], mas=mas,
                     interlace=w["interlace"], P0=w["P0"], window=w["window"])
    else:
        gal, ran = {"xyz": synthcat.periodic_catalog(N, L, int(w["n_p"] * frac), seed)}, None
        p = E.Params(N=N, L=L, edges=edges, ells=w["ells"], los="global", mas=mas, interlace=w["interlace"])
    return p, gal, ran


def _npairs(w, nb):
    return sum(nb * (nb + 1) // 2 if l1 == l2 else nb * nb for (l1, l2, _) in w["ells"])


def _time_oracle(w, N, nb):
    from oracle import estimator as E
    from oracle import threept as T

    p, gal, ran = _oracle_sample(w, N, nb)
    t0, c0 = time.perf_counter(), time.process_time()
    (T.measure if w.get("estimator") == "threept" else E.measure)(p, gal, ran)
    return time.perf_counter() - t0, time.process_time() - c0


def _pool_worker(job):
    import os as _os
    import sys as _sys
    _sys.path.insert(0, ROOT)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        _os.environ[v] = "1"
    from oracle import estimator as E
    from oracle import threept as T

    w, N, nb, pairs = job
    p, gal, ran = _oracle_sample(w, N, nb)
    (T.measure if w.get("estimator") == "threept" else E.measure)(p, gal, ran, pairs=pairs)
    return len(pairs)


def cpu_baseline(args, w):
    """The FP64 oracle as it stands, timed on the host cores on bounded samples of the workload,
    with its cost scaled to the workload by a model fitted to those samples.

    Samples: the workload's recipe on 32^3 and 64^3 meshes in the same box (particles in
    proportion to the cells) with its first 2, 3 and 4 bins.  Model: t(N, nb) = (N/64)^a
    (A + C nb + D np(nb)), np the bin pairs of the multipoles (fields cost ~ nb, mesh sums ~ np);
    a from the 2-bin runs at 32^3 and 64^3, A, C, D >= 0 from the three 64^3 runs (non-negative least
    squares).  One thread (numpy); the same 4-bin sample is also timed on the host cores with its
    k1 rows split over processes (each process computes its own spectra, as the oracle does per
    call), and that speed-up is reported beside it."""
    runs = {}
    cpu = 0.0
    for N, nb in ((32, 2), (64, 2), (64, 3), (64, 4)):
        dt, c = _time_oracle(w, N, nb)
        runs[(N, nb)] = dt
        cpu += c
    wall = sum(runs.values())
    a = float(np.log2(runs[(64, 2)] / runs[(32, 2)]))
    M = np.array([[1.0, nb, _npairs(w, nb)] for nb in (2, 3, 4)])
    try:  # non-negative costs (timing noise must not make a cost component negative)
        from scipy.optimize import nnls

        (A, Cc, D), _ = nnls(M, np.array([runs[(64, nb)] for nb in (2, 3, 4)]))
    except ImportError:
        A, Cc, D = np.maximum(np.linalg.lstsq(M, np.array([runs[(64, nb)] for nb in (2, 3, 4)]), rcond=None)[0], 0.0)
    nbw = len(w["edges"]) - 1
    t_model = (w["N"] / 64) ** a * (A + Cc * nbw + D * _npairs(w, nbw))
    value = n_bins_output(w) / t_model
    # all host cores on the 64^3, 4-bin sample: k1 rows over a spawn pool
    ncores = os.cpu_count() or 1
    par = None
    if ncores > 1:
        import multiprocessing as mp

        nb = 4
        rows = [[(b1, b2) for b2 in range(nb)] for b1 in range(nb)]
        try:
            ctx = mp.get_context("spawn")
            t0 = time.perf_counter()
            with ctx.Pool(min(ncores, len(rows))) as pool:
                pool.map(_pool_worker, [(w, 64, nb, r) for r in rows])
            tp = time.perf_counter() - t0
            par = {"cores": min(ncores, len(rows)), "seconds": tp, "speedup": runs[(64, 4)] / tp,
                   "value": value * runs[(64, 4)] / tp}
        except Exception as e:  # the one-thread figure stands
            par = {"error": str(e)[:200]}
    cores = max(1, int(round(cpu / wall)))
    model = platform_cpu()
    samp = ", ".join(f"{N}^3/{nb} bins {t:.2f} s" for (N, nb), t in runs.items())
    return {"value": value, "unit": "bins/s", "cores": cores, "kind": "oracle",
            "sample": f"oracle on the workload's recipe at 32^3 and 64^3 in the same box (particles in proportion "
                      f"to the cells), first bins: {samp}; fitted t = (N/64)^{a:.2f} (A + C nb + D np) with "
                      f"A = {A:.3g} s, C = {Cc:.3g} s, D = {D:.3g} s; modelled {w['N']}^3/{nbw}-bin step "
                      f"{t_model:.4g} s",
            "model_seconds_per_step": t_model, "measured_seconds": {f"{N}^3/{nb}": t for (N, nb), t in runs.items()},
            "scaling_exponent": a, "cpu_model": model, "host_cores": ncores, "all_cores": par}


def platform_cpu():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if "Model name" in line:
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform

    return platform.processor() or platform.machine()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="survey512", choices=list(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end (host buffers) leg")
    ap.add_argument("--no-fp64-baseline", action="store_true",
                    help="skip the one-step timing of the plain FP64 form beside the FP32 line")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"],
                    help="fp64: the plain FP64 form of the estimator (comparison line)")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    if args.impl == "reference" and w["kind"] == "batch":
        # the oracle's sample: one realisation of the larger mesh
        w = dict(kind="box", N=max(w["sizes"]), L=w["L"], n_gen=max(w["sizes"]) // 2,
                 n_p=sum(w["n_p_range"]) // 2, edges=w["edges"], ells=w["ells"], mas=w["mas"],
                 interlace=w["interlace"], P0=0.0, window=False)
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        if rank != 0:
            return
        t0 = time.perf_counter()
        # the cost model is fitted once (cpu_baseline); every step then times the 64^3, 2-bin
        # sample and converts it to the workload with that model (about 5 s per step)
        cb = cpu_baseline(args, w)
        scale = cb["model_seconds_per_step"] / cb["measured_seconds"]["64^3/2"]
        vals = []
        for i in range(args.warmup + args.steps):
            dt, _ = _time_oracle(w, 64, 2)
            if i >= args.warmup:
                vals.append(n_bins_output(w) / (dt * scale))
        v = float(np.mean(vals))
        cb = dict(cb)
        cb["value"] = v
        cb["sample"] = (f"per step the oracle on the 64^3, 2-bin sample, converted with the fitted model "
                        f"(x {scale:.4g}); " + cb["sample"])
        print(json.dumps({"impl": "reference", "metric": metric_name(w),
                          "value": v, "unit": "bins/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "config": config_of(args.workload, w, world), "cpu_baseline": cb,
                          "e2e": {"value": v, "unit": "bins/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                          "seconds": time.perf_counter() - t0}))
        return
    if w["kind"] == "batch":
        if rank == 0:
            print(json.dumps(run_batch(args, w)))
        return
    out = run_gpu(args, w, rank, world)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(args, w)
        print(json.dumps(out))


if __name__ == "__main__":
    main()
