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
    for _ in range(args.steps):
        step()
        inf = plan.info()
        ms_pair.append(inf["ms_pair"])
        pair_launches += inf["pair_launches"]
        pair_bytes += inf["pair_bytes"]
        launches += inf["kernel_launches"]
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    # end to end through the public API with host buffers (H2D and D2H inside); the plain
    # FP64 comparison line leaves it out (its device time already runs to tens of seconds)
    ms_e2e = 0.0
    if not f64 and not args.no_e2e:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step(dev_inputs=False)
        torch.cuda.synchronize()
        ms_e2e = (time.perf_counter() - t0) * 1e3
    ms, ms_e2e = replicas.max_over_ranks([ms, ms_e2e], dist, device="cuda")
    info = plan.info()
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
        "stages_ms": {"assign_data": info["ms_assign_data"], "assign_randoms": info["ms_assign_randoms"],
                      "measure": info["ms_measure"], "pair": info["ms_pair"]},
        "clocks": clk,
    }
    if fp64:
        out["fp64_gpu_baseline"] = fp64
    return out


def run_batch(args, w):
    """A campaign of independent realisations (mixed mesh sizes) through two plans, one per
    size, each realisation assigned and measured in turn; device-resident inputs."""
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
    stream = torch.cuda.Stream()
    plans = {N: bisp.Plan(N, w["L"], w["edges"], w["ells"], los="global", mas=w["mas"], interlace=w["interlace"],
                          stream=stream) for N in w["sizes"]}

    def step():
        st = {"launches": 0, "pair_ms": 0.0, "pair_bytes": 0.0, "pair_launches": 0}
        for N, xyz in cats:
            plans[N].assign(bisp.DATA, xyz)
            plans[N].measure()
            inf = plans[N].info()
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
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    tot = {"launches": 0, "pair_ms": 0.0, "pair_bytes": 0.0, "pair_launches": 0}
    for _ in range(args.steps):
        st = step()
        for k in tot:
            tot[k] += st[k]
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    for pl in plans.values():
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
                   "bins_per_step": nbins, "schedule": "two plans, realisations measured one after another",
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


def cpu_baseline(args, w):
    """The FP64 oracle on a bounded sample of the workload, timed on the host cores."""
    from oracle import estimator as E
    from oracle import threept as T

    import synthcat

    # sample: the same recipe scaled down to a 64^3 mesh in the same box (1/512 of the cells,
    # particles in proportion), on the bins below that mesh's Nyquist frequency
    N = 64
    L = w["L"]
    kN = np.pi * N / L
    three = w.get("estimator") == "threept"
    if three:  # r-bins of at least one cell of the sample's mesh
        edges = [e for e in w["edges"] if e >= 0.9 * L / N]
        if len(edges) < 3:
            edges = list(np.linspace(L / N, 5 * L / N, 4))
    else:
        edges = [e for e in w["edges"] if e < 0.9 * kN]
        if len(edges) < 3:
            edges = list(np.linspace(w["edges"][0], 0.9 * kN, 4))
    frac = (N / w["N"]) ** 3
    if w["kind"] == "survey":
        gal, ran = synthcat.survey_catalogs(N, L, w["observer"], int(w["n_gal"] * frac), int(w["n_ran"] * frac), 7)
        p = E.Params(N=N, L=L, edges=edges, ells=w["ells"], los="local", observer=w["observer"],
                     mas={"NGP": 1, "CIC": 2, "TSC": 3}[w["mas"]], interlace=w["interlace"], P0=w["P0"],
                     window=w["window"])
    else:
        gal, ran = {"xyz": synthcat.periodic_catalog(N, L, int(w["n_p"] * frac), 7)}, None
        p = E.Params(N=N, L=L, edges=edges, ells=w["ells"], los="global",
                     mas={"NGP": 1, "CIC": 2, "TSC": 3}[w["mas"]], interlace=w["interlace"])
    # repeat the sample until about 10 s of CPU work (at most 6 repetitions)
    t0 = time.perf_counter()
    c0 = time.process_time()
    reps = 0
    while reps < 6 and (reps == 0 or time.perf_counter() - t0 < 10.0):
        (T.measure if three else E.measure)(p, gal, ran)
        reps += 1
    dt = (time.perf_counter() - t0) / reps
    cpu = (time.process_time() - c0) / reps
    nb = len(edges) - 1
    nbins = sum(nb * (nb + 1) // 2 if l1 == l2 else nb * nb for (l1, l2, _) in w["ells"]) * (2 if w["window"] else 1)
    # threads actually used: process CPU time over wall time (numpy's FFT and bincount run on
    # one thread; BLAS calls may use more)
    cores = max(1, int(round(cpu / dt)))
    # in the metric's unit: the oracle's cost per output bin grows with the number of mesh
    # cells, so the sample's rate is scaled by the cell ratio to the workload's mesh
    return {"value": nbins / dt * frac, "unit": "bins/s", "cores": cores, "kind": "oracle",
            "sample": f"oracle on the same recipe at {N}^3 (1/{int(round(1 / frac))} of the cells and particles), "
                      f"{nb} bins {'of at least one cell' if three else 'below that mesh' + chr(39) + 's Nyquist'}, "
                      f"{nbins} bins in {dt:.1f} s (mean of {reps} runs) "
                      f"({nbins / dt:.3g} bins/s at {N}^3); value = that rate x {N}^3/{w['N']}^3",
            "sample_bins_per_s": nbins / dt, "seconds": dt, "cpu_seconds": cpu}


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
        vals = []
        for i in range(args.warmup + args.steps):
            cb = cpu_baseline(args, w)
            if i >= args.warmup:
                vals.append(cb)
        v = float(np.mean([c["value"] for c in vals]))
        cb = dict(vals[-1])
        cb["value"] = v
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
