#!/usr/bin/env python3
"""Benchmark of the multilayer Gaussian-graph fast summation + Lanczos hot path.

One step = one pass of the whole hot path over the workload: plan every
layer (domain scaling, parameter choice, sort, Fourier tables, degrees) and
compute the k smallest eigenpairs of the power mean Laplacian with the
Lanczos method, every operator application going through the NFFT-based
fast summation.  The headline value is the fast-summation throughput of that
step in points x vectors per second (n x layer-vector applications / step
time), the metric's unit; the step time itself is the k-eigenpair Lanczos
time (plan included), reported as lanczos_s.

Default workload: the large single image, n = 10,000,000 pixels, 2 layers of
d = 3 (RGB; x, y, texture), sigma = 0.15, k = 10 eigenpairs of L_1 (p = 1):
the FP32 form at 1e-4 relative error is the headline, the FP64 form at 1e-6
is timed on the same workload (`forms`).  Beside it: the apply-level rate of
each form (median of 50 normalised products after 5 warm-ups, `apply`), the
oracle on the host cores (`cpu_baseline`), the sampled error of each form
against the oracle, peaks measured in the run by the library's micro-kernels
(`peaks_measured`), and short runs of the image (n = 1e6, T = 3, FP64 form,
p = -1, k = 20) and mixture (n = 250k, 52 layers, FP32, per-layer k = 10,
block 8) workloads (`other_workloads`).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
                  [--workload NAME] [--prec f32|f64] [--p 1|-1] [--k K]
                  [--mode eig|apply|ac] [--no-extra] [--no-baseline]

With N > 1 (torchrun) every rank runs an independent replica of the
workload on its own GPU (the path has no exchange step); the value is the
sum over ranks and the time the maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# ------------------------------------------------------------- workloads
WORKLOADS = {
    "image_voronoi_n1e6_T3": dict(desc="1000x1000 image, 8 Voronoi colour regions + N(0,0.02) noise; layers RGB, "
                                       "(x,y,texture), 3x3 box-filtered RGB", n=1_000_000, T=3, d=3, sigma=0.2,
                                  prec="f64", target=1e-6, k=20, p=-1.0),
    "gmm_n250k_T52_d2": dict(desc="250k samples of a 12-component GMM in R^104, 52 layers of 2 features; k "
                                  "eigenpairs of each layer's L_sym, all layers batched, blocks of 8 vectors",
                             n=250_000, T=52, d=2, sigma="half_range", prec="f32", target=1e-4, k=10, p=1.0,
                             per_layer=True, block=8),
    "image_discs_n1e7_T2": dict(desc="4000x2500 image, 5 uniform-colour discs + noise; layers RGB, (x,y,texture)",
                                n=10_000_000, T=2, d=3, sigma=0.15, prec="f32", target=1e-4, k=10, p=1.0),
    "single_n2000_d3": dict(desc="n=2000 uniform in [-1/4,1/4]^3", n=2000, T=1, d=3, sigma=0.1, prec="f64",
                            target=1e-12, k=10, p=1.0),
    "laplace_disc_n1e6_d2": dict(desc="n=1e6 uniform in the unit disc, Laplacian kernel exp(-r/sigma) (Sec. 4) "
                                      "with its near-field correction", n=1_000_000, T=1, d=2, sigma=0.05,
                                 prec="f32", target=1e-4, k=10, p=1.0, kernel="laplace"),
}


def make_layers(name):
    from paper_2007_05239_gb300 import workloads as wl
    spec = WORKLOADS[name]
    if name == "image_voronoi_n1e6_T3":
        layers = wl.image_voronoi_layers(1000, 1000, 8, 0.02, seed=2)
    elif name == "gmm_n250k_T52_d2":
        layers, _ = wl.gmm_band_layers(250_000, 104, 12, seed=3)
    elif name == "image_discs_n1e7_T2":
        layers = wl.image_discs_layers(2500, 4000, 5, 0.02, seed=4)
    elif name == "laplace_disc_n1e6_d2":
        layers = [wl.uniform_ball(1_000_000, 2, seed=9)]
    else:
        layers = [wl.uniform_cube(2000, 3, seed=1)]
    if spec["sigma"] == "half_range":
        sig = [0.5 * float((L.max(0) - L.min(0)).max()) for L in layers]
    else:
        sig = [float(spec["sigma"])] * len(layers)
    return layers, sig


# ------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------- peaks
def measured_peaks_file():
    """The measured copy bandwidth and bf16 GEMM peaks of this machine."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def measure_peaks(ml):
    """ALU denominators measured in this run by the library's micro-kernels
    (FP32 and FP64 FMA chains, conflict-free shared-memory atomics), plus the
    HBM copy bandwidth from MEASURED_PEAKS.json."""
    f = measured_peaks_file()
    out = {"fp32_tflops": ml.ml_measure_peak("fp32"), "fp64_tflops": ml.ml_measure_peak("fp64"),
           "smem_atomic_per_s_1e12": ml.ml_measure_peak("smem_atomic"),
           "alu_source": "ml_measure_peak micro-kernels in this run (8 CTAs x 256 threads per SM, best of 3)"}
    if "hbm_gbs" in f:
        out["hbm_gbs"] = float(f["hbm_gbs"])
        out["hbm_source"] = "MEASURED_PEAKS.json hbm_gbs (copy bandwidth, measured)"
    else:
        out["hbm_gbs"] = 6800.0
        out["hbm_source"] = "fallback 6.8 TB/s (MEASURED_PEAKS.json absent)"
    return out


# the arithmetic each form computes in: the FP64 form keeps every window,
# grid and tap value as an unevaluated pair of floats on the FP32 pipes
DTYPE_LABEL = {"f32": "f32", "f64": "f32x2 double-word (FP64-class taps, ~48-bit)"}


# ------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    """The oracle (direct FP64 sums) timed on the host cores, as it stands."""
    if rank != 0:
        return 0
    from oracle import graph
    spec = WORKLOADS[args.workload]
    layers, sig = make_layers(args.workload)
    n, T = layers[0].shape[0], len(layers)
    rng = np.random.default_rng(0)
    v = rng.uniform(0, 1, n)

    kernel = spec.get("kernel", "gauss")

    def step(rows):
        for t in range(T):
            graph.W_apply(layers[t], sig[t], v, rows=rows, kernel=kernel)

    # size the per-step row sample to ~4 s
    r0 = np.sort(rng.choice(n, size=min(n, 16), replace=False))
    t0 = time.perf_counter()
    step(r0)
    dt = max(time.perf_counter() - t0, 1e-6)
    R = int(min(n, max(16, 16 * 4.0 / dt)))
    rows = np.sort(rng.choice(n, size=R, replace=False))
    for _ in range(args.warmup):
        step(rows)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step(rows)
    el = time.perf_counter() - t0
    val = R * T * args.steps / el / 1e9
    cores = graph.num_threads()
    line = {
        "impl": "reference", "metric": metric_name(spec), "value": val, "unit": "Gpts·vec/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(args, spec, n, T),
        "cpu_baseline": {"value": val, "unit": "Gpts·vec/s", "cores": cores, "kind": "oracle",
                         "sample": f"direct FP64 sum (W v) on {R} sampled rows of each of the {T} layers per step"},
        "e2e": {"value": val, "unit": "Gpts·vec/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def metric_name(spec):
    tol = f"{spec['target']:.0e}"
    if spec.get("per_layer"):
        return (f"fast-summation Gpts·vec/s ({spec['prec'].upper()} form, <= {tol} rel err vs FP64) inside the "
                f"per-layer k={spec['k']} block-{spec['block']} Lanczos step")
    return (f"fast-summation Gpts·vec/s ({spec['prec'].upper()} form, <= {tol} rel err vs FP64) inside the "
            f"k={spec['k']} Lanczos step (p={int(spec['p'])})")


def config_dict(args, spec, n, T):
    return {"workload": args.workload, "desc": spec["desc"], "n": n, "layers": T, "d": spec["d"],
            "sigma": spec["sigma"], "prec": spec["prec"], "target_rel_err": spec["target"], "k": spec["k"],
            "p": spec["p"], "kernel": spec.get("kernel", "gauss"), "planner": getattr(args, "planner", "rule"),
            "l2": "inputs exceed L2 (per-layer point data and the Krylov basis are > 129 MB)",
            "parallelism": f"replicas{args.gpus}"}


# ------------------------------------------------------------- ranks
def reduce_over_ranks(ms, work, device="cpu"):
    """(max time over ranks, total work over ranks); the identity on one rank."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(ms), float(work)
    t = torch.tensor([float(ms), float(work)], dtype=torch.float64, device=device)
    parts = [torch.zeros_like(t) for _ in range(dist.get_world_size())]
    dist.all_gather(parts, t)
    return max(float(p[0]) for p in parts), sum(float(p[1]) for p in parts)


# ------------------------------------------------------------- our arm
def build_planners(ml, prec, target, kernel, planner_kind):
    planner = make_planner(planner_kind, prec, target, ml, kernel)
    plan_all = make_planner("many", prec, target, ml, kernel) if planner_kind == "rule" else None
    return planner, plan_all


def eig_step_fn(ml, spec, sig, planner, plan_all, n):
    """One pass of the hot path: plan every layer, then the k eigenpairs.
    Returns (eigenvalues, converged pairs, point-vectors applied, plan infos)."""
    k, p = spec["k"], spec["p"]

    def step(dl, evecs):
        t0 = time.perf_counter()
        plans = plan_all(dl, sig) if plan_all else [planner(x, s) for x, s in zip(dl, sig)]
        step.plan_s.append(time.perf_counter() - t0)   # the plan calls synchronise their streams
        if spec.get("per_layer"):
            lam, nconv, st = ml.ml_lanczos_eigs_layers(plans, k, block=spec["block"], tol=1e-8, seed=1, evecs=evecs)
            lam, nconv = lam[0], int(nconv.min())
        else:
            lam, nconv, st = ml.ml_lanczos_eigs(plans, k, p=p, tol=1e-8, seed=1, evecs=evecs)
        applied = sum(pl.info["applied_vectors"] for pl in plans) * n
        infos = [pl.info for pl in plans]
        for pl in plans:
            pl.destroy()
        return lam, nconv, applied, infos
    step.plan_s = []
    return step


def time_steps(step, dev_layers, evecs, steps, warmup, barrier, torch, sample_clocks=None):
    """warm-up, then `steps` steps between CUDA events on the current stream
    (barrier + synchronize on both sides).  Returns (ms, applied, last result)."""
    for _ in range(warmup):
        step(dev_layers, evecs)
    torch.cuda.synchronize()
    barrier()
    if sample_clocks:
        sample_clocks.start()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    e0.record(stream)
    applied, res = 0, None
    for _ in range(steps):
        res = step(dev_layers, evecs)
        applied += res[2]
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = sample_clocks.stop() if sample_clocks else None
    return e0.elapsed_time(e1), applied, res, clk


def profiled_step(step, dev_layers, evecs, ml, torch):
    """One more step with CUDA events around every library launch on its
    stream (per-kernel events cannot sit inside a graph: eager launches)."""
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ml.ml_profile_reset()
    ml.ml_profile_enable(True)
    torch.cuda.synchronize()
    e0.record(stream)
    res = step(dev_layers, evecs)
    e1.record(stream)
    torch.cuda.synchronize()
    ml.ml_profile_enable(False)
    return res, ml.ml_profile_read(), e0.elapsed_time(e1)


def apply_median(ml, torch, plans, n, b=1, reps=50, warmup=5):
    """The apply-level metric: one multilayer normalised product of b vectors,
    each call between CUDA events on the current stream, median of `reps`
    calls after `warmup` untimed ones; n x T x b / t in Gpts·vec/s."""
    X = torch.as_tensor(np.random.default_rng(7).uniform(0, 1, (n, b)), device="cuda")
    Y = torch.empty_like(X)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        ml.ml_fastsum_apply(plans, X, Y, mode="normalized")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    torch.cuda.synchronize()
    for a, z in ev:
        a.record(stream)
        ml.ml_fastsum_apply(plans, X, Y, mode="normalized")
        z.record(stream)
    torch.cuda.synchronize()
    ms = statistics.median(a.elapsed_time(z) for a, z in ev)
    return {"value": n * len(plans) * b / (ms / 1e3) / 1e9, "unit": "Gpts·vec/s", "ms_median": ms, "calls": reps,
            "warmup_calls": warmup, "b": b, "mode": "normalized"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--prec", default=None, choices=["f32", "f64"])
    ap.add_argument("--p", type=float, default=None)
    ap.add_argument("--k", type=int, default=None)
    ap.add_argument("--no-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the second precision form and the other workloads' short runs")
    ap.add_argument("--mode", default="eig", choices=["eig", "apply", "ac"],
                    help="eig: plan + k eigenpairs per step (default); apply: one multilayer normalised "
                         "product of b vectors per step on plans made before the timed region; ac: the "
                         "Allen-Cahn classifier (Alg. 2) on eigenpairs computed before the timed region")
    ap.add_argument("--b", type=int, default=1, help="vectors per product in --mode apply")
    ap.add_argument("--target", type=float, default=None, help="relative error target (default per precision)")
    ap.add_argument("--combined", action="store_true",
                    help="per-layer workloads: eigenpairs of the combined power mean operator instead")
    ap.add_argument("--planner", default="rule", choices=["rule", "learned"],
                    help="NFFT parameters of each layer: the automatic rule, or the learned model "
                         "(paper_2007_05239_gb300/paramnet_<prec>_<target>.npz)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    spec = dict(WORKLOADS[args.workload])
    forced_prec = args.prec is not None
    if args.prec:
        spec["prec"] = args.prec
        spec["target"] = 1e-6 if args.prec == "f64" else 1e-4
    if args.p is not None:
        spec["p"] = args.p
    if args.k is not None:
        spec["k"] = args.k
    if args.target is not None:
        spec["target"] = args.target
    if args.combined:
        spec["per_layer"] = False
    WORKLOADS[args.workload] = spec
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    from paper_2007_05239_gb300 import _lib as ml

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    if args.mode == "ac":
        return run_ac(args, spec, rank, world, barrier)

    peaks = measure_peaks(ml)
    layers, sig = make_layers(args.workload)
    n, T = layers[0].shape[0], len(layers)
    dev_layers = [torch.as_tensor(L, device="cuda") for L in layers]
    k, p, prec, target = spec["k"], spec["p"], spec["prec"], spec["target"]

    kernel = spec.get("kernel", "gauss")
    if kernel != "gauss" and args.planner != "rule":
        raise SystemExit("the learned planner covers the Gaussian kernel only")
    planner, plan_all = build_planners(ml, prec, target, kernel, args.planner)
    per_layer = bool(spec.get("per_layer"))
    nev = n * k * (T if per_layer else 1)

    if args.mode == "apply":
        apply_plans = [planner(x, s) for x, s in zip(dev_layers, sig)]
        Xa = torch.as_tensor(np.random.default_rng(7).uniform(0, 1, (n, args.b)), device="cuda")
        Ya = torch.empty_like(Xa)

        def step(dl, evecs):
            before = sum(pl.info["applied_vectors"] for pl in apply_plans)
            ml.ml_fastsum_apply(apply_plans, Xa, Ya, mode="normalized")
            applied = (sum(pl.info["applied_vectors"] for pl in apply_plans) - before) * n
            return None, 0, applied, [pl.info for pl in apply_plans]
        evecs = None
    else:
        step = eig_step_fn(ml, spec, sig, planner, plan_all, n)
        evecs = torch.empty(nev, dtype=torch.float64, device="cuda")

    # ---- timed region (device-resident inputs; kernel timing off, so the inner
    #      conjugate-gradient iterations replay their CUDA graphs)
    clocks = ClockSampler(local)
    ms_total, applied, res, clk = time_steps(step, dev_layers, evecs, args.steps, args.warmup, barrier, torch, clocks)
    lam, nconv = res[0], res[1]
    t_max, tot_applied = reduce_over_ranks(ms_total, applied, "cuda")
    value = tot_applied / (t_max / 1e3) / 1e9

    # ---- kernel timing and the roofline of the dominant kernel family
    (_, _, applied_prof, msz), prof, prof_step_ms = profiled_step(step, dev_layers, evecs, ml, torch)
    launches = int(sum(v[0] for v in prof.values())) * args.steps   # a graph replay runs the same kernels
    nv = min(args.b, 8) if args.mode == "apply" else (spec.get("block", 1) if per_layer else 1)
    roofline = kernel_roofline(args.workload, spec, prof, msz, applied_prof, n, T, nv, prec, prof_step_ms, peaks)

    # ---- end to end through the C ABI with host buffers (pinned)
    e2e = run_e2e(args, ml, torch, step, layers, nev, n, barrier, apply_plans if args.mode == "apply" else None,
                  Xa if args.mode == "apply" else None)

    line = {
        "metric": metric_name(spec), "value": value, "unit": "Gpts·vec/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE_LABEL[prec], "data": "synthetic", "config": config_dict(args, spec, n, T),
        "mode": args.mode, "gpu_launches": launches, "e2e": e2e, "roofline": roofline, "clocks": clk,
        "peaks_measured": peaks,
        "plans": [{key: info[key] for key in ("N", "n_os", "taps", "L", "bin", "nbins", "nsub", "sigma_s")}
                  for info in msz],
    }
    if args.mode == "eig":
        line["lanczos_s"] = t_max / args.steps / 1e3
        line["plan_s_median"] = statistics.median(step.plan_s) if step.plan_s else None
        line["eigenvalues"] = [float(x) for x in lam[:min(5, k)]]
        line["nconv"] = int(nconv)
    else:
        line["metric"] = (f"fast-summation Gpts·vec/s ({prec.upper()} form) of one multilayer normalised product, "
                          f"b={args.b}")
        line["config"]["b"] = args.b

    single = rank == 0 and world == 1
    # ---- the second precision form on the same workload (the metric is quoted
    #      at 1e-4 for the FP32 form and 1e-6 for the FP64 form)
    other = None
    if args.mode == "eig" and not args.no_extra and not forced_prec and args.workload in TWO_FORMS:
        other = "f64" if prec == "f32" else "f32"
        ospec = dict(spec, prec=other, target=1e-6 if other == "f64" else 1e-4)
        oplanner, oplan_all = build_planners(ml, other, ospec["target"], kernel, "rule")
        ostep = eig_step_fn(ml, ospec, sig, oplanner, oplan_all, n)
        ow = min(args.warmup, 2)
        oms, oapp, ores, _ = time_steps(ostep, dev_layers, evecs, args.steps, ow, barrier, torch)
        ot, oa = reduce_over_ranks(oms, oapp, "cuda")
        line["forms"] = {prec: {"value": value, "ms_per_step": t_max / args.steps, "target_rel_err": target,
                                "dtype": DTYPE_LABEL[prec]},
                         other: {"value": oa / (ot / 1e3) / 1e9, "ms_per_step": ot / args.steps,
                                 "target_rel_err": ospec["target"], "dtype": DTYPE_LABEL[other],
                                 "warmup": ow, "steps": args.steps, "nconv": int(ores[1]),
                                 "eigenvalues": [float(x) for x in ores[0][:min(5, k)]]}}

    # ---- apply-level metric: median of 50 normalised products (each form)
    if args.mode == "eig" and not per_layer:
        line["apply"] = {}
        for form in [prec] + ([other] if other else []):
            ftarget = target if form == prec else (1e-6 if form == "f64" else 1e-4)
            fpl, _ = build_planners(ml, form, ftarget, kernel, "rule")
            plans = [fpl(x, s) for x, s in zip(dev_layers, sig)]
            line["apply"][form] = apply_median(ml, torch, plans, n)
            line["apply"][form]["target_rel_err"] = ftarget
            for pl in plans:
                pl.destroy()

    # ---- CPU baseline (oracle on the host cores) and sampled accuracy, rank 0 at N = 1
    if single and not args.no_baseline:
        forms = [(prec, target)] + ([(other, 1e-6 if other == "f64" else 1e-4)] if other else [])
        line["cpu_baseline"], errs = cpu_baseline(layers, sig, ml, torch, dev_layers, forms, kernel,
                                                  per_layer=per_layer, nv=nv)
        line["rel_err_sampled"] = errs[prec]
        if other:
            line["forms"][prec]["rel_err_sampled"] = errs[prec]
            line["forms"][other]["rel_err_sampled"] = errs[other]

    # ---- the other large workloads, short runs (their step rate and accuracy)
    if args.mode == "eig" and not args.no_extra and args.workload == DEFAULT_WORKLOAD:
        line["other_workloads"] = {}
        del dev_layers, evecs
        torch.cuda.empty_cache()
        for wname in EXTRA_WORKLOADS:
            line["other_workloads"][wname] = run_extra(wname, ml, torch, barrier, single and not args.no_baseline)
            torch.cuda.empty_cache()
        line["other_workloads"]["learned_params_200_clouds"] = run_params_extra()

    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_e2e(args, ml, torch, step, layers, nev, n, barrier, apply_plans, Xa):
    """The same metric end to end through the C ABI: host (pinned) inputs and
    outputs, every host<->device copy inside the timed region."""
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    host_layers = [torch.as_tensor(L).pin_memory() for L in layers]
    if args.mode == "apply":
        hx = Xa.cpu().pin_memory()
        hy = torch.empty_like(hx).pin_memory()
        h2d, d2h = hx.numel() * 8, hy.numel() * 8
    else:
        host_evecs = torch.empty(nev, dtype=torch.float64).pin_memory()
        h2d = sum(L.numel() * 8 for L in host_layers)
        d2h = nev * 8 + nev // n * 8
    torch.cuda.synchronize()
    barrier()
    e0.record(stream)
    applied = 0
    for _ in range(args.steps):
        if args.mode == "apply":
            before = sum(pl.info["applied_vectors"] for pl in apply_plans)
            ml.ml_fastsum_apply(apply_plans, hx, hy, mode="normalized")   # host buffers: staged by the library
            applied += (sum(pl.info["applied_vectors"] for pl in apply_plans) - before) * n
            continue
        # the plans take the pinned host layers through the C ABI and copy them
        # to the device themselves (the learned planner reads device points)
        dl = host_layers if args.planner == "rule" else [x.to("cuda", non_blocking=True) for x in host_layers]
        applied += step(dl, host_evecs)[2]
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    t, work = reduce_over_ranks(e0.elapsed_time(e1), applied, "cuda")
    return {"value": work / (t / 1e3) / 1e9, "unit": "Gpts·vec/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h}


def run_params_extra():
    """The learned NFFT-parameter workload: the MLP trained on 5000 (cloud,
    candidate) -> (error, time) samples the method generates (500 clouds, 10
    candidates each, 10 % of the clouds held out for the per-factor error
    margins at the 0.999 quantile), then the learned choice against the fixed rule on 200 unseen
    clouds at target 1e-4 (errors judged by the direct sum on sampled rows)."""
    from paper_2007_05239_gb300 import paramnet
    t0 = time.perf_counter()
    X, Y, ids = paramnet.make_dataset(0, 500, 10, "f32", 1e-4)
    t1 = time.perf_counter()
    fit = ids < 450
    model, losses, _ = paramnet.train(X[fit], Y[fit], epochs=4000)
    margins = paramnet.calibrate_margins(model, X[~fit], Y[~fit], 0.999)
    model.set_margins(margins)
    t2 = time.perf_counter()
    ev = paramnet.evaluate(model, 5000, 200, "f32", 1e-4, margin=max(margins))
    t3 = time.perf_counter()
    return {"samples": int(X.shape[0]), "fit_samples": int(fit.sum()), "margins": margins,
            "loss_first": float(losses[0]), "loss_last": float(losses[-1]),
            "success_learned": ev["success_learned"], "success_fixed": ev["success_fixed"],
            "time_ratio_geomean": ev["time_ratio_geomean"], "eval_clouds": 200, "target_rel_err": 1e-4,
            "data_s": t1 - t0, "train_s": t2 - t1, "eval_s": t3 - t2,
            "desc": "learned (N factor, window width, oversampling) vs the fixed rule; time ratio < 1 = faster"}


def run_extra(wname, ml, torch, barrier, with_err):
    """One warm-up and two timed steps of another workload (plan + its
    eigenproblem), with the sampled error of its product when asked."""
    spec = WORKLOADS[wname]
    layers, sig = make_layers(wname)
    n, T = layers[0].shape[0], len(layers)
    dev_layers = [torch.as_tensor(L, device="cuda") for L in layers]
    planner, plan_all = build_planners(ml, spec["prec"], spec["target"], spec.get("kernel", "gauss"), "rule")
    step = eig_step_fn(ml, spec, sig, planner, plan_all, n)
    per_layer = bool(spec.get("per_layer"))
    evecs = torch.empty(n * spec["k"] * (T if per_layer else 1), dtype=torch.float64, device="cuda")
    ms, applied, res, clk = time_steps(step, dev_layers, evecs, 2, 1, barrier, torch, ClockSampler(
        int(os.environ.get("LOCAL_RANK", "0"))))
    out = {"metric": metric_name(spec), "value": applied / (ms / 1e3) / 1e9, "unit": "Gpts·vec/s",
           "ms_per_step": ms / 2, "steps": 2, "warmup": 1, "dtype": DTYPE_LABEL[spec["prec"]],
           "target_rel_err": spec["target"], "k": spec["k"], "p": spec["p"], "nconv": int(res[1]),
           "eigenvalues": [float(x) for x in res[0][:5]], "clocks": clk, "desc": spec["desc"],
           "plan_s_median": statistics.median(step.plan_s) if step.plan_s else None}
    if with_err:
        nv = spec.get("block", 1) if per_layer else 1
        _, errs = cpu_baseline(layers, sig, ml, torch, dev_layers, [(spec["prec"], spec["target"])],
                               spec.get("kernel", "gauss"), seconds=3.0, per_layer=per_layer, nv=nv)
        out["rel_err_sampled"] = errs[spec["prec"]]
    return out


def run_ac(args, spec, rank, world, barrier):
    """Alg. 2 steps 2-4 (the multiclass Allen-Cahn scheme) on a workload with a
    ground truth: eigenpairs of the power mean Laplacian are computed before
    the timed region; each timed step runs the scheme to its tolerance with
    the paper's parameters for that kind of data (image: eps 0.005, omega0
    1000, dt 0.01, max_iter 500; hyperspectral: eps 0.5, omega0 1e4, dt 0.01,
    max_iter 300; c = omega0 + 3/eps, tol 1e-6) and 4 % known labels."""
    import torch
    from paper_2007_05239_gb300 import _lib as ml
    from paper_2007_05239_gb300 import workloads as wl
    if args.workload == "image_voronoi_n1e6_T3":
        layers, truth = wl.image_voronoi_layers(1000, 1000, 8, 0.02, seed=2, return_labels=True)
        m = 8
        sig = [float(spec["sigma"])] * len(layers)
        # the image experiments' parameters (Sec. 8)
        prm = dict(eps=0.005, omega0=1000.0, dt=0.01, tol=1e-6, max_iter=500)
    elif args.workload == "gmm_n250k_T52_d2":
        layers, truth = wl.gmm_band_layers(250_000, 104, 12, seed=3)
        m = 12
        sig = [0.5 * float((L.max(0) - L.min(0)).max()) for L in layers]
        # the hyperspectral experiment's parameters (Sec. 8)
        prm = dict(eps=0.5, omega0=10000.0, dt=0.01, tol=1e-6, max_iter=300)
    else:
        raise SystemExit("--mode ac runs on the workloads with a ground truth: image_voronoi_n1e6_T3, gmm_n250k_T52_d2")
    n, k = layers[0].shape[0], spec["k"]
    plans = ml.ml_fastsum_plan_many([torch.as_tensor(L, device="cuda") for L in layers], sig, prec=spec["prec"],
                                    target_rel_err=spec["target"])
    Phi = torch.empty(n * k, dtype=torch.float64, device="cuda")
    lam, nconv, _ = ml.ml_lanczos_eigs(plans, k, p=spec["p"], tol=1e-8, seed=1, evecs=Phi)
    for pl in plans:
        pl.destroy()
    labels_h = wl.known_labels(truth, 0.04, seed=5)
    labels = torch.as_tensor(labels_h, device="cuda")
    U = torch.empty(n * m, dtype=torch.float64, device="cuda")
    pred = torch.empty(n, dtype=torch.int32, device="cuda")
    for _ in range(args.warmup):
        ml.ml_allen_cahn(Phi, lam, labels, m, U=U, pred=pred, **prm)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    ml.ml_profile_reset()
    ml.ml_profile_enable(True)
    torch.cuda.synchronize()
    barrier()
    e0.record(stream)
    iters = 0
    for _ in range(args.steps):
        _, _, it, chg = ml.ml_allen_cahn(Phi, lam, labels, m, U=U, pred=pred, **prm)
        iters += it
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ml.ml_profile_enable(False)
    clk = clocks.stop()
    prof = ml.ml_profile_read()
    ms = e0.elapsed_time(e1)
    t_max, tot = reduce_over_ranks(ms, n * iters, "cuda")
    acc = float((pred.cpu().numpy() == truth).mean())
    # roofline: every pass does Phi_k V (2 k m flop per node) and Phi_k^T R (2 k m) in FP64
    # on ~(8k + 16m + 4) bytes per node: above the FP64 ridge, so the FP64 pipe binds
    passes = iters + args.steps
    bytes_pass = n * (k * 8 + 2 * m * 8 + 4)
    flops_pass = n * 4.0 * k * m
    fam_launches, fam_ms = prof.get("allen_cahn", (0, 0.0))
    achieved = flops_pass * passes / (fam_ms / 1e3) / 1e12 if fam_ms > 0 else 0.0
    gbs = bytes_pass * passes / (fam_ms / 1e3) / 1e9 if fam_ms > 0 else 0.0
    peak = ml.ml_measure_peak("fp64")
    # end to end: eigenvectors and labels from pinned host memory, scores and classes back
    hPhi = Phi.cpu().pin_memory()
    hlab = labels.cpu().pin_memory()
    hU = torch.empty(n * m, dtype=torch.float64).pin_memory()
    hpred = torch.empty(n, dtype=torch.int32).pin_memory()
    torch.cuda.synchronize()
    e0.record(stream)
    it_e2e = 0
    for _ in range(args.steps):
        dPhi = hPhi.to("cuda", non_blocking=True)
        dlab = hlab.to("cuda", non_blocking=True)
        _, _, it, _ = ml.ml_allen_cahn(dPhi, lam, dlab, m, U=U, pred=pred, **prm)
        hU.copy_(U, non_blocking=True)
        hpred.copy_(pred, non_blocking=True)
        it_e2e += it
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    line = {
        "metric": f"Allen-Cahn scheme (Alg. 2) node-iterations/s on k={k} eigenpairs (p={int(spec['p'])}), m={m}",
        "value": tot / (t_max / 1e3) / 1e9, "unit": "Gnode·it/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n": n, "classes": m, "k": k, "p": spec["p"], "known": 0.04,
                   "params": prm, "parallelism": f"replicas{world}",
                   "l2": f"inputs exceed L2 (eigenvectors {n * k * 8 / 1e6:.0f} MB per pass)" if n * k * 8 > 129e6 else "eigenvectors fit in L2"},
        "mode": "ac", "iterations_per_step": iters / args.steps, "accuracy": acc,
        "gpu_launches": int(sum(v[0] for v in prof.values())),
        "e2e": {"value": n * it_e2e / (e2e_ms / 1e3) / 1e9, "unit": "Gnode·it/s",
                "h2d_bytes_per_step": n * k * 8 + n * 4, "d2h_bytes_per_step": n * m * 8 + n * 4},
        "roofline": {"bound": "alu", "kernel": "allen_cahn", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "peak_source": "FP64 FMA pipe, measured in this run (ml_measure_peak)",
                     "work": f"{flops_pass:.3g} flop and {bytes_pass} B per pass (eigenvectors n*k*8, scores in/out "
                             f"2*n*m*8, labels n*4)", "hbm_gbs_achieved": gbs,
                     "family_ms": {f: v[1] for f, v in prof.items()}},
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def make_planner(kind, prec, target, ml, kernel="gauss"):
    """plan(points, sigma) with the automatic rule, or with the learned model
    trained for this precision and target (falls back to the rule where no
    candidate qualifies)."""
    if kind == "rule":
        if kernel != "gauss":
            return lambda x, s: ml.ml_fastsum_plan_ex(x, s, prec=prec, target_rel_err=target, kernel=kernel)
        return lambda x, s: ml.ml_fastsum_plan(x, s, prec=prec, target_rel_err=target)
    if kind == "many":   # all layers at once (concurrent set-up)
        return lambda xs, ss: ml.ml_fastsum_plan_many(xs, ss, prec=prec, target_rel_err=target, kernel=kernel)
    from paper_2007_05239_gb300 import paramnet
    path = os.path.join(ROOT, "paper_2007_05239_gb300", f"paramnet_{prec}_{target:.0e}.npz")
    if not os.path.exists(path):
        raise SystemExit(f"--planner learned needs {path}: python -m paper_2007_05239_gb300.paramnet "
                         f"--prec {prec} --target {target:.0e} --out {path}")
    model, margin = paramnet.load_model(path)
    return lambda x, s: ml.ml_fastsum_plan_learned(x, s, model, prec=prec, target_rel_err=target, margin=margin)[0]


# in-range share of the pairs the near-field pass examines, for a uniform
# cloud and cells of edge eps_I: ball(eps_I) / (3 eps_I)^d
NEAR_IN_RANGE = {1: 2.0 / 3.0, 2: math.pi / 9.0, 3: 4.0 * math.pi / 81.0}

DEFAULT_WORKLOAD = "image_discs_n1e7_T2"
TWO_FORMS = {"image_discs_n1e7_T2"}          # the metric is quoted for both forms here
EXTRA_WORKLOADS = ["image_voronoi_n1e6_T3", "gmm_n250k_T52_d2"]

# what a step's largest kernel family is, where it is not the product itself
FAMILY_NOTES = {
    "dots": "FP64-class products Q^T x of the Lanczos steps' Gram-Schmidt pass (double-word FP32 by default), "
            "bound by HBM",
    "update": "FP64-class basis updates x -= Q h of the Lanczos steps",
    "dots2": "second Gram-Schmidt pass, run only when the first removed more than half of the norm squared",
    "update2": "second Gram-Schmidt pass, run only when the first removed more than half of the norm squared",
    "ritz": "Ritz vectors Q S at each restart",
    "plan": "plan set-up of every layer (bounding box, sort, Fourier tables, degrees): chains of small kernels "
            "and host synchronisations; the timed steps build the layers' plans concurrently, so the summed event "
            "times of the profiled step overstate its share",
}

# ncu DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch,
# keyed by (workload, form, kernel family, window width, vectors per pass),
# with the hash of the kernel sources at the time of the capture: a changed
# source makes the figure stale and the line reports null
DW_OPS_PER_FMA = 10

NCU_TRAFFIC = {
    # k_spread_f32<3,5,1>, both layers of the 10-megapixel image (one launch
    # each, ncu --set full of the apply-mode run): 515.2 and 346.4 MB, mean
    # 430.8 MB per launch
    ("image_discs_n1e7_T2", "f32", "spread", 5, 1): (430.8e6, "a75fdb2bef51fef1",
                                                      "ncu dram__bytes_read.sum + dram__bytes_write.sum, mean of "
                                                      "the two layers' launches; the tiles are written only within "
                                                      "the box of cells each subproblem's taps reach (14 MB); the "
                                                      "rest is the point data and 32-byte sectors of the random "
                                                      "input gathers"),
}
KERNEL_SOURCES = ["paper_2007_05239_gb300/csrc/kernels.cuh", "paper_2007_05239_gb300/csrc/launch.cuh"]


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def kernel_roofline(workload, spec, prof, infos, applied, n, T, nv, prec, prof_step_ms, peaks):
    """Roofline of the product's dominant kernel family in the profiled step.
    Algorithmic work: one multiply-add (2 flop) per tap and point-vector,
    W^d taps; bytes per point and pass (window table 8 d W + packed taps 4 in
    the FP64 form, coordinates 4 d in the FP32 form; permutation 4, D^{-1/2}
    8) plus 8 B per vector read (spread) or read and written (interp)."""
    fam = max(("spread", "interp", "near"), key=lambda f: prof.get(f, (0, 0.0))[1])
    if fam == "near":
        return near_roofline(prof, infos, applied, n, T, spec["d"], nv, prec, prof_step_ms, peaks)
    d = spec["d"]
    W = infos[0]["taps"]
    taps = W ** d
    fam_launches, fam_ms = prof.get(fam, (0, 0.0))
    sec = fam_ms / 1e3
    flops = applied * 2.0 * taps
    achieved = flops / sec / 1e12 if sec > 0 else 0.0
    # the FP64 form's taps are double-word multiply-adds on the FP32 pipe: an
    # exact product by FMA (4 lane operations) and an exact two-sum (6), so its
    # ALU roof is the measured FP32 rate / 10 in FP64-class flops
    peak = peaks["fp32_tflops"] if prec == "f32" else peaks["fp32_tflops"] / DW_OPS_PER_FMA
    point_bytes = (8 * d * W + 4 if prec == "f64" else 4 * d) + 4 + 8
    vec_bytes = 8 if fam == "spread" else 16
    hbm_bytes = applied / nv * point_bytes + applied * vec_bytes
    hbm_gbs = hbm_bytes / sec / 1e9 if sec > 0 else 0.0
    per_launch = hbm_bytes / fam_launches if fam_launches else None
    key = (workload, prec, fam, W, nv)
    traffic, traffic_note = None, "no ncu capture of this kernel on this workload"
    if key in NCU_TRAFFIC:
        tb, src_hash, note = NCU_TRAFFIC[key]
        if src_hash == kernel_source_hash():
            traffic, traffic_note = tb, note
        else:
            traffic_note = "stale: the kernel sources changed since the capture"
    out = {"bound": "alu", "kernel": fam, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
           "frac": achieved / peak if peak else None, "traffic": traffic, "traffic_note": traffic_note,
           "algorithmic_bytes_per_launch": per_launch,
           "peak_source": "FP32 FMA pipe, measured in this run (ml_measure_peak fp32)"
                          + (f"; FP64 form: / {DW_OPS_PER_FMA} lane operations per double-word multiply-add"
                             if prec == "f64" else ""),
           "work": f"2 flop per tap, W^d = {taps} taps per point-vector, W = {W}, {nv} vector(s) per pass",
           "hbm": {"achieved": hbm_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                   "frac": hbm_gbs / peaks["hbm_gbs"], "bytes_per_point_pass": point_bytes,
                   "bytes_per_point_vector": vec_bytes, "peak_source": peaks["hbm_source"]},
           "family_ms": {f: v[1] for f, v in prof.items()}, "family_launches": {f: v[0] for f, v in prof.items()},
           "region": "one extra step after the timed region with per-kernel CUDA events (eager launches), "
                     f"{prof_step_ms:.1f} ms"}
    if fam == "spread":
        # shared-memory accumulation: one 32-bit atomic per tap and vector
        # (FP32 form) or two (the FP64 form's hi and lo words)
        per_tap = 1 if prec == "f32" else 2
        atom = applied * taps * per_tap / sec / 1e12 if sec > 0 else 0.0
        out["smem_atomics"] = {"achieved": atom, "peak": peaks["smem_atomic_per_s_1e12"], "unit": "1e12/s",
                               "frac": atom / peaks["smem_atomic_per_s_1e12"],
                               "per_tap_and_vector": per_tap,
                               "peak_source": "conflict-free 32-bit shared atomics, measured in this run",
                               "note": ("tap accumulations per second; warps whose points share their first tap "
                                        "(the row products) issue one atomic per 32 taps, so the atomics "
                                        "themselves are fewer" if prec == "f32" else
                                        "two 32-bit atomics (fixed-point hi and lo) per tap")}
    largest = max(prof, key=lambda f: prof[f][1]) if prof else None
    out["largest_family"] = largest
    if largest in FAMILY_NOTES:
        out["largest_family_note"] = FAMILY_NOTES[largest]
    return out


def near_roofline(prof, infos, applied, n, T, d, nv, prec, prof_step_ms, peaks):
    """ALU roofline of the Laplacian's near-field pass: per examined pair 2d
    flop (coordinate differences and squares), and for the in-range share
    18 flop (square root, scaling, exponential, 7 polynomial multiply-adds,
    difference) plus 2 per vector; one pass per nv vectors."""
    launches, ms = prof.get("near", (0, 0.0))
    passes = applied / n / T / nv          # near-field passes per layer
    f_in = NEAR_IN_RANGE[d]
    per_pair = 2 * d + f_in * (18 + 2 * nv)
    pairs = sum(i["near_pairs"] for i in infos) * passes
    flops = pairs * per_pair
    achieved = flops / (ms / 1e3) / 1e12 if ms > 0 else 0.0
    peak = peaks["fp32_tflops"] if prec == "f32" else peaks["fp64_tflops"]
    return {"bound": "alu", "kernel": "near", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": None,
            "peak_source": f"{'FP32' if prec == 'f32' else 'FP64'} FMA pipe, measured in this run (ml_measure_peak)",
            "work": f"{per_pair:.2f} flop per examined pair ({2 * d} for the distance, in-range share "
                    f"{f_in:.3f} x (18 + 2 x {nv})); {pairs:.3g} examined pairs in the profiled step",
            "pairs_per_s": pairs / (ms / 1e3) if ms > 0 else 0.0,
            "family_ms": {f: v[1] for f, v in prof.items()}, "family_launches": {f: v[0] for f, v in prof.items()},
            "region": "one extra step after the timed region with per-kernel CUDA events (eager launches), "
                      f"{prof_step_ms:.1f} ms"}


def cpu_baseline(layers, sig, ml, torch, dev_layers, forms, kernel="gauss", seconds=12.0, per_layer=False, nv=1):
    """Time the oracle's direct FP64 sum of (1/T) sum_t W_t V on a bounded row
    sample (about `seconds` of host time), and compare each GPU form's product
    on the same rows: E2 = ||y - y*||_2 / ||y*||_2 and the element-wise
    E_inf = max |y - y*| / ||v||_1 per vector."""
    from oracle import graph
    n, T = layers[0].shape[0], len(layers)
    b = nv if per_layer else 1
    rng = np.random.default_rng(123)
    V = rng.uniform(0, 1, (n, b))
    graph.W_apply(layers[0][:1000], sig[0], V[:1000], rows=np.arange(8))   # load the library, start threads
    r0 = np.sort(rng.choice(n, size=min(n, 64), replace=False))
    t0 = time.perf_counter()
    for t in range(T):
        graph.W_apply(layers[t], sig[t], V, rows=r0, kernel=kernel)
    dt = max(time.perf_counter() - t0, 1e-6)
    R = int(min(n, max(64, 64 * seconds / dt)))
    rows = np.sort(rng.choice(n, size=R, replace=False))
    t0 = time.perf_counter()
    ref = sum(graph.W_apply(layers[t], sig[t], V, rows=rows, kernel=kernel) for t in range(T)) / T
    el = time.perf_counter() - t0
    errs = {}
    for prec, target in forms:
        if kernel == "gauss":
            plans = [ml.ml_fastsum_plan(x, s, prec=prec, target_rel_err=target) for x, s in zip(dev_layers, sig)]
        else:
            plans = [ml.ml_fastsum_plan_ex(x, s, prec=prec, target_rel_err=target, kernel=kernel)
                     for x, s in zip(dev_layers, sig)]
        Y = torch.empty(n, b, dtype=torch.float64, device="cuda")
        ml.ml_fastsum_apply(plans, torch.as_tensor(V, device="cuda"), Y, mode="raw")
        got = Y.cpu().numpy()[rows]
        for pl in plans:
            pl.destroy()
        e2 = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        einf = float((np.abs(got - ref).max(axis=0) / np.abs(V).sum(axis=0)).max())
        errs[prec] = {"E2": e2, "E_inf": einf, "target": target, "rows": R, "vectors": b,
                      "vector": "uniform [0,1]", "operator": "(1/T) sum_t W_t"}
    base = {"value": R * T * b / el / 1e9, "unit": "Gpts·vec/s", "cores": graph.num_threads(), "kind": "oracle",
            "sample": f"direct FP64 sum of (1/T) sum_t W_t V, V of {b} column(s), on {R} sampled rows x {T} layers "
                      f"({el:.1f} s)"}
    return base, errs


if __name__ == "__main__":
    sys.exit(main())
