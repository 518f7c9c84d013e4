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

Default workload: the image-like multilayer graph, n = 1,000,000 pixels,
3 layers of d = 3 (RGB; x, y, texture; box-filtered RGB), sigma = 0.2, FP64
form at 1e-6 relative error, k = 20 eigenpairs of L_{-1,delta} (p = -1).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
                  [--workload NAME] [--prec f32|f64] [--p 1|-1] [--k K]

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
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# ALU roofs at 152 SMs x 2070 MHz.  FP32 form: 128 FFMA lanes per SM and clock,
# 2 flop each.  FP64 form: every tap is a double-word multiply-add on the same
# FP32 lanes, at least 10 lane operations per FP64 multiply-add (exact product
# by FMA: 4; exact two-sum: 6), i.e. 2 flop per 10 lane operations.
FP32_LANE_OPS = 152 * 2.070e9 * 128
ALU_PEAK_TFLOPS = {"f32": FP32_LANE_OPS * 2 / 1e12, "f64": FP32_LANE_OPS * 2 / 10 / 1e12}
ALU_PEAK_SOURCE = {
    "f32": "FP32 pipe: 152 SMs x 2070 MHz x 128 FFMA/clk x 2 flop",
    "f64": "double-word FP64 multiply-adds on the FP32 pipe: 152 SMs x 2070 MHz x 128 lane ops/clk "
           "/ 10 lane ops per multiply-add x 2 flop",
}


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
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="image_voronoi_n1e6_T3", choices=sorted(WORKLOADS))
    ap.add_argument("--prec", default=None, choices=["f32", "f64"])
    ap.add_argument("--p", type=float, default=None)
    ap.add_argument("--k", type=int, default=None)
    ap.add_argument("--no-baseline", action="store_true")
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

    layers, sig = make_layers(args.workload)
    n, T = layers[0].shape[0], len(layers)
    dev_layers = [torch.as_tensor(L, device="cuda") for L in layers]
    k, p, prec, target = spec["k"], spec["p"], spec["prec"], spec["target"]

    kernel = spec.get("kernel", "gauss")
    if kernel != "gauss" and args.planner != "rule":
        raise SystemExit("the learned planner covers the Gaussian kernel only")
    planner = make_planner(args.planner, prec, target, ml, kernel)
    plan_all = make_planner("many", prec, target, ml, kernel) if args.planner == "rule" else None
    apply_plans = None
    if args.mode == "apply":
        apply_plans = [planner(x, s) for x, s in zip(dev_layers, sig)]
        Xa = torch.as_tensor(np.random.default_rng(7).uniform(0, 1, (n, args.b)), device="cuda")
        Ya = torch.empty_like(Xa)

    def step(dl, evecs):
        if apply_plans is not None:
            before = sum(pl.info["applied_vectors"] for pl in apply_plans)
            ml.ml_fastsum_apply(apply_plans, Xa, Ya, mode="normalized")
            applied = (sum(pl.info["applied_vectors"] for pl in apply_plans) - before) * n
            return None, 0, applied, [pl.info for pl in apply_plans]
        plans = plan_all(dl, sig) if plan_all else [planner(x, s) for x, s in zip(dl, sig)]
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

    nev = n * k * (T if spec.get("per_layer") else 1)
    evecs = torch.empty(nev, dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        step(dev_layers, evecs)
    torch.cuda.synchronize()
    barrier()

    # ---- timed region (device-resident inputs; kernel timing off, so the inner
    #      conjugate-gradient iterations replay their CUDA graphs)
    clocks = ClockSampler(local)
    clocks.start()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    e0.record(stream)
    applied = 0
    for _ in range(args.steps):
        lam, nconv, a, msz = step(dev_layers, evecs)
        applied += a
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms_total = e0.elapsed_time(e1)
    t_max, tot_applied = reduce_over_ranks(ms_total, applied, "cuda")
    value = tot_applied / (t_max / 1e3) / 1e9

    # ---- kernel timing: one more step with CUDA events around every library
    #      launch on its stream (per-kernel events cannot sit inside a graph,
    #      so this step launches eagerly)
    ml.ml_profile_reset()
    ml.ml_profile_enable(True)
    torch.cuda.synchronize()
    e0.record(stream)
    _, _, applied_prof, msz = step(dev_layers, evecs)
    e1.record(stream)
    torch.cuda.synchronize()
    ml.ml_profile_enable(False)
    prof_step_ms = e0.elapsed_time(e1)
    prof = ml.ml_profile_read()
    launches = int(sum(v[0] for v in prof.values())) * args.steps   # a graph replay runs the same kernels

    # ---- roofline of the dominant kernel family
    d = spec["d"]
    W = msz[0]["taps"]
    taps = W ** d
    fam = max(("spread", "interp", "near"), key=lambda f: prof.get(f, (0, 0.0))[1])
    fam_launches, fam_ms = prof.get(fam, (0, 0.0))
    flops = applied_prof * 2.0 * taps             # one multiply-add per tap and point-vector
    achieved = flops / (fam_ms / 1e3) / 1e12 if fam_ms > 0 else 0.0
    peak = ALU_PEAK_TFLOPS[prec]
    # the same kernel against the HBM roof: algorithmic bytes per point and pass
    # (window table 8 d W + packed taps 4 in the FP64 form, coordinates 4 d in the
    # FP32 form; permutation 4, D^{-1/2} 8) plus 8 B per vector read (spread) or
    # read and written (interp); a pass carries nv vectors
    nv = min(args.b, 8) if args.mode == "apply" else (spec.get("block", 1) if spec.get("per_layer") else 1)
    if fam == "near":
        roofline = near_roofline(prof, msz, applied_prof, n, T, d, nv, prec, prof_step_ms)
    point_bytes = (8 * d * W + 4 if prec == "f64" else 4 * d) + 4 + 8
    vec_bytes = 8 if fam == "spread" else 16
    hbm_bytes = applied_prof / nv * point_bytes + applied_prof * vec_bytes
    hbm_gbs = hbm_bytes / (fam_ms / 1e3) / 1e9 if fam_ms > 0 else 0.0
    hbm_peak = float(measured_peaks().get("hbm_gbs", 6800.0))
    # DRAM traffic per launch from the ncu capture of this kernel on this workload
    # (dram__bytes_read.sum + dram__bytes_write.sum; one launch = one layer,
    # 1e6 points, one vector), only where that capture applies
    traffic, traffic_src = None, None
    key = (args.workload, prec, fam, W, nv)
    if key in NCU_TRAFFIC:
        traffic, traffic_src = NCU_TRAFFIC[key]
    # the step's largest kernel family by time (on the per-layer workload the
    # FP64 Gram / update products of the block Lanczos steps, not the product)
    largest = max(prof, key=lambda f: prof[f][1]) if prof else None
    if fam != "near":
        roofline = {"bound": "alu", "kernel": fam, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": traffic, "traffic_source": traffic_src,
                    "algorithmic_bytes_per_launch": hbm_bytes / fam_launches if fam_launches else None,
                    "peak_source": ALU_PEAK_SOURCE[prec],
                    "work": f"2 flop per tap, W^d = {taps} taps per point-vector, W = {W}",
                    "hbm": {"achieved": hbm_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": hbm_gbs / hbm_peak,
                            "bytes_per_point_pass": point_bytes, "bytes_per_point_vector": vec_bytes,
                            "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth)"},
                    "family_ms": {f: v[1] for f, v in prof.items()}, "family_launches": {f: v[0] for f, v in prof.items()},
                    "region": "one extra step after the timed region with per-kernel CUDA events (eager launches), "
                              f"{prof_step_ms:.1f} ms"}

    roofline["largest_family"] = largest
    if largest in FAMILY_NOTES:
        roofline["largest_family_note"] = FAMILY_NOTES[largest]

    # ---- end to end through the C ABI with host buffers (pinned)
    host_layers = [torch.as_tensor(L).pin_memory() for L in layers]
    host_evecs = torch.empty(nev, dtype=torch.float64).pin_memory()
    if args.mode == "apply":
        hx = Xa.cpu().pin_memory()
        hy = torch.empty_like(hx).pin_memory()
        h2d, d2h = hx.numel() * 8, hy.numel() * 8
    else:
        h2d = sum(L.numel() * 8 for L in host_layers)
        d2h = nev * 8 + nev // n * 8
    torch.cuda.synchronize()
    barrier()
    e0.record(stream)
    applied_e2e = 0
    for _ in range(args.steps):
        if args.mode == "apply":
            before = sum(pl.info["applied_vectors"] for pl in apply_plans)
            ml.ml_fastsum_apply(apply_plans, hx, hy, mode="normalized")   # host buffers: staged by the library
            applied_e2e += (sum(pl.info["applied_vectors"] for pl in apply_plans) - before) * n
            continue
        # the plans take the pinned host layers through the C ABI and copy them
        # to the device themselves (the learned planner reads device points)
        dl = host_layers if args.planner == "rule" else [x.to("cuda", non_blocking=True) for x in host_layers]
        lam_e, _, a, _ = step(dl, host_evecs)
        applied_e2e += a
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    e2e_ms = e0.elapsed_time(e1)
    e2e_t, e2e_work = reduce_over_ranks(e2e_ms, applied_e2e, "cuda")
    e2e_val = e2e_work / (e2e_t / 1e3) / 1e9

    line = {
        "metric": metric_name(spec), "value": value, "unit": "Gpts·vec/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": prec, "data": "synthetic", "config": config_dict(args, spec, n, T),
        "mode": args.mode, "gpu_launches": launches,
        "e2e": {"value": e2e_val, "unit": "Gpts·vec/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "roofline": roofline, "clocks": clk,
    }

    # ---- CPU baseline (oracle on the host cores) and sampled accuracy, rank 0 at N = 1
    if rank == 0 and world == 1 and not args.no_baseline:
        line["cpu_baseline"], line["rel_err_sampled"] = cpu_baseline(layers, sig, planner, dev_layers, ml, torch,
                                                                     kernel)
    if args.mode == "eig":
        line["lanczos_s"] = t_max / args.steps / 1e3
        line["eigenvalues"] = [float(x) for x in lam[:min(5, k)]]
        line["nconv"] = int(nconv)
    else:
        line["metric"] = (f"fast-summation Gpts·vec/s ({prec.upper()} form) of one multilayer normalised product, "
                          f"b={args.b}")
        line["config"]["b"] = args.b
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


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
    peak = 152 * 2.070e9 * 4 / 1e12
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
                     "peak_source": "FP64 pipe: 152 SMs x 2070 MHz x 2 DFMA/clk x 2 flop",
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
FP64_PIPE_TFLOPS = 152 * 2.070e9 * 2 * 2 / 1e12   # 2 DFMA per SM and clock

# what a step's largest kernel family is, where it is not the product itself
FAMILY_NOTES = {
    "dots": "FP64 Gram products of the Lanczos steps, bound by the FP64 pipe "
            "(profiles/lgram_block_lanczos_mixture_T52.md)",
    "update": "FP64 basis updates of the Lanczos steps, bound by the FP64 pipe",
    "plan": "plan set-up of every layer (bounding box, sort, Fourier tables, degrees): chains of small kernels "
            "and host synchronisations; the timed steps build the layers' plans concurrently, so the summed event "
            "times of the profiled step overstate its share",
}

# ncu DRAM bytes (read + write) of one launch, keyed by (workload, form, kernel
# family, window width, vectors per pass); valid while the kernel is unchanged
# since the capture named beside it
NCU_TRAFFIC = {
    ("image_voronoi_n1e6_T3", "f64", "spread", 7, 1):
        (192.6e6 + 10.4e6, "profiles/spread_interp_f64_image_n1e6.md: k_spread_f64<3,7,1>, one layer"),
    ("image_voronoi_n1e6_T3", "f64", "interp", 7, 1):
        (195.7e6 + 7.6e6, "profiles/spread_interp_f64_image_n1e6.md: k_interp_f64<3,7,1>, one layer"),
}


def near_roofline(prof, infos, applied, n, T, d, nv, prec, prof_step_ms):
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
    peak = ALU_PEAK_TFLOPS["f32"] if prec == "f32" else FP64_PIPE_TFLOPS
    return {"bound": "alu", "kernel": "near", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": None,
            "peak_source": ALU_PEAK_SOURCE["f32"] if prec == "f32" else
            "FP64 pipe: 152 SMs x 2070 MHz x 2 DFMA/clk x 2 flop",
            "work": f"{per_pair:.2f} flop per examined pair ({2 * d} for the distance, in-range share "
                    f"{f_in:.3f} x (18 + 2 x {nv})); {pairs:.3g} examined pairs in the profiled step",
            "pairs_per_s": pairs / (ms / 1e3) if ms > 0 else 0.0,
            "family_ms": {f: v[1] for f, v in prof.items()}, "family_launches": {f: v[0] for f, v in prof.items()},
            "region": "one extra step after the timed region with per-kernel CUDA events (eager launches), "
                      f"{prof_step_ms:.1f} ms"}


def cpu_baseline(layers, sig, planner, dev_layers, ml, torch, kernel="gauss"):
    """Time the oracle's direct FP64 sum of (1/T) sum_t W_t v on a bounded row
    sample (~12 s), and compare the GPU's FP64/FP32-form result on the same rows."""
    from oracle import graph
    n, T = layers[0].shape[0], len(layers)
    rng = np.random.default_rng(123)
    v = rng.uniform(0, 1, n)
    graph.W_apply(layers[0][:1000], sig[0], v[:1000], rows=np.arange(8))   # load the library, start threads
    r0 = np.sort(rng.choice(n, size=min(n, 64), replace=False))
    t0 = time.perf_counter()
    for t in range(T):
        graph.W_apply(layers[t], sig[t], v, rows=r0, kernel=kernel)
    dt = max(time.perf_counter() - t0, 1e-6)
    R = int(min(n, max(64, 64 * 12.0 / dt)))
    rows = np.sort(rng.choice(n, size=R, replace=False))
    t0 = time.perf_counter()
    ref = sum(graph.W_apply(layers[t], sig[t], v, rows=rows, kernel=kernel) for t in range(T)) / T
    el = time.perf_counter() - t0
    plans = [planner(x, s) for x, s in zip(dev_layers, sig)]
    Y = torch.empty(n, 1, dtype=torch.float64, device="cuda")
    ml.ml_fastsum_apply(plans, torch.as_tensor(v[:, None].copy(), device="cuda"), Y, mode="raw")
    got = Y.cpu().numpy()[rows, 0]
    for pl in plans:
        pl.destroy()
    err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    base = {"value": R * T / el / 1e9, "unit": "Gpts·vec/s", "cores": graph.num_threads(), "kind": "oracle",
            "sample": f"direct FP64 sum of (1/T) sum_t W_t v on {R} sampled rows x {T} layers ({el:.1f} s)"}
    return base, {"E2": err, "rows": R, "vector": "uniform [0,1]", "operator": "(1/T) sum_t W_t"}


if __name__ == "__main__":
    sys.exit(main())
