"""Learned choice of a layer's NFFT parameters (bandwidth factor, window width,
oversampling) from point-cloud statistics.

Every number used for training comes from the method itself through the C
ABI: `ml_fastsum_plan_ex` with the candidate parameters, `ml_fastsum_apply`
for the product (its time measured with CUDA events) and `ml_direct_sum_rows`,
the exact product on sampled rows, as the measure of the error.  The model is
the library's FP32 MLP (`ml_mlp_*`, trained on the GPU by the library's own
kernels); `ml_fastsum_plan_learned` uses it, and falls back to the calibrated
fixed rule of `ml_fastsum_plan` when no candidate qualifies.

    python -m paper_2007_05239_gb300.paramnet --train 500 --per-cloud 10 --eval 200 --out paramnet_f32.npz

Inputs: the seeded clouds of `workloads.cloud_for_mlp` (n log-uniform in
[1e4, 1e6], d in 1..3, uniform / Gaussian-mixture / piecewise-constant).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import _lib as ml
from . import workloads

FACTORS = (0.7, 0.85, 1.0)
TAPS = (4, 5, 6, 7, 8)
OVERSAMPLING = (2.0, 2.5, 3.0)
CANDIDATES = [(f, w, s) for f in FACTORS for w in TAPS for s in OVERSAMPLING]


def _torch():
    import torch
    return torch


def reference(points, sigma, v, rows):
    """Exact (W v)[rows] (GPU direct summation)."""
    return ml.ml_direct_sum_rows(points, sigma, v, rows)


def apply_time_ms(plan, v, repeats=3):
    torch = _torch()
    Y = torch.empty_like(v)
    ml.ml_fastsum_apply([plan], v, Y, mode="raw")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(repeats):
        ml.ml_fastsum_apply([plan], v, Y, mode="raw")
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / repeats, Y


def measure(points, sigma, prec, target, cand, v, rows, ref, N0):
    """(log10 E2 on the sampled rows, log10 product time in ms) of one candidate."""
    f, w, s = cand
    N = max(4, 2 * int(round(0.5 * f * N0)))
    plan = ml.ml_fastsum_plan_ex(points, sigma, N=N, taps=w, oversampling=s, prec=prec, target_rel_err=target)
    t, Y = apply_time_ms(plan, v)
    got = Y[rows, 0]
    err = float((got - ref).norm() / ref.norm())
    plan.destroy()
    return np.log10(max(err, 1e-16)), np.log10(max(t, 1e-4))


def cloud(i, rows_per_cloud=256):
    torch = _torch()
    X, sigma = workloads.cloud_for_mlp(i)
    pts = torch.as_tensor(X, device="cuda")
    rng = np.random.default_rng(777 + i)
    v = torch.as_tensor(rng.uniform(0, 1, (X.shape[0], 1)), device="cuda")
    rows = torch.as_tensor(np.sort(rng.choice(X.shape[0], size=min(rows_per_cloud, X.shape[0]), replace=False)),
                           device="cuda")
    ref = reference(pts, sigma, v[:, 0].contiguous(), rows)
    return pts, sigma, v, rows, ref


def auto_bandwidth(pts, sigma, prec, target):
    plan = ml.ml_fastsum_plan(pts, sigma, prec=prec, target_rel_err=target)
    N0 = plan.info["N"]
    plan.destroy()
    return N0


def make_dataset(first, count, per_cloud, prec, target, seed=0):
    rng = np.random.default_rng(seed)
    Xs, Ys, ids = [], [], []
    for i in range(first, first + count):
        pts, sigma, v, rows, ref = cloud(i)
        if float(ref.norm()) == 0.0:
            continue
        feat = ml.ml_cloud_features(pts, sigma)
        N0 = auto_bandwidth(pts, sigma, prec, target)
        for ci in rng.choice(len(CANDIDATES), size=per_cloud, replace=False):
            cand = CANDIDATES[ci]
            try:
                le, lt = measure(pts, sigma, prec, target, cand, v, rows, ref, N0)
            except ml.MLError as e:   # a candidate the library refuses (e.g. a grid beyond the limits)
                print(f"cloud {i} candidate {cand}: {e}", flush=True)
                continue
            Xs.append(np.concatenate([feat, np.asarray(cand, dtype=np.float32)]))
            Ys.append([le, lt])
            ids.append(i)
    return np.asarray(Xs, dtype=np.float32), np.asarray(Ys, dtype=np.float32), np.asarray(ids)


def train(X, Y, hidden=64, epochs=4000, lr=3e-3, seed=1):
    model = ml.Mlp(X.shape[1], hidden, Y.shape[1], seed=seed)
    mx, sx = X.mean(0), X.std(0) + 1e-6
    my, sy = Y.mean(0), Y.std(0) + 1e-6
    model.set_norm(mx, sx, my, sy)
    losses = model.train(X, Y, epochs, lr)
    return model, losses, (mx, sx, my, sy)


def calibrate_margin(model, X, Y, quantile=0.99):
    """Safety factor on the error target from held-out samples: the planner
    keeps a candidate when its predicted error is at most target / margin, so
    margin = 10^q with q the given quantile of (measured - predicted) log10
    error; at least 1."""
    r = Y[:, 0] - model.forward(X)[:, 0]
    return float(10.0 ** max(0.0, float(np.quantile(r, quantile))))


def calibrate_margins(model, X, Y, quantile=0.995):
    """One safety factor per bandwidth factor f of the candidates: 10^q_f with
    q_f the quantile of (measured - predicted) log10 error over the held-out
    samples of that f (the cut bandwidths err more, and less predictably);
    at least 1."""
    r = Y[:, 0] - model.forward(X)[:, 0]
    out = []
    for f in FACTORS:
        sel = np.isclose(X[:, ml.ML_FEATURES], f)
        q = float(np.quantile(r[sel] if sel.any() else r, quantile))
        out.append(float(10.0 ** max(0.0, q)))
    return out


def evaluate(model, first, count, prec, target, margin=2.0):
    """Learned choice vs the fixed rule on unseen clouds: error (against the
    direct sum) and product time for both."""
    rows_out = []
    for i in range(first, first + count):
        pts, sigma, v, rows, ref = cloud(i)
        out = {"cloud": i, "n": int(pts.shape[0]), "d": int(pts.shape[1])}
        for name, mdl in (("learned", model), ("fixed", None)):
            plan, chosen = ml.ml_fastsum_plan_learned(pts, sigma, mdl, prec=prec, target_rel_err=target, margin=margin)
            t, Y = apply_time_ms(plan, v)
            err = float((Y[rows, 0] - ref).norm() / ref.norm())
            info = plan.info
            out[name] = {"E2": err, "ms": t, "taps": info["taps"], "N": info["N"], "n_os": info["n_os"],
                         "chosen": list(chosen)}
            plan.destroy()
        rows_out.append(out)
    ok_l = np.mean([r["learned"]["E2"] <= target for r in rows_out])
    ok_f = np.mean([r["fixed"]["E2"] <= target for r in rows_out])
    ratio = float(np.exp(np.mean([np.log(r["learned"]["ms"] / r["fixed"]["ms"]) for r in rows_out])))
    return {"success_learned": float(ok_l), "success_fixed": float(ok_f), "time_ratio_geomean": ratio,
            "clouds": rows_out}


def save(path, model, norm, margin, margins=None):
    np.savez(path, params=model.get_params(), in_mean=norm[0], in_std=norm[1], out_mean=norm[2], out_std=norm[3],
             hidden=model.hidden, margin=margin, margins=np.zeros(3) if margins is None else np.asarray(margins))


def load_model(path):
    """(model, margin) saved by `save`; per-factor margins are set on the model."""
    z = np.load(path)
    model = ml.Mlp(len(z["in_mean"]), int(z["hidden"]), len(z["out_mean"]))
    model.set_params(z["params"])
    model.set_norm(z["in_mean"], z["in_std"], z["out_mean"], z["out_std"])
    if "margins" in z:
        model.set_margins(z["margins"])
    return model, float(z["margin"])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=500, help="training clouds")
    ap.add_argument("--per-cloud", type=int, default=10, help="candidates measured per training cloud")
    ap.add_argument("--eval", type=int, default=200, help="unseen evaluation clouds")
    ap.add_argument("--prec", default="f32")
    ap.add_argument("--target", type=float, default=1e-4)
    ap.add_argument("--epochs", type=int, default=4000)
    ap.add_argument("--holdout", type=float, default=0.1, help="share of training clouds held out for the margin")
    ap.add_argument("--quantile", type=float, default=0.995,
                    help="quantile of held-out error residuals (per bandwidth factor)")
    ap.add_argument("--out", default=None)
    ap.add_argument("--report", default=None)
    a = ap.parse_args()
    t0 = time.time()
    X, Y, ids = make_dataset(0, a.train, a.per_cloud, a.prec, a.target)
    t1 = time.time()
    fit = ids < a.train * (1.0 - a.holdout)
    model, losses, norm = train(X[fit], Y[fit], epochs=a.epochs)
    margins = calibrate_margins(model, X[~fit], Y[~fit], a.quantile)
    model.set_margins(margins)
    margin = max(margins)
    t2 = time.time()
    ev = evaluate(model, 5000, a.eval, a.prec, a.target, margin=margin)
    t3 = time.time()
    rep = {"samples": int(X.shape[0]), "fit_samples": int(fit.sum()), "margins": margins,
           "final_loss": float(losses[-1]), "first_loss": float(losses[0]),
           "data_s": t1 - t0, "train_s": t2 - t1, "eval_s": t3 - t2,
           **{k: v for k, v in ev.items() if k != "clouds"}}
    print(json.dumps(rep))
    if a.out:
        save(a.out, model, norm, margin, margins)
    if a.report:
        with open(a.report, "w") as f:
            json.dump({**rep, "clouds": ev["clouds"]}, f)


if __name__ == "__main__":
    main()
