"""GPU tests of the parameter-model pieces: the MLP's loss and gradients against
the FP64 oracle, training, the exact direct summation of sampled rows, the
cloud statistics against their definitions, explicit-parameter plans, and a
small end-to-end run of the learned parameter choice."""
import numpy as np
import pytest
import torch

from oracle import graph
from oracle import mlp as omlp
from paper_2007_05239_gb300 import _lib as ml
from paper_2007_05239_gb300 import paramnet, workloads

pytestmark = pytest.mark.gpu


def test_mlp_loss_and_gradient_match_oracle():
    rng = np.random.default_rng(0)
    n_in, h, n_out, B = 12, 16, 2, 64
    m = ml.Mlp(n_in, h, n_out, seed=3)
    norm = (rng.normal(0, 1, n_in), rng.uniform(0.5, 2, n_in), rng.normal(0, 1, n_out), rng.uniform(0.5, 2, n_out))
    m.set_norm(*norm)
    X = rng.normal(0, 1, (B, n_in)).astype(np.float32)
    Y = rng.normal(0, 1, (B, n_out)).astype(np.float32)
    p = m.get_params().astype(np.float64)
    loss, g = m.loss_grad(X, Y)
    lref, gref = omlp.loss_grad(p, X, Y, n_in, h, n_out, norm)
    assert abs(loss - lref) <= 1e-5 * abs(lref)
    assert np.abs(g - gref).max() <= 1e-4 * np.abs(gref).max()
    Yp = m.forward(X)
    assert np.abs(Yp - omlp.forward(p, X, n_in, h, n_out, norm)).max() <= 1e-5 * np.abs(Yp).max()


def test_mlp_training_fits_a_smooth_function():
    rng = np.random.default_rng(1)
    X = rng.uniform(-2, 2, (512, 3)).astype(np.float32)
    Y = np.stack([np.sin(X[:, 0]) * X[:, 1], np.cos(X[:, 2])], axis=1).astype(np.float32)
    m = ml.Mlp(3, 32, 2, seed=5)
    m.set_norm(X.mean(0), X.std(0), Y.mean(0), Y.std(0))
    losses = m.train(X, Y, 1500, 3e-3)
    assert losses[-1] < 0.05 * losses[0]
    # the trained parameters evaluate the same on the oracle
    p = m.get_params().astype(np.float64)
    norm = (X.mean(0), X.std(0), Y.mean(0), Y.std(0))
    assert np.abs(m.forward(X) - omlp.forward(p, X, 3, 32, 2, norm)).max() <= 1e-4


def test_direct_sum_rows_is_exact():
    X = workloads.uniform_cube(5000, 3, seed=40)
    v = np.random.default_rng(2).uniform(-1, 1, 5000)
    rows = np.array([0, 17, 999, 4999], dtype=np.int64)
    got = ml.ml_direct_sum_rows(torch.as_tensor(X, device="cuda"), 0.07, torch.as_tensor(v, device="cuda"),
                                torch.as_tensor(rows, device="cuda")).cpu().numpy()
    ref = graph.W_apply(X, 0.07, v, rows=rows)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(v).sum()


def test_cloud_features_match_definition():
    X, sigma = workloads.cloud_for_mlp(3)
    f = ml.ml_cloud_features(torch.as_tensor(X, device="cuda"), sigma)
    n, d = X.shape
    ext = np.sort(X.max(0) - X.min(0))[::-1]
    box = ext[0]
    S = min(n, 2048)
    samp = X[np.arange(S) * (n // S)]
    D = np.sqrt(((samp[:, None, :] - samp[None, :, :]) ** 2).sum(-1))
    np.fill_diagonal(D, np.inf)
    nn = np.sort(D.min(1))
    q = [np.log10(nn[int(np.floor(a * (S - 1)))] / sigma) for a in (0.05, 0.5, 0.95)]
    ref = [np.log10(n), d, np.log10(sigma / box)] + list(np.pad(ext / box, (0, 3 - d))) + q
    assert np.allclose(f, ref, rtol=1e-5, atol=1e-5)


@pytest.mark.parametrize("taps,over", [(5, 2.5), (6, 2.0), (7, 3.0)])
def test_explicit_window_parameters(taps, over):
    X = workloads.uniform_cube(4000, 3, seed=41)
    v = np.random.default_rng(3).uniform(0, 1, 4000)
    plan = ml.ml_fastsum_plan_ex(torch.as_tensor(X, device="cuda"), 0.1, taps=taps, oversampling=over, prec="f64",
                                 target_rel_err=1e-8)
    info = plan.info
    assert info["taps"] == taps and abs(info["n_os"] / info["N"] - over) <= 2.0 / info["N"]
    Y = torch.empty(4000, 1, dtype=torch.float64, device="cuda")
    ml.ml_fastsum_apply([plan], torch.as_tensor(v[:, None].copy(), device="cuda"), Y, mode="raw")
    ref = graph.W_apply(X, 0.1, v)
    err = np.linalg.norm(Y.cpu().numpy()[:, 0] - ref) / np.linalg.norm(ref)
    # the calibrated worst-case model 9 exp(-pi W sqrt(1 - 1/sigma_os)) bounds the error
    assert err <= 9.0 * np.exp(-np.pi * taps * np.sqrt(1 - 1 / over))


def test_learned_choice_small_end_to_end():
    # a small version of the learned-parameter workload (the full run trains on
    # 500 clouds and evaluates 200: python -m paper_2007_05239_gb300.paramnet):
    # train on the method's own measurements of 30 clouds, then compare with
    # the fixed rule on 8 unseen clouds
    X, Y, ids = paramnet.make_dataset(0, 30, 8, "f32", 1e-4)
    assert X.shape == (240, ml.ML_FEATURES + 3) and np.isfinite(Y).all() and ids.shape == (240,)
    fit = ids < 25
    model, losses, _ = paramnet.train(X[fit], Y[fit], epochs=1500)
    assert losses[-1] < 0.5 * losses[0]
    margin = paramnet.calibrate_margin(model, X[~fit], Y[~fit])
    assert margin >= 1.0
    ev = paramnet.evaluate(model, 5000, 8, "f32", 1e-4, margin=max(margin, 2.0))
    assert ev["success_fixed"] == 1.0
    assert ev["success_learned"] >= 0.75
    # without a model the learned planner is the fixed rule
    pts, sigma, *_ = paramnet.cloud(5000)
    plan, chosen = ml.ml_fastsum_plan_learned(pts, sigma, None, prec="f32", target_rel_err=1e-4)
    ref = ml.ml_fastsum_plan(pts, sigma, prec="f32", target_rel_err=1e-4)
    assert chosen == (0.0, 0.0, 0.0) and plan.info["taps"] == ref.info["taps"] and plan.info["N"] == ref.info["N"]


def test_per_factor_margins_exclude_cut_bandwidths():
    # a model whose per-factor margins make every cut bandwidth (f < 1)
    # unreachable may only pick the full bandwidth, or fall back to the rule
    m = ml.Mlp(ml.ML_FEATURES + 3, 16, 2, seed=4)
    m.set_norm(np.zeros(ml.ML_FEATURES + 3), np.ones(ml.ML_FEATURES + 3), np.array([-6.0, -1.0]), np.ones(2))
    m.set_margins([1e30, 1e30, 0.0])
    pts, sigma, *_ = paramnet.cloud(5001)
    plan, chosen = ml.ml_fastsum_plan_learned(pts, sigma, m, prec="f32", target_rel_err=1e-4, margin=1.0)
    assert chosen[0] in (0.0, 1.0)
    with pytest.raises(ml.MLError):
        m.set_margins([1.0, 2.0])


def test_learned_choice_gains_over_fixed_rule():
    # what the trained network gains: trained on the method's own error and
    # time measurements of 300 clouds (10 candidates each, 10 % of the clouds
    # held out to calibrate one error margin per bandwidth factor at the 0.999
    # quantile of the held-out residuals), then on 24 unseen clouds every
    # learned choice must meet the 1e-4 target (judged by the direct sum on
    # sampled rows) and the products must be faster than with the fixed rule
    # (geometric mean of the time ratios below 1)
    X, Y, ids = paramnet.make_dataset(0, 300, 10, "f32", 1e-4)
    fit = ids < 270
    model, losses, _ = paramnet.train(X[fit], Y[fit], epochs=3000)
    margins = paramnet.calibrate_margins(model, X[~fit], Y[~fit], 0.999)
    model.set_margins(margins)
    ev = paramnet.evaluate(model, 6000, 24, "f32", 1e-4, margin=max(margins))
    assert ev["success_fixed"] == 1.0
    assert ev["success_learned"] == 1.0, [c["learned"] for c in ev["clouds"] if c["learned"]["E2"] > 1e-4]
    assert ev["time_ratio_geomean"] < 1.0, ev["time_ratio_geomean"]
