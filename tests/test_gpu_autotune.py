"""The measured choice of the spreading tile edge (a GPU tuning step, not
from the paper) changes only how the work is tiled: the tuned plan's product
(Alg. 1) matches the oracle's direct sum and the automatic plan's product."""
import numpy as np
import pytest
import torch

from oracle import graph
from paper_2007_05239_gb300 import _lib as ml
from paper_2007_05239_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [("f64", 1e-6), ("f32", 1e-4)])
def test_autotuned_plan_matches_rule_and_oracle(prec, tol):
    layers = workloads.image_voronoi_layers(300, 400, 8, 0.02, seed=21)
    X = layers[0]
    n = X.shape[0]
    dX = torch.as_tensor(X, device="cuda")
    v = np.random.default_rng(4).uniform(0, 1, n)
    dv = torch.as_tensor(v[:, None].copy(), device="cuda")
    rule = ml.ml_fastsum_plan_ex(dX, 0.2, prec=prec)
    tuned, b = ml.ml_fastsum_plan_autotune(dX, 0.2, nv=1, prec=prec)
    assert rule.info["nbins"] > 1            # a multi-tile grid: something to tune
    assert b == tuned.info["bin"] and b >= 2
    assert tuned.info["N"] == rule.info["N"] and tuned.info["taps"] == rule.info["taps"]
    Y0 = torch.empty_like(dv)
    Y1 = torch.empty_like(dv)
    ml.ml_fastsum_apply([rule], dv, Y0, mode="raw")
    ml.ml_fastsum_apply([tuned], dv, Y1, mode="raw")
    y0, y1 = Y0.cpu().numpy()[:, 0], Y1.cpu().numpy()[:, 0]
    # same method and parameters, other tiling: equal up to summation order
    assert np.linalg.norm(y1 - y0) / np.linalg.norm(y0) <= (1e-12 if prec == "f64" else 1e-5)
    rows = np.sort(np.random.default_rng(5).choice(n, 400, replace=False))
    ref = graph.W_apply(X, 0.2, v, rows=rows)
    assert np.linalg.norm(y1[rows] - ref) / np.linalg.norm(ref) <= tol
    # a second plan of the same shape takes the cached edge
    again, b2 = ml.ml_fastsum_plan_autotune(dX, 0.2, nv=1, prec=prec)
    assert b2 == b and again.info["bin"] == b


def test_bin_edge_beyond_shared_memory_is_refused():
    X = workloads.uniform_cube(5000, 3, seed=22)
    with pytest.raises(ml.MLError):
        ml.ml_fastsum_plan_ex(torch.as_tensor(X, device="cuda"), 0.02, prec="f64", bin=60)
