"""Parity at the full sizes of the three large synthetic workloads, in the
launch configuration the bench uses, on rows the oracle computes exactly
(direct FP64 sums over all n points), plus the eigen residual check that
holds at any size (a dense eigensolve of a 10^6-node graph is infeasible).
"""
import numpy as np
import pytest
import torch

from oracle import graph
from paper_2007_05239_gb300 import _lib as ml
from paper_2007_05239_gb300 import workloads

pytestmark = pytest.mark.gpu


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def sampled_parity(layers, sig, prec, target, rows_n, b=1, seed=0):
    n = layers[0].shape[0]
    rng = np.random.default_rng(seed)
    rows = np.sort(rng.choice(n, size=rows_n, replace=False))
    V = rng.uniform(0, 1, (n, b))
    plans = [ml.ml_fastsum_plan(dev(L), s, prec=prec, target_rel_err=target) for L, s in zip(layers, sig)]
    Y = torch.empty(n, b, dtype=torch.float64, device="cuda")
    ml.ml_fastsum_apply(plans, dev(V), Y, mode="raw")
    got = Y.cpu().numpy()[rows]
    ref = sum(graph.W_apply(L, s, V, rows=rows) for L, s in zip(layers, sig)) / len(layers)
    err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    # degrees of the first layer on the same rows
    deg = plans[0].table(2)[rows]
    dref = graph.degrees(layers[0], sig[0], rows=rows)
    derr = float(np.linalg.norm(deg - dref) / np.linalg.norm(dref))
    for p in plans:
        p.destroy()
    return err, derr


def test_image_n1e6_three_layers_f64():
    layers = workloads.image_voronoi_layers(1000, 1000, 8, 0.02, seed=2)
    err, derr = sampled_parity(layers, [0.2] * 3, "f64", 1e-6, 512)
    assert err <= 1e-6 and derr <= 1e-6, (err, derr)


def test_gmm_n250k_52_layers_f32_batched():
    layers, _ = workloads.gmm_band_layers(250_000, 104, 12, seed=3)
    sig = [0.5 * float((L.max(0) - L.min(0)).max()) for L in layers]
    err, derr = sampled_parity(layers, sig, "f32", 1e-4, 256, b=8)
    assert err <= 1e-4 and derr <= 1e-4, (err, derr)


@pytest.mark.parametrize("prec,target", [("f32", 1e-4), ("f64", 1e-6)])
def test_image_n1e7_two_layers(prec, target):
    layers = workloads.image_discs_layers(2500, 4000, 5, 0.02, seed=4)
    err, derr = sampled_parity(layers, [0.15] * 2, prec, target, 128)
    assert err <= target and derr <= target, (err, derr)


def test_eigen_residuals_image_n1e6():
    # eigenpairs of L_1 at full size: residuals of the GPU operator, the
    # spectrum inside [0, 2], orthonormal vectors; one layer alone has
    # lambda_0 = 0 (null vector D^{1/2} 1); the mean of layers with different
    # degrees has lambda_0 > 0
    layers = workloads.image_voronoi_layers(1000, 1000, 8, 0.02, seed=2)
    n, k = 1_000_000, 8
    plans = [ml.ml_fastsum_plan(dev(L), 0.2, prec="f64", target_rel_err=1e-8) for L in layers]
    V = torch.empty(n * k, dtype=torch.float64, device="cuda")
    lam, nconv, st = ml.ml_lanczos_eigs(plans, k, p=1.0, tol=1e-9, seed=2, evecs=V)
    assert st == ml.ML_OK and nconv == k
    assert (lam >= -1e-9).all() and (lam <= 2).all()
    lam1, _, st1 = ml.ml_lanczos_eigs(plans[:1], 3, p=1.0, tol=1e-9, seed=3)
    assert st1 == ml.ML_OK and abs(lam1[0]) <= 1e-8
    Phi = V.view(k, n).T.contiguous()
    APhi = torch.empty_like(Phi)
    ml.ml_fastsum_apply(plans, Phi, APhi, mode="normalized")
    theta = torch.as_tensor(1.0 - lam, device="cuda")
    res = torch.linalg.norm(APhi - Phi * theta[None, :], dim=0).cpu().numpy()
    assert res.max() <= 1e-7, res
    G = (Phi.T @ Phi).cpu().numpy()
    assert np.abs(G - np.eye(k)).max() <= 1e-10
