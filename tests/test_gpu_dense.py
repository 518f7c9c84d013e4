"""Dense layers (the explicit regime for small graphs, any feature
dimension; W of Sec. 2 stored): products against the oracle's direct sums,
eigenpairs against dense eigensolves, mixed with fast-summation layers, and
from a given weight matrix (a stochastic block model)."""
import numpy as np
import pytest
import torch

from oracle import eigen, graph
from paper_2007_05239_gb300 import _lib as ml
from paper_2007_05239_gb300 import workloads

pytestmark = pytest.mark.gpu


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def high_d_layers(n, seed):
    layers, truth = workloads.gmm_band_layers(n, 104, 6, seed=seed, group=52)   # two layers of d = 52
    return layers, truth


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-6)])
def test_dense_products_match_direct_sums(prec, tol):
    layers, _ = high_d_layers(1500, 50)
    X = layers[0]
    n = X.shape[0]
    plan = ml.ml_dense_plan(dev(X), 1.0, prec=prec)
    assert plan.info["dense"] == 1
    rng = np.random.default_rng(1)
    V = rng.uniform(0, 1, (n, 4))
    Y = torch.empty(n, 4, dtype=torch.float64, device="cuda")
    ml.ml_fastsum_apply([plan], dev(V), Y, mode="raw")
    ref = graph.W_apply(X, 1.0, V)
    assert np.linalg.norm(Y.cpu().numpy() - ref) / np.linalg.norm(ref) <= tol
    # degrees and the normalised operator
    deg = graph.degrees(X, 1.0)
    assert np.abs(plan.table(2) - deg).max() / deg.max() <= tol
    Y1 = torch.empty(n, 1, dtype=torch.float64, device="cuda")
    ml.ml_fastsum_apply([plan], dev(V[:, :1]), Y1, mode="normalized")
    ref1 = graph.A_apply(X, 1.0, V[:, 0])
    assert np.linalg.norm(Y1.cpu().numpy()[:, 0] - ref1) / np.linalg.norm(ref1) <= tol


def test_dense_eigenpairs_and_mixed_layers():
    layers, _ = high_d_layers(1200, 51)
    n, k = 1200, 6
    dplan = ml.ml_dense_plan(dev(layers[0]), 1.0, prec="f64")
    V = torch.empty(k * n, dtype=torch.float64, device="cuda")
    lam, nconv, st = ml.ml_lanczos_eigs([dplan], k, p=1.0, tol=1e-11, seed=2, evecs=V)
    lam_ref, V_ref = eigen.lsym_eigs(layers[0], 1.0, k + 3)
    assert np.abs(lam - lam_ref[:k]).max() <= 1e-8
    for g in eigen.eigen_groups(lam_ref, rel_gap=1e-6):
        if max(g) < k:
            assert eigen.subspace_angle(V.cpu().numpy().reshape(k, n).T[:, g], V_ref[:, g]) <= 1e-6
    # a dense d = 52 layer with a fast-summation d = 2 layer, p = -1
    X2 = workloads.uniform_cube(n, 2, seed=52)
    fplan = ml.ml_fastsum_plan(dev(X2), 0.08, prec="f64", target_rel_err=1e-12)
    lam, nconv, st = ml.ml_lanczos_eigs([dplan, fplan], 5, p=-1.0, tol=1e-10, seed=3)
    lam_ref, _ = eigen.Lp_eigs([layers[0], X2], [1.0, 0.08], -1.0, 5)
    assert np.abs(lam - lam_ref).max() <= 1e-8


def test_dense_layer_from_a_block_model_matrix():
    # two-block stochastic block model (p_in 0.3, p_out 0.05), seeded
    n, k = 600, 4
    rng = np.random.default_rng(53)
    blocks = np.repeat([0, 1], n // 2)
    P = np.where(blocks[:, None] == blocks[None, :], 0.3, 0.05)
    A = (rng.uniform(size=(n, n)) < P).astype(np.float64)
    A = np.triu(A, 1)
    A = A + A.T
    plan = ml.ml_dense_plan_matrix(dev(A), prec="f64")
    V = torch.empty(k * n, dtype=torch.float64, device="cuda")
    lam, nconv, st = ml.ml_lanczos_eigs([plan], k, p=1.0, tol=1e-11, seed=4, evecs=V)
    lam_ref, V_ref = eigen.smallest_eigs(graph.L_sym_from_W(A), k + 2)
    assert np.abs(lam - lam_ref[:k]).max() <= 1e-8
    # the Fiedler vector separates the two blocks
    f = V.cpu().numpy().reshape(k, n)[1]
    agree = np.mean((f > 0) == (blocks == blocks[np.argmax(np.abs(f))] ))
    assert max(agree, 1 - agree) >= 0.95


def test_dense_argument_errors():
    X = workloads.uniform_cube(10, 3, seed=54)
    with pytest.raises(ml.MLError):
        ml.ml_dense_plan(dev(X), -1.0)
    with pytest.raises(ml.MLError):
        ml.ml_dense_plan(dev(X[:1]), 0.1)
