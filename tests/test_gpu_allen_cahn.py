"""GPU parity of the multiclass multilayer graph Allen-Cahn scheme (Alg. 2,
steps 2-4) against the FP64 oracle on the same eigenpairs: scores within
1e-10, the same iteration count, identical class predictions where the top
score is unique."""
import numpy as np
import pytest
import torch

from oracle import allen_cahn as oac
from oracle import eigen
from paper_2007_05239_gb300 import _lib as ml
from paper_2007_05239_gb300 import workloads

pytestmark = pytest.mark.gpu

PAPER = dict(eps=0.005, omega0=1000.0, dt=0.01)   # the image experiments' parameters (Sec. 8)


def run_both(Phi, lam, labels, m, tol, max_iter, **prm):
    n, k = Phi.shape
    dPhi = torch.as_tensor(np.ascontiguousarray(Phi.T).ravel(), device="cuda")   # column-major
    dlab = torch.as_tensor(labels.astype(np.int32), device="cuda")
    c = prm["omega0"] + 3.0 / prm["eps"]
    U, pred, it, chg = ml.ml_allen_cahn(dPhi, lam, dlab, m, eps=prm["eps"], omega0=prm["omega0"], c=c,
                                        dt=prm["dt"], tol=tol, max_iter=max_iter)
    Ur, itr, chr_ = oac.allen_cahn(Phi, lam, labels, m, prm["eps"], prm["omega0"], c, prm["dt"], tol, max_iter)
    return U.cpu().numpy().reshape(n, m), pred.cpu().numpy(), it, chg, Ur, itr, chr_


def check(U, pred, it, chg, Ur, itr, chr_):
    assert it == itr
    assert np.abs(U - Ur).max() <= 1e-10
    assert abs(chg - chr_[-1]) <= 1e-10 * max(1.0, chr_[-1])
    top = np.sort(Ur, axis=1)
    unique = top[:, -1] - top[:, -2] > 1e-9
    assert (pred[unique] == oac.predict(Ur)[unique]).all()


@pytest.mark.parametrize("m,seed", [(3, 1), (5, 2), (2, 3)])
def test_scores_match_oracle_on_dense_eigenpairs(m, seed):
    n = 900
    layers, truth = workloads.image_voronoi_layers(30, 30, m, 0.02, seed=seed, return_labels=True)
    sig = [0.2, 0.2, 0.2]
    lam, Phi = eigen.L1_eigs(layers, sig, 10)
    labels = workloads.known_labels(truth, 0.05, seed)
    for tol, max_iter in ((1e-6, 300), (0.0, 7), (0.0, 1)):
        check(*run_both(Phi, lam, labels, m, tol, max_iter, **PAPER))


def test_end_to_end_segmentation_from_gpu_eigenpairs():
    # GPU plans and Lanczos eigenpairs of L_1 for a small image, then Alg. 2;
    # the oracle runs the scheme on the GPU's eigenpairs
    h, w, m, k = 60, 80, 4, 12
    layers, truth = workloads.image_voronoi_layers(h, w, m, 0.02, seed=7, return_labels=True)
    n = h * w
    plans = [ml.ml_fastsum_plan(torch.as_tensor(L, device="cuda"), 0.2, prec="f64") for L in layers]
    V = torch.empty(n * k, dtype=torch.float64, device="cuda")
    lam, nconv, st = ml.ml_lanczos_eigs(plans, k, p=1.0, tol=1e-8, seed=3, evecs=V)
    assert st == ml.ML_OK
    Phi = V.cpu().numpy().reshape(k, n).T
    labels = workloads.known_labels(truth, 0.04, 11)
    U, pred, it, chg, Ur, itr, chr_ = run_both(Phi, lam, labels, m, 1e-6, 500, **PAPER)
    check(U, pred, it, chg, Ur, itr, chr_)
    # labelled nodes keep their class; the segmentation is far better than chance
    lab = labels >= 0
    assert (pred[lab] == labels[lab]).mean() >= 0.95
    assert (pred == truth).mean() >= 0.6


def test_argument_errors():
    Phi = torch.zeros(10 * 2, dtype=torch.float64, device="cuda")
    bad = torch.as_tensor(np.array([0, 1, 5, -1, 0, 0, 0, 0, 0, 0], dtype=np.int32), device="cuda")
    with pytest.raises(ml.MLError):
        ml.ml_allen_cahn(Phi, np.array([0.0, 0.1]), bad, 3)
    ok = torch.zeros(10, dtype=torch.int32, device="cuda")
    with pytest.raises(ml.MLError):
        ml.ml_allen_cahn(Phi, np.array([0.0, 0.1]), ok, 17)
