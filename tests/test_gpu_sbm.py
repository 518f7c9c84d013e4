"""The stochastic-block-model example of Sec. 9 through the library.

Two layers of a two-class block model (50 nodes per class), the first
informative (p_in 0.7, p_out 0.3), the second pure noise (p_in = p_out = 0.5).
Dense layers are planned from the sampled adjacency matrices, the k = 2
smallest eigenpairs of the power mean Laplacian come from the Lanczos solver
(p = 1, and p = -20, the power of the paper's example), and Alg. 2 classifies
from them with the paper's parameters.  Each step is compared with the oracle:
eigenvalues within 1e-8 and eigenvector angles within 1e-6 of the dense
eigensolve, Allen-Cahn scores within 1e-10 of the oracle's scheme on the same
eigenpairs, the same iteration count and predictions.
"""
import numpy as np
import pytest
import torch

from oracle import allen_cahn as oac
from oracle import eigen, graph
from paper_2007_05239_gb300 import _lib as ml
from paper_2007_05239_gb300 import workloads

pytestmark = pytest.mark.gpu

AC = dict(eps=0.005, omega0=1000.0, dt=0.01, tol=1e-6, max_iter=300)   # Sec. 9


@pytest.mark.parametrize("p", [1.0, -20.0])
def test_block_model_example_matches_oracle(p):
    n, k, m = 100, 2, 2
    c = AC["omega0"] + 3.0 / AC["eps"]
    errs = []
    for g in range(6):
        Ws, truth = workloads.block_model_layers([50, 50], [0.7, 0.5], [0.3, 0.5], seed=900 + g)
        plans = [ml.ml_dense_plan_matrix(torch.as_tensor(W, device="cuda"), prec="f64") for W in Ws]
        V = torch.empty(k * n, dtype=torch.float64, device="cuda")
        lam, nconv, st = ml.ml_lanczos_eigs(plans, k, p=p, tol=1e-11, seed=g + 1, evecs=V)
        assert st == ml.ML_OK and nconv >= k
        lam_ref, Phi_ref = eigen.power_mean_eigs([graph.L_sym_from_W(W) for W in Ws], p, k + 2)
        assert np.abs(lam - lam_ref[:k]).max() <= 1e-8, (g, lam, lam_ref[:k])
        Phi = V.cpu().numpy().reshape(k, n).T
        for grp in eigen.eigen_groups(lam_ref, rel_gap=1e-6):
            if max(grp) < k:
                assert eigen.subspace_angle(Phi[:, grp], Phi_ref[:, grp]) <= 1e-6
        labels = workloads.known_labels(truth, 0.04, seed=1900 + g)
        dPhi = torch.as_tensor(np.ascontiguousarray(Phi.T).ravel(), device="cuda")   # column-major
        dlab = torch.as_tensor(labels.astype(np.int32), device="cuda")
        U, pred, it, _ = ml.ml_allen_cahn(dPhi, lam, dlab, m, eps=AC["eps"], omega0=AC["omega0"], c=c,
                                          dt=AC["dt"], tol=AC["tol"], max_iter=AC["max_iter"])
        Ur, itr, _ = oac.allen_cahn(Phi, lam, labels, m, AC["eps"], AC["omega0"], c, AC["dt"], AC["tol"],
                                    AC["max_iter"])
        U = U.cpu().numpy().reshape(n, m)
        pred = pred.cpu().numpy()
        assert it == itr
        assert np.abs(U - Ur).max() <= 1e-10
        top = np.sort(Ur, axis=1)
        unique = top[:, -1] - top[:, -2] > 1e-9
        assert (pred[unique] == oac.predict(Ur)[unique]).all()
        errs.append(float(np.mean(pred != truth)))
    # the informative layer carries the classes through the noise layer (the
    # paper prints 7.7 % for p = 1 and 1.8 % for p = -20 over 100 graphs)
    assert np.mean(errs) <= 0.10, errs
