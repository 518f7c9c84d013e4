"""GPU parity of the Lanczos eigensolver (Sec. 3) against dense eigensolves of
the oracle: eigenvalues within 1e-8, eigenvector (or, inside clusters of
near-degenerate eigenvalues, subspace) angles within 1e-6."""
import math

import numpy as np
import pytest
import torch

from oracle import eigen, graph
from paper_2007_05239_gb300 import _lib as ml
from paper_2007_05239_gb300 import workloads

pytestmark = pytest.mark.gpu


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def check_pairs(lam, V, lam_ref, V_ref, k, tol_val=1e-8, tol_ang=1e-6):
    assert np.abs(lam - lam_ref).max() <= tol_val, (lam, lam_ref)
    groups = eigen.eigen_groups(lam_ref, rel_gap=1e-6)
    for g in groups:
        if max(g) >= k:
            continue
        ang = eigen.subspace_angle(V[:, g], V_ref[:, g])
        assert ang <= tol_ang, (g, ang)


def test_single_layer_n2000_d3_k10():
    # the small FP64 workload: n = 2000 uniform in [-1/4,1/4]^3, sigma = 0.1
    X = workloads.uniform_cube(2000, 3, seed=1)
    sigma, k = 0.1, 10
    plan = ml.ml_fastsum_plan(dev(X), sigma, prec="f64", target_rel_err=1e-12)
    V = torch.empty(k * 2000, dtype=torch.float64, device="cuda")
    lam, nconv, st = ml.ml_lanczos_eigs([plan], k, p=1.0, tol=1e-11, seed=3, evecs=V)
    assert st == ml.ML_OK and nconv == k
    V = V.cpu().numpy().reshape(k, 2000).T
    lam_ref, V_ref = eigen.lsym_eigs(X, sigma, k + 3)
    check_pairs(lam, V, lam_ref[:k], V_ref[:, :k], k)
    assert abs(lam[0]) <= 1e-9
    v0 = np.sqrt(graph.degrees(X, sigma))
    assert abs(abs(V[:, 0] @ v0) / np.linalg.norm(v0) - 1) <= 1e-9


def test_multilayer_p1():
    n = 1500
    layers = [workloads.uniform_cube(n, 3, seed=100), workloads.uniform_cube(n, 2, seed=101)]
    sig = [0.1, 0.08]
    plans = [ml.ml_fastsum_plan(dev(L), s, prec="f64", target_rel_err=1e-12) for L, s in zip(layers, sig)]
    k = 8
    V = np.empty(k * n)
    lam, nconv, st = ml.ml_lanczos_eigs(plans, k, p=1.0, tol=1e-11, seed=5, evecs=V)   # host output
    assert st == ml.ML_OK
    lam_ref, V_ref = eigen.L1_eigs(layers, sig, k + 3)
    check_pairs(lam, V.reshape(k, n).T, lam_ref[:k], V_ref[:, :k], k)


def test_power_mean_p_minus_one():
    n = 800
    layers = [workloads.uniform_cube(n, 3, seed=110), workloads.uniform_cube(n, 2, seed=111)]
    sig = [0.1, 0.1]
    plans = [ml.ml_fastsum_plan(dev(L), s, prec="f64", target_rel_err=1e-12) for L, s in zip(layers, sig)]
    k = 6
    V = torch.empty(k * n, dtype=torch.float64, device="cuda")
    lam, nconv, st = ml.ml_lanczos_eigs(plans, k, p=-1.0, tol=1e-10, seed=7, evecs=V)
    assert st == ml.ML_OK
    lam_ref, V_ref = eigen.Lp_eigs(layers, sig, -1.0, k + 3)
    check_pairs(lam, V.cpu().numpy().reshape(k, n).T, lam_ref[:k], V_ref[:, :k], k, tol_val=1e-8, tol_ang=1e-6)
    # every eigenvalue of L_{-1,delta} is at least delta = log 2 (each shifted
    # layer term is >= delta I, and so is their harmonic mean)
    assert lam[0] >= math.log(2.0) - 1e-10


def test_argument_errors():
    X = workloads.uniform_cube(100, 3, seed=120)
    plan = ml.ml_fastsum_plan(dev(X), 0.1, prec="f64")
    for bad in (dict(k=0), dict(k=51), dict(k=3, p=2.0)):
        with pytest.raises(ml.MLError):
            ml.ml_lanczos_eigs([plan], **bad)


@pytest.mark.parametrize("p", [-10.0, -2.5])
def test_power_mean_general_p(p):
    # the paper's preferred p = -10 (integer power: tridiagonal solves) and a
    # fractional power (tridiagonal eigendecomposition), each layer term by
    # the Lanczos approximation of the matrix power
    n = 600
    layers = [workloads.uniform_cube(n, 3, seed=130), workloads.uniform_cube(n, 2, seed=131)]
    sig = [0.1, 0.1]
    plans = [ml.ml_fastsum_plan(dev(L), s, prec="f64", target_rel_err=1e-12) for L, s in zip(layers, sig)]
    k = 5
    V = torch.empty(k * n, dtype=torch.float64, device="cuda")
    lam, nconv, st = ml.ml_lanczos_eigs(plans, k, p=p, tol=1e-10, seed=7, evecs=V)
    assert st == ml.ML_OK
    lam_ref, V_ref = eigen.Lp_eigs(layers, sig, p, k + 3)
    check_pairs(lam, V.cpu().numpy().reshape(k, n).T, lam_ref[:k], V_ref[:, :k], k, tol_val=1e-8, tol_ang=1e-6)
    # every eigenvalue of L_{p,delta} is at least delta = log(1 + |p|)
    assert lam[0] >= math.log1p(abs(p)) - 1e-10


def test_graph_replay_matches_eager_launches():
    # with kernel timing on, every inner CG iteration launches eagerly; with
    # it off, the iterations replay a captured CUDA graph: same kernels, same
    # order, so the same eigenpairs and the same work counters
    n = 700
    layers = [workloads.uniform_cube(n, 3, seed=140), workloads.uniform_cube(n, 2, seed=141)]
    sig = [0.1, 0.1]
    out = []
    for prof in (True, False):
        plans = [ml.ml_fastsum_plan(dev(L), s, prec="f64", target_rel_err=1e-10) for L, s in zip(layers, sig)]
        replays0 = ml.ml_graph_replays()
        ml.ml_profile_enable(prof)
        V = torch.empty(4 * n, dtype=torch.float64, device="cuda")
        lam, nconv, st = ml.ml_lanczos_eigs(plans, 4, p=-1.0, tol=1e-9, seed=3, evecs=V)
        ml.ml_profile_enable(False)
        replays = ml.ml_graph_replays() - replays0
        assert (replays == 0) if prof else (replays > 0)   # eager while timing kernels, graphs otherwise
        out.append((lam, V.cpu().numpy(), [pl.info["applied_vectors"] for pl in plans]))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]


def test_same_plan_twice_at_p_minus_one():
    # T identical layers: L_{-1,delta} = L_sym + delta I (Eq. L_p_delta_power_p);
    # the two CG solves share one plan and must not run concurrently on it
    n = 800
    X = workloads.uniform_cube(n, 3, seed=150)
    plan = ml.ml_fastsum_plan(dev(X), 0.1, prec="f64", target_rel_err=1e-12)
    lam, nconv, st = ml.ml_lanczos_eigs([plan, plan], 4, p=-1.0, tol=1e-10, seed=5)
    lam_ref, _ = eigen.lsym_eigs(X, 0.1, 4)
    assert np.abs(lam - (lam_ref + math.log(2.0))).max() <= 1e-8
