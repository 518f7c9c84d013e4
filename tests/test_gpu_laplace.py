"""GPU parity of the Laplacian kernel exp(-||y||/sigma) of Sec. 4 in the fast
summation (Alg. 1 on the regularised kernel K_R plus the direct near-field
pass over ||x_i - x_j|| < eps_I) against the oracle's direct sums, through
the C ABI.

Tolerances are those of the Gaussian path: relative 2-norm error <= 1e-4 for
the FP32 form and <= 1e-6 for the FP64 form against the exact direct sum, for
v = 1 and v ~ U[0, 1], on the raw W v, the degrees and the normalised A v.
The plan's Fourier table must equal the oracle's b_l of the same K_R (same
N, eps_B, eps_I, degree) to 1e-10 absolute, K(0) = 1 (the two FP64 solves of
the inner polynomial's ill-conditioned system round differently at ~1e-12).
Eigenpairs of the FP64 form (near field in FP64): eigenvalues within 1e-8,
eigenvector or cluster-subspace angles within 1e-6, as for the Gaussian.
"""
import numpy as np
import pytest
import torch

from oracle import alg1, eigen, graph
from paper_2007_05239_gb300 import _lib as ml
from paper_2007_05239_gb300 import workloads

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-6, "f32": 1e-4}


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def rel2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def ball(n, d, seed, radius=1.0):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d))
    X /= np.linalg.norm(X, axis=1)[:, None]
    return radius * X * rng.random(n)[:, None] ** (1.0 / d)


def clustered(n, d, seed, k=6, spread=0.05):
    rng = np.random.default_rng(seed)
    mu = rng.uniform(0, 1, size=(k, d))
    return mu[rng.integers(0, k, size=n)] + spread * rng.standard_normal((n, d))


def plan_lap(X, sigma, prec, **kw):
    return ml.ml_fastsum_plan_ex(dev(X), sigma, prec=prec, kernel="laplace", **kw)


def apply(plans, V, mode):
    V2 = V.reshape(V.shape[0], -1)
    Y = torch.empty(V2.shape, dtype=torch.float64, device="cuda")
    ml.ml_fastsum_apply(plans, dev(V2), Y, mode=mode)
    torch.cuda.synchronize()
    return Y.cpu().numpy().reshape(V.shape)


# sizes span many near-field cells, cells with more than 128 points (several
# tasks per cell) and ragged last tasks
CASES = [
    ("ball3", lambda: ball(6001, 3, 41), 0.15),
    ("cube2", lambda: workloads.uniform_cube(20011, 2, seed=42), 0.05),
    ("clust2", lambda: clustered(5003, 2, 43), 0.1),
    ("line1", lambda: workloads.uniform_cube(3001, 1, half=1.0, seed=44), 0.05),
]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("name,gen,sigma", CASES, ids=[c[0] for c in CASES])
def test_raw_W_matches_direct_sum(name, gen, sigma, prec):
    X = gen()
    n = X.shape[0]
    plan = plan_lap(X, sigma, prec)
    info = plan.info
    assert info["kernel"] == ml.ML_KERNEL_LAPLACE and info["domain"] == 1
    assert 0 < info["kernel_err"] <= 0.5 * TOL[prec]
    assert info["near_pairs"] >= n   # every point meets itself
    rng = np.random.default_rng(5)
    for v in (np.ones(n), rng.random(n)):
        y = apply([plan], v, "raw")
        ref = graph.W_apply(X, sigma, v, kernel="laplace")
        assert rel2(y, ref) <= TOL[prec], (name, prec, rel2(y, ref), info["N"], info["eps_I"])


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_degrees_and_normalised(prec):
    X = ball(7000, 3, 45)
    sigma = 0.2
    plan = plan_lap(X, sigma, prec)
    deg_ref = graph.degrees(X, sigma, kernel="laplace")
    Y = torch.empty((X.shape[0], 1), dtype=torch.float64, device="cuda")
    ml.ml_fastsum_apply([plan], None, Y, mode="degree")
    torch.cuda.synchronize()
    assert rel2(Y.cpu().numpy()[:, 0], deg_ref) <= TOL[prec]
    v = np.random.default_rng(6).random(X.shape[0])
    y = apply([plan], v, "normalized")
    ref = graph.A_apply(X, sigma, v, deg=deg_ref, kernel="laplace")
    assert rel2(y, ref) <= TOL[prec]


@pytest.mark.parametrize("b", [8, 5])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_block_of_vectors(prec, b):
    X = workloads.uniform_cube(9000, 2, seed=46)
    sigma = 0.08
    plan = plan_lap(X, sigma, prec)
    V = np.random.default_rng(7).random((X.shape[0], b))
    Y = apply([plan], V, "raw")
    ref = graph.W_apply(X, sigma, V, kernel="laplace")
    for c in range(b):
        assert rel2(Y[:, c], ref[:, c]) <= TOL[prec]
    # a block equals its columns applied one at a time (same arithmetic per column
    # up to the pass width of the window sums)
    y0 = apply([plan], V[:, 0].copy(), "raw")
    assert rel2(Y[:, 0], y0) <= 0.1 * TOL[prec]


@pytest.mark.parametrize("d", [1, 2, 3])
def test_bhat_table_matches_oracle(d):
    X = ball(800, d, 50 + d)
    sigma, N, eps_I = 0.5, 32, 6.0 / 32
    plan = plan_lap(X, sigma, "f64", N=N, eps_I=eps_I, target_rel_err=1e-3)
    info = plan.info
    assert info["N"] == N and abs(info["eps_I"] - eps_I) < 1e-15
    eps_B, p = info["eps_B"], info["p_reg"]
    assert eps_B == max(1.0 / 16, eps_I) and p == 8
    ref = alg1.bhat(info["sigma_s"], N, d, eps_B, p, "laplace", eps_I)
    H = N // 2 + 1
    got = plan.table(0).reshape((H,) * d)
    idx = np.arange(H)
    src = np.where(idx == N // 2, 0, N // 2 + idx)
    ref_full = ref[np.ix_(*([src] * d))]
    if d > 1:
        ref_full = np.transpose(ref_full)
    # the inner polynomial comes from a Vandermonde-like system in powers of
    # eps_I up to 2p - 2; two different FP64 solvers give samples of K_R that
    # agree to ~1e-12 absolute (K(0) = 1), and the b_l inherit that
    assert np.abs(got - ref_full).max() <= 1e-10


def test_explicit_parameters_reported():
    X = ball(3000, 2, 55)
    plan = plan_lap(X, 0.3, "f64", N=128, eps_I=1.0 / 16, p_reg=6, target_rel_err=1e-4)
    info = plan.info
    assert info["N"] == 128 and info["eps_I"] == 1.0 / 16 and info["p_reg"] == 6
    assert info["eps_B"] == 1.0 / 16
    y = apply([plan], np.ones(3000), "raw")
    assert rel2(y, graph.degrees(X, 0.3, kernel="laplace")) <= 1e-4


def test_mixed_kernels_multilayer():
    # a Gaussian and a Laplacian layer of one node set, normalised multilayer
    # product (Eq. I-L_1): concurrent layer terms summed in layer order
    n = 5000
    A = ball(n, 3, 60)
    B = workloads.uniform_cube(n, 2, seed=61)
    pg = ml.ml_fastsum_plan(dev(A), 0.2, prec="f64")
    pl = plan_lap(B, 0.1, "f64")
    v = np.random.default_rng(8).random(n)
    y = apply([pg, pl], v, "normalized")
    ref = 0.5 * (graph.A_apply(A, 0.2, v) + graph.A_apply(B, 0.1, v, kernel="laplace"))
    assert rel2(y, ref) <= 1e-6


def test_eigenpairs_small_graph():
    n, k = 1800, 6
    X = ball(n, 3, 70)
    sigma = 0.3
    plan = plan_lap(X, sigma, "f64", target_rel_err=1e-8)
    V = torch.empty(k * n, dtype=torch.float64, device="cuda")
    lam, nconv, st = ml.ml_lanczos_eigs([plan], k, p=1.0, tol=1e-9, seed=3, evecs=V)
    assert st == ml.ML_OK and nconv == k
    V = V.cpu().numpy().reshape(k, n).T
    lam_ref, V_ref = eigen.lsym_eigs(X, sigma, k + 3, kernel="laplace")
    assert np.abs(lam - lam_ref[:k]).max() <= 1e-8, (lam, lam_ref[:k])
    for g in eigen.eigen_groups(lam_ref[:k + 3], rel_gap=1e-6):
        if max(g) >= k:
            continue
        assert eigen.subspace_angle(V[:, g], V_ref[:, g]) <= 1e-6


def test_power_mean_p_minus_one_mixed_kernels():
    # L_{-1,delta} of a Laplacian and a Gaussian layer: the inner CG solves
    # replay CUDA graphs that contain the near-field pass
    n, k = 700, 6
    A = ball(n, 3, 90)
    B = workloads.uniform_cube(n, 2, seed=91)
    pl = plan_lap(A, 0.4, "f64", target_rel_err=1e-8)
    pg = ml.ml_fastsum_plan(dev(B), 0.1, prec="f64", target_rel_err=1e-12)
    replays = ml.ml_graph_replays()
    V = torch.empty(k * n, dtype=torch.float64, device="cuda")
    lam, nconv, st = ml.ml_lanczos_eigs([pl, pg], k, p=-1.0, tol=1e-10, seed=7, evecs=V)
    assert st == ml.ML_OK and nconv == k
    assert ml.ml_graph_replays() > replays
    lam_ref, V_ref = eigen.Lp_eigs([A, B], [0.4, 0.1], -1.0, k + 3, kernel=["laplace", "gauss"])
    assert np.abs(lam - lam_ref[:k]).max() <= 1e-8, (lam, lam_ref[:k])
    V = V.cpu().numpy().reshape(k, n).T
    for g in eigen.eigen_groups(lam_ref[:k + 3], rel_gap=1e-6):
        if max(g) >= k:
            continue
        assert eigen.subspace_angle(V[:, g], V_ref[:, g]) <= 1e-6


@pytest.mark.parametrize("block", [1, 3])
def test_per_layer_block_lanczos(block):
    # every layer's L_sym at once (Laplacian layers run their own kernels)
    n, k = 900, 5
    layers = [ball(n, 3, 95), workloads.uniform_cube(n, 2, seed=96)]
    sig = [0.3, 0.1]
    plans = [plan_lap(L, s, "f64", target_rel_err=1e-8) for L, s in zip(layers, sig)]
    V = torch.empty(len(layers) * n * k, dtype=torch.float64, device="cuda")
    lam, nconv, st = ml.ml_lanczos_eigs_layers(plans, k, block=block, tol=1e-10, seed=11, evecs=V)
    assert st == ml.ML_OK and (nconv == k).all()
    V = V.cpu().numpy().reshape(len(layers), k, n)
    for t, (X, s) in enumerate(zip(layers, sig)):
        lam_ref, V_ref = eigen.lsym_eigs(X, s, k + 3, kernel="laplace")
        assert np.abs(lam[t] - lam_ref[:k]).max() <= 1e-8, (t, lam[t], lam_ref[:k])
        for g in eigen.eigen_groups(lam_ref, rel_gap=1e-6):
            if max(g) >= k:
                continue
            assert eigen.subspace_angle(V[t][g].T, V_ref[:, g]) <= 1e-6


def test_argument_errors():
    X = dev(ball(500, 2, 80))
    with pytest.raises(ml.MLError) as e:
        ml.ml_fastsum_plan_ex(X, 0.1, kernel=7)
    assert e.value.status == ml.ML_ERR_ARG
    with pytest.raises(ml.MLError) as e:
        ml.ml_fastsum_plan_ex(X, 0.1, kernel="gauss", eps_I=0.05)
    assert e.value.status == ml.ML_ERR_ARG
    with pytest.raises(ml.MLError) as e:
        ml.ml_fastsum_plan_ex(X, 0.1, kernel="laplace", eps_I=0.3)
    assert e.value.status == ml.ML_ERR_ARG
    with pytest.raises(ml.MLError) as e:
        ml.ml_fastsum_plan_ex(X, 0.1, kernel="laplace", target_rel_err=1e-11)
    assert e.value.status == ml.ML_ERR_DOMAIN
    # fixed N and eps_I that cannot reach the target: the plan's own check refuses
    with pytest.raises(ml.MLError) as e:
        ml.ml_fastsum_plan_ex(X, 0.1, kernel="laplace", N=16, eps_I=1.0 / 16, target_rel_err=1e-7)
    assert e.value.status == ml.ML_ERR_DOMAIN
