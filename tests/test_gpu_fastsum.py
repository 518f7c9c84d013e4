"""GPU parity of the fast summation (Alg. 1 + the D^{-1/2} epilogue of Eq. I-L_1)
against the CPU oracle, through the C ABI.

Tolerances: the FP64 form must reach relative 2-norm error <= 1e-6 and the
FP32 form <= 1e-4 against the exact direct sum (the accuracy targets of the
two forms); against the oracle's Alg. 1 with exact Fourier sums, which shares
the bandwidth N and the kernel's Fourier coefficients, the FP64 form with the
widest window (m = 8) must agree to E_inf = ||y - y*||_inf / ||v||_1 <= 1e-11,
which isolates the window / grid / interpolation machinery from the K_RF
truncation.
"""
import numpy as np
import pytest
import torch

from oracle import alg1, graph
from paper_2007_05239_gb300 import _lib as ml
from paper_2007_05239_gb300 import workloads

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-6, "f32": 1e-4}


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def rel2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def check_errors(got, ref, v, tol, what=""):
    """The relative 2-norm error E2 and two element-wise measures, each within
    the form's target: E_inf = ||y - y*||_inf / (K(0) ||v||_1) (the usual
    fast-summation measure, K(0) = 1) and the largest entry error relative to
    the largest entry, max |y - y*| / max |y*|.  A localised error on a few
    entries that the 2-norm averages away fails the element-wise gates."""
    got, ref, v = np.asarray(got), np.asarray(ref), np.asarray(v)
    e2 = rel2(got, ref)
    err = np.abs(got - ref)
    einf = float(err.max() / np.abs(v).sum())
    emax = float(err.max() / np.abs(ref).max())
    assert e2 <= tol and einf <= tol and emax <= tol, f"{what}: E2 {e2:.3e} E_inf {einf:.3e} Emax {emax:.3e}"


def clustered(n, d, seed, k=5, spread=0.02):
    rng = np.random.default_rng(seed)
    mu = rng.uniform(0, 1, size=(k, d))
    lab = rng.integers(0, k, size=n)
    return mu[lab] + spread * rng.standard_normal((n, d))


def W_gpu(X, sigma, v, prec, **kw):
    plan = ml.ml_fastsum_plan(dev(X), sigma, prec=prec, **kw)
    V = dev(v.reshape(len(v), -1))
    Y = torch.empty_like(V)
    ml.ml_fastsum_apply([plan], V, Y, mode="raw")
    torch.cuda.synchronize()
    return Y.cpu().numpy().reshape(v.shape), plan


CASES = [
    ("cube3", lambda: workloads.uniform_cube(3001, 3, seed=31), 0.1),
    ("clust3", lambda: clustered(2777, 3, 32), 0.15),
    ("clust2", lambda: clustered(2500, 2, 33), 0.08),
    ("line1", lambda: workloads.uniform_cube(1713, 1, half=1.0, seed=34), 0.05),
]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("name,gen,sigma", CASES, ids=[c[0] for c in CASES])
def test_raw_W_matches_direct_sum(name, gen, sigma, prec):
    X = gen()
    rng = np.random.default_rng(5)
    for v in (np.ones(X.shape[0]), rng.uniform(0, 1, X.shape[0])):
        got, plan = W_gpu(X, sigma, v, prec)
        ref = graph.W_apply(X, sigma, v)
        check_errors(got, ref, v, TOL[prec], f"{name} {prec} {plan.info}")


@pytest.mark.parametrize("d", [1, 2, 3])
def test_matches_alg1_oracle_tightly(d):
    # Same bandwidth and the same box-domain scaling (isotropic map) on both sides;
    # the widest window makes the NFFT error negligible.
    n = {1: 900, 2: 1200, 3: 1500}[d]
    X = workloads.uniform_cube(n, d, seed=40 + d)
    sigma, N, target = 0.12, {1: 32, 2: 24, 3: 20}[d], 1e-12
    v = np.random.default_rng(6).uniform(-1, 1, n)
    got, plan = W_gpu(X, sigma, v, "f64", N=N, m=8, target_rel_err=target)
    Xs, ss, c, s = alg1.scale_to_domain(X, sigma, eps_B=0.0, eps_wrap=0.1 * target)
    info = plan.info
    assert abs(info["sigma_s"] - ss) <= 1e-14 * ss
    ref = alg1.fastsum_W(Xs, v, alg1.bhat(ss, N, d))
    # v has mixed signs, so measure against ||v||_1 (the usual fast-summation
    # error measure E_inf = ||y - y*||_inf / ||v||_1)
    e = float(np.abs(got - ref).max() / np.abs(v).sum())
    assert e <= 1e-11, f"d={d}: E_inf {e:.3e}"


@pytest.mark.parametrize("eps_B,p_reg", [(0.0, 0), (1.0 / 16, 4)])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_bhat_table_matches_oracle(d, eps_B, p_reg):
    X = workloads.uniform_cube(500, d, seed=50 + d)
    sigma, N = 0.3, 16
    plan = ml.ml_fastsum_plan(dev(X), sigma, N=N, m=4, eps_B=eps_B, p_reg=p_reg, prec="f64")
    Xs, ss, _, _ = alg1.scale_to_domain(X, sigma, eps_B=eps_B, eps_wrap=0.1 * 1e-6)
    ref = alg1.bhat(ss, N, d, eps_B, p_reg)
    # the table holds l = 0..N/2 per dim with dim 0 fastest; the oracle's
    # array is indexed [l_0 + N/2, ..., l_{d-1} + N/2].  l = N/2 is not in I_N;
    # by evenness b_{N/2} = b_{-N/2} (oracle index 0).
    H = N // 2 + 1
    got = plan.table(0).reshape((H,) * d)
    idx = np.arange(H)
    src = np.where(idx == N // 2, 0, N // 2 + idx)  # l = N/2 -> index 0 (l = -N/2)
    ref_full = ref[np.ix_(*([src] * d))]
    if d > 1:
        ref_full = np.transpose(ref_full)
    assert np.abs(got - ref_full).max() <= 1e-13 * np.abs(ref_full).max()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_degrees_and_normalised_multilayer(prec):
    n = 4003
    rng = np.random.default_rng(7)
    layers = [clustered(n, 3, 61), workloads.uniform_cube(n, 2, seed=62), clustered(n, 1, 63, spread=0.05)]
    sig = [0.15, 0.1, 0.05]
    plans = [ml.ml_fastsum_plan(dev(L), s, prec=prec) for L, s in zip(layers, sig)]
    for p, L, s in zip(plans, layers, sig):
        assert rel2(p.table(2), graph.degrees(L, s)) <= TOL[prec]
    v = rng.uniform(0, 1, n)
    Y = torch.empty(n, 1, dtype=torch.float64, device="cuda")
    ml.ml_fastsum_apply(plans, dev(v[:, None]), Y, mode="normalized")
    ref = graph.multilayer_A_apply(layers, sig, v)
    check_errors(Y.cpu().numpy()[:, 0], ref, v, TOL[prec], "normalised")
    # degree mode = mean degree
    ml.ml_fastsum_apply(plans, None, Y, mode="degree")
    ref = sum(graph.degrees(L, s) for L, s in zip(layers, sig)) / 3
    check_errors(Y.cpu().numpy()[:, 0], ref, np.ones(n), TOL[prec], "degrees")


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_multivector_passes_match_single(prec):
    n = 3100
    X = clustered(n, 3, 70)
    plan = ml.ml_fastsum_plan(dev(X), 0.12, prec=prec)
    V = np.random.default_rng(8).uniform(-1, 1, (n, 13))   # passes of 8, 4, 1
    Yb = torch.empty(n, 13, dtype=torch.float64, device="cuda")
    ml.ml_fastsum_apply([plan], dev(V), Yb, mode="normalized")
    Yb = Yb.cpu().numpy()
    for c in range(13):
        y1 = torch.empty(n, 1, dtype=torch.float64, device="cuda")
        ml.ml_fastsum_apply([plan], dev(V[:, c:c + 1]), y1, mode="normalized")
        y1 = y1.cpu().numpy()[:, 0]
        if prec == "f32":
            assert np.array_equal(Yb[:, c], y1)   # fixed-point spreading: order-free
        else:
            assert np.abs(Yb[:, c] - y1).max() <= 1e-13 * np.abs(y1).max()


def test_per_layer_mode():
    n = 2048
    layers = [workloads.uniform_cube(n, 2, seed=80 + t) for t in range(3)]
    plans = [ml.ml_fastsum_plan(dev(L), 0.1, prec="f64") for L in layers]
    X = np.random.default_rng(9).uniform(0, 1, (3, n, 2))
    Y = torch.empty(3, n, 2, dtype=torch.float64, device="cuda")
    ml.ml_fastsum_apply(plans, dev(X), Y, mode="normalized", per_layer=True)
    Y = Y.cpu().numpy()
    for t in range(3):
        ref = graph.A_apply(layers[t], 0.1, X[t])
        assert rel2(Y[t], ref) <= 1e-6


def test_f32_is_deterministic():
    X = clustered(5000, 3, 90)
    plan = ml.ml_fastsum_plan(dev(X), 0.1, prec="f32")
    V = dev(np.random.default_rng(10).uniform(-1, 1, (5000, 1)))
    Y1, Y2 = torch.empty_like(V), torch.empty_like(V)
    ml.ml_fastsum_apply([plan], V, Y1, mode="normalized")
    ml.ml_fastsum_apply([plan], V, Y2, mode="normalized")
    assert torch.equal(Y1, Y2)


def test_host_buffers_match_device():
    X = workloads.uniform_cube(2500, 3, seed=91)
    plan = ml.ml_fastsum_plan(dev(X), 0.1, prec="f32")
    v = np.random.default_rng(11).uniform(0, 1, (2500, 1))
    Yd = torch.empty(2500, 1, dtype=torch.float64, device="cuda")
    ml.ml_fastsum_apply([plan], dev(v), Yd, mode="normalized")
    Yh = np.empty((2500, 1))
    ml.ml_fastsum_apply([plan], v.copy(), Yh, mode="normalized")
    assert np.array_equal(Yd.cpu().numpy(), Yh)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_plans_from_host_points_match_device(prec):
    # host point arrays (numpy, pinned torch) are copied by the plan call; the
    # plans then equal those made from device points, bit for bit
    layers = [workloads.uniform_cube(3000, 3, seed=92), workloads.uniform_cube(3000, 2, seed=93)]
    pd = [ml.ml_fastsum_plan(dev(L), 0.1, prec=prec) for L in layers]
    ph = [ml.ml_fastsum_plan(L.copy(), 0.1, prec=prec) for L in layers]
    pm = ml.ml_fastsum_plan_many([torch.as_tensor(L).pin_memory() for L in layers], [0.1, 0.1], prec=prec)
    v = dev(np.random.default_rng(12).uniform(0, 1, (3000, 2)))
    ref = torch.empty_like(v)
    ml.ml_fastsum_apply(pd, v, ref, mode="normalized")
    for plans in (ph, pm):
        got = torch.empty_like(v)
        ml.ml_fastsum_apply(plans, v, got, mode="normalized")
        assert torch.equal(got, ref)
        for a, b in zip(plans, pd):
            assert np.array_equal(a.table(2), b.table(2))     # degrees


# ------------------------------------------------------------ edge cases
def test_two_points_closed_form():
    X = np.array([[0.0, 0.0, 0.0], [0.05, 0.0, 0.0]])
    sigma = 0.1
    w = np.exp(-0.25)
    got, _ = W_gpu(X, sigma, np.array([2.0, -3.0]), "f64")
    assert rel2(got, [-3 * w, 2 * w]) <= 1e-6


def test_identical_points():
    # all distances zero: W = 11^T - I, degrees n - 1
    X = np.full((257, 2), 0.3)
    got, plan = W_gpu(X, 0.5, np.ones(257), "f64")
    assert np.allclose(got, 256.0, rtol=1e-6)


def test_degenerate_flat_cloud_in_3d():
    # points on a line inside R^3 (one active extent per dim is a single cell)
    t = np.linspace(0, 1, 1500)
    X = np.stack([t, 0.5 * t, np.zeros_like(t)], axis=1)
    v = np.random.default_rng(12).uniform(0, 1, 1500)
    got, _ = W_gpu(X, 0.05, v, "f64")
    assert rel2(got, graph.W_apply(X, 0.05, v)) <= 1e-6


def test_heavy_bin_many_subproblems():
    # 20000 points inside one grid cell's neighbourhood: one bin, many subproblems
    rng = np.random.default_rng(13)
    X = np.concatenate([0.5 + 1e-3 * rng.standard_normal((20000, 3)), rng.uniform(0, 1, (500, 3))])
    v = rng.uniform(0, 1, X.shape[0])
    for prec in ("f64", "f32"):
        got, plan = W_gpu(X, 0.2, v, prec)
        assert plan.info["nsub"] > 10
        assert rel2(got, graph.W_apply(X, 0.2, v)) <= TOL[prec]


def test_domain_error_for_unreachable_bandwidth():
    X = workloads.uniform_cube(100, 3, seed=14)
    with pytest.raises(ml.MLError) as e:
        ml.ml_fastsum_plan(dev(X), 1e-4, prec="f64")
    assert e.value.status == ml.ML_ERR_DOMAIN


@pytest.mark.parametrize("b", [1, 8])
def test_batched_small_grid_layers(b):
    # FP32 layers whose grids are single tiles run as one batch (one launch per
    # stage, layer sum in registers); compare with the oracle and with the
    # per-layer mode (launched layer by layer) summed on the host.
    n = 5000
    layers, _ = workloads.gmm_band_layers(n, 8, 4, seed=15)
    sig = [0.5 * float((L.max(0) - L.min(0)).max()) for L in layers]
    plans = [ml.ml_fastsum_plan(dev(L), s, prec="f32") for L, s in zip(layers, sig)]
    assert all(p.info["nbins"] == 1 for p in plans)
    X = np.random.default_rng(16).uniform(0, 1, (n, b))
    Y = torch.empty(n, b, dtype=torch.float64, device="cuda")
    ml.ml_fastsum_apply(plans, dev(X), Y, mode="normalized")
    Y = Y.cpu().numpy()
    ref = graph.multilayer_A_apply(layers, sig, X)
    assert rel2(Y, ref) <= 1e-4
    T = len(layers)
    Yp = torch.empty(T, n, b, dtype=torch.float64, device="cuda")
    ml.ml_fastsum_apply(plans, dev(np.broadcast_to(X, (T, n, b))), Yp, mode="normalized", per_layer=True)
    assert rel2(Y, Yp.cpu().numpy().mean(axis=0)) <= 2e-6


def test_isolated_point_degree_error_only_for_normalised_products():
    # a far isolated point: its exact degree underflows, the FP32 approximation
    # may return <= 0; raw products must still work, normalised ones report it
    rng = np.random.default_rng(17)
    X = np.concatenate([rng.uniform(0, 0.6, (3000, 2)), [[1.0, 1.0]]])   # >= 11 sigma from the rest
    plan = ml.ml_fastsum_plan(dev(X), 0.05, prec="f32")
    V = dev(np.ones((X.shape[0], 1)))
    Y = torch.empty_like(V)
    ml.ml_fastsum_apply([plan], V, Y, mode="raw")
    if plan.info["deg_min"] <= 0:
        with pytest.raises(ml.MLError) as e:
            ml.ml_fastsum_apply([plan], V, Y, mode="normalized")
        assert e.value.status == ml.ML_ERR_DEGREE


def test_more_tile_groups_than_a_grid_dimension():
    # a narrow kernel in a 3-D cloud at oversampling 3 spreads 158k points over
    # more than 65,535 tiles: the tile sums must not depend on gridDim.y
    X, sigma = workloads.cloud_for_mlp(17)
    n = X.shape[0]
    plan = ml.ml_fastsum_plan_ex(torch.as_tensor(X, device="cuda"), sigma, taps=8, oversampling=3.0, prec="f64",
                                 target_rel_err=1e-6)
    assert plan.info["nsub"] > 65535
    v = np.random.default_rng(9).uniform(0, 1, n)
    Y = torch.empty(n, 1, dtype=torch.float64, device="cuda")
    ml.ml_fastsum_apply([plan], torch.as_tensor(v[:, None].copy(), device="cuda"), Y, mode="raw")
    rows = np.sort(np.random.default_rng(10).choice(n, 300, replace=False))
    ref = graph.W_apply(X, sigma, v, rows=rows)
    got = Y.cpu().numpy()[rows, 0]
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-6


def test_plan_many_equals_single_plans():
    # concurrent set-up of several layers gives the same plans as one at a time
    layers, _ = workloads.gmm_band_layers(20000, 16, 4, seed=60)
    sig = [0.5 * float((L.max(0) - L.min(0)).max()) for L in layers]
    dl = [torch.as_tensor(L, device="cuda") for L in layers]
    many = ml.ml_fastsum_plan_many(dl, sig, prec="f32")
    single = [ml.ml_fastsum_plan(x, s, prec="f32") for x, s in zip(dl, sig)]
    v = torch.as_tensor(np.random.default_rng(61).uniform(0, 1, (20000, 1)), device="cuda")
    for a, b in zip(many, single):
        ia, ib = a.info, b.info
        for key in ("N", "taps", "n_os", "bin", "nsub", "deg_min", "deg_max"):
            assert ia[key] == ib[key], key
        Ya, Yb = torch.empty_like(v), torch.empty_like(v)
        ml.ml_fastsum_apply([a], v, Ya, mode="normalized")
        ml.ml_fastsum_apply([b], v, Yb, mode="normalized")
        assert torch.equal(Ya, Yb)


def test_concurrent_layer_terms_equal_sequential():
    # with kernel timing off the layers' terms run on concurrent streams and
    # are summed in layer order; with it on they accumulate one after another:
    # the same FP64 additions, so the same bits
    layers = workloads.image_voronoi_layers(120, 150, 6, 0.02, seed=62)
    n = layers[0].shape[0]
    plans = [ml.ml_fastsum_plan(torch.as_tensor(L, device="cuda"), 0.2, prec="f64") for L in layers]
    X = torch.as_tensor(np.random.default_rng(63).uniform(-1, 1, (n, 4)), device="cuda")
    out = []
    for prof in (True, False):
        ml.ml_profile_enable(prof)
        Y = torch.empty_like(X)
        ml.ml_fastsum_apply(plans, X, Y, mode="normalized")
        ml.ml_profile_enable(False)
        out.append(Y.cpu())
    assert torch.equal(out[0], out[1])


def test_plans_reuse_cached_device_blocks():
    # a plan destroyed leaves its large blocks in the library's cache; the next
    # plan of the same size takes them (no new device memory), and releasing
    # the cache gives the memory back to the driver
    X = dev(workloads.uniform_cube(400_000, 3, seed=71))
    ml.ml_release_cached_memory()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    p = ml.ml_fastsum_plan(X, 0.05, prec="f32")
    owned = p.info["device_bytes"]
    p.destroy()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free0 - free1 >= owned // 2          # the blocks stay reserved by the cache
    q = ml.ml_fastsum_plan(X, 0.05, prec="f32")
    torch.cuda.synchronize()
    free2, _ = torch.cuda.mem_get_info()
    assert free2 >= free1 - (64 << 20)          # the new plan was served from the cache
    q.destroy()
    ml.ml_release_cached_memory()
    torch.cuda.synchronize()
    free3, _ = torch.cuda.mem_get_info()
    assert free3 >= free0 - (64 << 20)
