"""Pins for the CPU oracle: each check ties an oracle function to something
other than itself (a closed form, an identity of analysis, a library routine
on a special case, or an invariant), so that a dropped term, a wrong sign or
index, or a transposed operand fails one of them."""
import math
import os

import numpy as np
import pytest

from oracle import alg1, eigen, graph
from paper_2007_05239_gb300 import workloads


# ------------------------------------------------------------------ graph
def test_two_points_closed_form():
    # W = [[0, w], [w, 0]], w = exp(-r^2/sigma^2); L_sym = [[1,-1],[-1,1]].
    r, sigma = 0.3, 0.2
    X = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    w = math.exp(-r * r / sigma ** 2)
    out = graph.W_apply(X, sigma, np.array([2.0, -3.0]))
    assert np.allclose(out, [-3.0 * w, 2.0 * w], rtol=1e-15, atol=0)
    L = graph.L_sym_dense(X, sigma)
    assert np.allclose(L, [[1, -1], [-1, 1]], atol=1e-15)


def test_regular_tetrahedron_closed_form():
    # All pair distances equal (2 sqrt 2): W = w (11^T - I), deg = 3w,
    # spectrum of L_sym = {0, 4/3, 4/3, 4/3}.
    X = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=float)
    sigma = 2.5
    w = math.exp(-8.0 / sigma ** 2)
    assert np.allclose(graph.degrees(X, sigma), 3 * w, rtol=1e-15)
    lam, _ = eigen.lsym_eigs(X, sigma, 4)
    assert np.allclose(lam, [0, 4 / 3, 4 / 3, 4 / 3], atol=1e-14)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_lattice_degree_poisson_summation(d):
    # Centre of the lattice h*Z^d truncated to |k| <= M: by Poisson summation
    # sum_{k in Z^d} exp(-|k h|^2/sigma^2) = (sigma sqrt(pi)/h)^d (1 + 2 sum_l e^{-pi^2 sigma^2 l^2/h^2})^d.
    h, sigma, M = 1.0, 2.0, 10
    g = np.arange(-M, M + 1, dtype=float) * h
    X = np.stack(np.meshgrid(*([g] * d), indexing="ij"), axis=-1).reshape(-1, d)
    centre = int(np.argmin((X ** 2).sum(axis=1)))
    q = math.exp(-(math.pi * sigma / h) ** 2)
    theta = (sigma * math.sqrt(math.pi) / h) * (1 + 2 * sum(q ** (l * l) for l in range(1, 5)))
    expect = theta ** d - 1.0          # minus the excluded self term K(0) = 1
    got = graph.degrees(X, sigma, rows=np.array([centre]))[0]
    assert abs(got - expect) <= 1e-9 * expect


def test_sigma_infinity_limit():
    # W -> 11^T - I: A = W/(n-1) has eigenvalues 1 (once) and -1/(n-1).
    X = workloads.uniform_cube(40, 2, seed=7)
    n = X.shape[0]
    L = graph.L_sym_dense(X, 1e7)
    lam = np.linalg.eigvalsh(np.eye(n) - L)
    assert abs(lam[-1] - 1.0) < 1e-10
    assert np.allclose(lam[:-1], -1.0 / (n - 1), atol=1e-10)


def test_normalised_operator_invariants():
    X = workloads.uniform_cube(300, 3, seed=5)
    sigma = 0.1
    deg = graph.degrees(X, sigma)
    s = np.sqrt(deg)
    # A D^{1/2} 1 = D^{-1/2} W 1 = D^{1/2} 1
    assert np.allclose(graph.A_apply(X, sigma, s, deg), s, rtol=1e-12)
    L = graph.L_sym_dense(X, sigma)
    assert abs(np.trace(L) - X.shape[0]) < 1e-10          # trace A = 0
    # dense W against the C direct sum on a random vector
    v = np.random.default_rng(0).standard_normal(300)
    assert np.allclose(graph.weight_matrix(X, sigma) @ v, graph.W_apply(X, sigma, v), rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------ multilayer mean
def test_multilayer_two_point_layers_closed_form():
    # Every connected two-point layer has D^{-1/2} W D^{-1/2} = [[0, 1], [1, 0]]
    # whatever its weight w_t, so the mean over layers (Eq. I-L_1) swaps the two
    # entries of v exactly, while the raw mean (1/T) sum_t W_t scales the swap
    # by the mean weight.  A dropped 1/T, or W summed in place of the
    # normalised A, fails here.
    dists, sigmas = [0.1, 0.3, 0.5], [0.2, 0.25, 0.4]
    layers = [np.array([[0.0, 0.0], [r, 0.0]]) for r in dists]
    v = np.array([2.0, -3.0])
    got = graph.multilayer_A_apply(layers, sigmas, v)
    assert np.allclose(got, [-3.0, 2.0], rtol=1e-15, atol=0)
    wbar = np.mean([math.exp(-r * r / s ** 2) for r, s in zip(dists, sigmas)])
    got_w = graph.multilayer_W_apply(layers, sigmas, v)
    assert np.allclose(got_w, [-3.0 * wbar, 2.0 * wbar], rtol=1e-14, atol=0)


def test_multilayer_three_point_layers_closed_form():
    # Layer 1: three points on a line at 0, r, 2r: weights a = e^{-r^2/s^2}
    # (neighbours) and c = e^{-4r^2/s^2} (ends), degrees (a + c, 2a, a + c).
    # Layer 2: an equilateral triangle: D^{-1/2} W D^{-1/2} = (J - I)/2.
    r, s1 = 0.2, 0.3
    a, c = math.exp(-r * r / s1 ** 2), math.exp(-4 * r * r / s1 ** 2)
    line = np.array([[0.0, 0.0], [r, 0.0], [2 * r, 0.0]])
    tri = np.array([[0.0, 0.0], [1.0, 0.0], [0.5, math.sqrt(3) / 2]])
    x = math.sqrt(a / (2 * (a + c)))            # a / sqrt((a + c) 2a)
    A1 = np.array([[0, x, c / (a + c)], [x, 0, x], [c / (a + c), x, 0]])
    A2 = (np.ones((3, 3)) - np.eye(3)) / 2
    V = np.random.default_rng(1).standard_normal((3, 2))
    got = graph.multilayer_A_apply([line, tri], [s1, 0.7], V)
    assert np.allclose(got, (A1 + A2) @ V / 2, rtol=1e-13, atol=1e-15)
    w = math.exp(-1.0 / 0.49)
    W1 = np.array([[0, a, c], [a, 0, a], [c, a, 0]])
    W2 = w * (np.ones((3, 3)) - np.eye(3))
    got_w = graph.multilayer_W_apply([line, tri], [s1, 0.7], V)
    assert np.allclose(got_w, (W1 + W2) @ V / 2, rtol=1e-13, atol=1e-15)


def test_multilayer_identical_layers_and_order():
    # T copies of one layer give that layer's operator; the mean does not
    # depend on the order of the layers; W applied to ones is the mean of the
    # layers' degrees.
    X = workloads.uniform_cube(250, 3, seed=21)
    Y = workloads.uniform_cube(250, 2, seed=22)
    V = np.random.default_rng(2).standard_normal((250, 3))
    one = graph.A_apply(X, 0.12, V)
    assert np.allclose(graph.multilayer_A_apply([X] * 4, [0.12] * 4, V), one, rtol=1e-13, atol=1e-14)
    assert np.allclose(graph.multilayer_W_apply([X] * 3, [0.12] * 3, V), graph.W_apply(X, 0.12, V),
                       rtol=1e-13, atol=1e-14)
    ab = graph.multilayer_A_apply([X, Y], [0.12, 0.2], V)
    ba = graph.multilayer_A_apply([Y, X], [0.2, 0.12], V)
    assert np.allclose(ab, ba, rtol=1e-14, atol=1e-15)
    dmean = graph.multilayer_W_apply([X, Y], [0.12, 0.2], np.ones(250))
    assert np.allclose(dmean, (graph.degrees(X, 0.12) + graph.degrees(Y, 0.2)) / 2, rtol=1e-14)


def test_multilayer_mean_matches_dense_L1():
    # The product with the identity is the dense I - L_1 (numpy weight matrices,
    # a code path separate from the C direct sum); its spectrum is that of
    # eigen.L1_eigs; it is symmetric with zero trace (no self-edges), and every
    # eigenvalue of I - L_1 lies in [-1, 1] (each layer's lies there).
    X = workloads.uniform_cube(120, 3, seed=23)
    Y = workloads.uniform_cube(120, 1, seed=24)
    M = np.hstack([graph.multilayer_A_apply([X, Y], [0.1, 0.05], E) for E in np.split(np.eye(120), 8, axis=1)])
    dense = (2 * np.eye(120) - graph.L_sym_dense(X, 0.1) - graph.L_sym_dense(Y, 0.05)) / 2
    assert np.abs(M - dense).max() <= 1e-13
    assert np.abs(M - M.T).max() <= 1e-14 and abs(np.trace(M)) <= 1e-12
    theta = np.linalg.eigvalsh(0.5 * (M + M.T))
    assert theta.min() >= -1 - 1e-12 and theta.max() <= 1 + 1e-12
    lam, _ = eigen.L1_eigs([X, Y], [0.1, 0.05], 8)
    assert np.allclose(np.sort(1 - theta)[:8], lam, atol=1e-12)


def test_spectrum_bounds_and_null_vector():
    X = workloads.uniform_cube(200, 3, seed=3)
    sigma = 0.1
    lam, Phi = eigen.lsym_eigs(X, sigma, 200)
    assert lam.min() > -1e-12 and lam.max() < 2 + 1e-12
    assert abs(lam[0]) < 1e-12
    assert abs(lam.sum() - 200) < 1e-9
    v0 = np.sqrt(graph.degrees(X, sigma))
    v0 /= np.linalg.norm(v0)
    assert abs(abs(Phi[:, 0] @ v0) - 1) < 1e-10


def test_jacobi_matches_lapack():
    X = workloads.uniform_cube(60, 3, seed=11)
    L = graph.L_sym_dense(X, 0.12)
    lj, Vj = eigen.jacobi_eigh(L)
    le, Ve = np.linalg.eigh(L)
    assert np.allclose(lj, le, atol=1e-12)
    # eigenvector check through residuals (independent of sign/order ties)
    assert np.abs(L @ Vj - Vj * lj[None, :]).max() < 1e-11
    # closed 2x2 case
    lam, _ = eigen.jacobi_eigh(np.array([[2.0, 1.0], [1.0, 2.0]]))
    assert np.allclose(lam, [1.0, 3.0], atol=1e-15)


def test_power_mean_identical_layers():
    # T identical layers: L_{p,delta} = L_sym + delta I for every p; p=1 gives L_sym.
    X = workloads.uniform_cube(80, 2, seed=4)
    lam, _ = eigen.lsym_eigs(X, 0.15, 6)
    lp, _ = eigen.Lp_eigs([X, X, X], [0.15] * 3, -1.0, 6)
    assert np.allclose(lp, lam + math.log(2.0), atol=1e-10)
    l1, _ = eigen.L1_eigs([X, X], [0.15] * 2, 6)
    assert np.allclose(l1, lam, atol=1e-12)


def test_power_mean_two_commuting_layers():
    # Any connected 2-node graph has L_sym = [[1,-1],[-1,1]] with spectrum {0, 2},
    # whatever its weight; so two such layers give L_{-1,delta} = L_sym + delta I
    # with eigenvalues {delta, 2 + delta}, delta = log 2.
    X = np.array([[0.0], [0.3]])
    lp, _ = eigen.Lp_eigs([X, X * 2], [0.2, 0.5], -1.0, 2)
    assert np.allclose(lp, [math.log(2), 2 + math.log(2)], atol=1e-12)


@pytest.mark.parametrize("p", [10.0, 2.0, 1.0, -1.0, -20.0])
def test_power_mean_of_commuting_layers_is_the_scalar_power_mean(p):
    # Two symmetric layers with a common eigenbasis Q and spectra a, b: the
    # power mean (Eq. power_mean_laplacian_shifted) has the same eigenvectors
    # and the eigenvalues ((a_i + delta)^p + (b_i + delta)^p)/2)^(1/p), delta =
    # log(1 + |p|) for p < 0 and 0 for p > 0 (Sec. 2); p = 1 is the plain mean.
    rng = np.random.default_rng(12)
    Q, _ = np.linalg.qr(rng.standard_normal((7, 7)))
    a = np.array([0.0, 0.3, 0.9, 1.4, 2.0, 0.05, 1.7])
    b = np.array([0.0, 1.1, 0.2, 1.9, 0.5, 0.6, 1.2])
    La, Lb = (Q * a) @ Q.T, (Q * b) @ Q.T
    delta = math.log1p(abs(p)) if p < 0 else 0.0
    mu = (((a + delta) ** p + (b + delta) ** p) / 2.0) ** (1.0 / p) if p != 1 else (a + b) / 2.0
    order = np.argsort(mu)
    k = 4
    lam, Phi = eigen.power_mean_eigs([La, Lb], p, k)
    ref = mu[order][:k]
    if p == 1:
        assert np.allclose(lam, ref, rtol=1e-10, atol=1e-12)
    else:
        # lambda^p is the mean of the shifted powers (well conditioned); lambda
        # itself is checked away from 0, where the p-th root of a rounding-level
        # eigenvalue is not (p > 0: (1e-17)^(1/p) is far from 0)
        scale = np.abs(ref ** p).max()
        assert np.allclose(lam ** p, ref ** p, rtol=1e-10, atol=1e-14 * scale)
        big = ref > 1e-3
        assert np.allclose(lam[big], ref[big], rtol=1e-10)
    for i in range(k):
        assert abs(abs(Phi[:, i] @ Q[:, order[i]]) - 1.0) <= 1e-8


# ------------------------------------------------------------------ Alg. 1
@pytest.mark.parametrize("d", [1, 2, 3])
def test_bhat_box_matches_poisson(d):
    # Samples of the 1-periodised Gaussian: by Poisson summation its Fourier
    # coefficients are c(j) = s sqrt(pi) exp(-pi^2 s^2 j^2), and sampling on
    # k/N aliases them: b_l = prod_a sum_r c(l_a + rN) exactly.  A wide s
    # makes the periodisation matter.
    s, N = 0.3, 16
    b = alg1.bhat(s, N, d)
    l = np.arange(-N // 2, N // 2)
    c1 = sum(s * math.sqrt(math.pi) * np.exp(-(math.pi * s * (l + r * N)) ** 2) for r in range(-3, 4))
    expect = c1
    for _ in range(d - 1):
        expect = np.multiply.outer(expect, c1)
    assert np.abs(b - expect).max() < 1e-14


def test_adjoint_ndft_on_grid_is_fft():
    # Nodes on the equispaced grid k/N: step 1 of Alg. 1 is a plain DFT.
    N = 8
    k = np.arange(-N // 2, N // 2)
    Xs = (np.stack(np.meshgrid(k, k, indexing="ij"), -1).reshape(-1, 2)) / N
    v = np.random.default_rng(1).standard_normal(Xs.shape[0])
    got = alg1.adjoint_ndft(Xs, v, N)
    V = v.reshape(N, N)
    F = np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(V)))
    assert np.allclose(got, F, atol=1e-12)
    # and step 3 is the inverse DFT times N^d
    back = alg1.ndft(Xs, F, N).reshape(N, N)
    assert np.allclose(back, N * N * V, atol=1e-9)


def _tail_bound(s, N, d, a=0.25):
    """Bound on max |K_RF - K| over differences of nodes in [-a, a]^d for the
    box reading: per dimension twice the Fourier tail beyond N/2 (truncation
    plus aliasing) and the wrap term 2 exp(-(1-2a)^2/s^2), times 3d."""
    tail = 2 * sum(s * math.sqrt(math.pi) * math.exp(-(math.pi * s * l) ** 2) for l in range(N // 2, N // 2 + 200))
    wrap = 2 * math.exp(-((1 - 2 * a) ** 2) / s ** 2)
    return 3 * d * (2 * tail + wrap)


@pytest.mark.parametrize("d,N", [(1, 32), (2, 24), (3, 16)])
def test_alg1_against_direct_sum(d, N):
    X = workloads.uniform_cube(400, d, seed=21)
    sigma = 0.12
    Xs, ss, _, _ = alg1.scale_to_domain(X, sigma, eps_B=0.0, eps_wrap=1e-12)
    assert np.abs(Xs).max() <= 0.25 + 1e-15
    v = np.random.default_rng(2).uniform(0, 1, X.shape[0])
    b = alg1.bhat(ss, N, d)
    got = alg1.fastsum_W(Xs, v, b)
    ref = graph.W_apply(X, sigma, v)
    bound = _tail_bound(ss, N, d, a=np.abs(Xs).max()) * np.abs(v).sum()
    err = np.abs(got - ref).max()
    assert err <= bound
    # a coarser bandwidth must be visibly worse (the comparison has teeth)
    b2 = alg1.bhat(ss, N // 2, d)
    err2 = np.abs(alg1.fastsum_W(Xs, v, b2) - ref).max()
    assert err2 > 10 * err


@pytest.mark.parametrize("d,N", [(2, 32), (3, 24)])
def test_alg1_ball_domain_against_direct_sum(d, N):
    # ball domain (eps_B = 1/16, K_R = K on every pair distance): Alg. 1 with
    # exact Fourier sums reproduces the direct sum of W v, and half the
    # bandwidth is visibly worse
    X = workloads.uniform_ball(400, d, radius=1.0, seed=22)
    sigma, eps_B = 0.5, 1.0 / 16
    Xs, ss, _, _ = alg1.scale_to_domain(X, sigma, eps_B=eps_B)
    assert np.linalg.norm(Xs, axis=1).max() <= 0.25 - eps_B / 2 + 1e-15
    v = np.random.default_rng(3).uniform(0, 1, X.shape[0])
    ref = graph.W_apply(X, sigma, v)
    err = np.abs(alg1.fastsum_W(Xs, v, alg1.bhat(ss, N, d, eps_B, 4)) - ref).max() / np.abs(v).sum()
    err2 = np.abs(alg1.fastsum_W(Xs, v, alg1.bhat(ss, N // 2, d, eps_B, 4)) - ref).max() / np.abs(v).sum()
    assert err <= 1e-9 and err2 >= 100 * err


@pytest.mark.parametrize("p", [1, 2, 4])
def test_regulariser_smoothness_sets_the_convergence_rate(p):
    # a wide kernel (K = 0.37 at the ball's edge) makes the outer regulariser
    # matter: K_R matches p derivatives, so its Fourier coefficients decay like
    # N^-(p+1) and the truncation error of Alg. 1 at least like N^-p; from
    # N = 64 to 256 it must fall by 4^p (a factor 2 of slack)
    X = workloads.uniform_cube(400, 1, seed=22)
    sigma, eps_B = 0.5, 1.0 / 16
    Xs, ss, _, _ = alg1.scale_to_domain(X, sigma, eps_B=eps_B)
    v = np.random.default_rng(3).uniform(0, 1, X.shape[0])
    ref = graph.W_apply(X, sigma, v)
    err = [np.abs(alg1.fastsum_W(Xs, v, alg1.bhat(ss, N, 1, eps_B, p)) - ref).max() / np.abs(v).sum()
           for N in (64, 256)]
    assert err[0] / err[1] >= 0.5 * 4.0 ** p, err


def test_regulariser_matching_conditions():
    sigma, eps_B, p = 0.3, 1.0 / 16, 4
    rI = 0.5 - eps_B
    q = alg1.regulariser_poly(sigma, eps_B, p)
    P = np.polynomial.Polynomial(q)
    dK = alg1._gauss_derivs(rI, sigma, p)
    # derivatives k at t=0 equal eps^k K^{(k)}(r_I) (finite differences of the
    # closed-form Gaussian as an independent check of _gauss_derivs)
    hstep = 1e-4
    fd1 = (math.exp(-(rI + hstep) ** 2 / sigma ** 2) - math.exp(-(rI - hstep) ** 2 / sigma ** 2)) / (2 * hstep)
    assert abs(fd1 - dK[1]) < 1e-7
    for k in range(p):
        assert abs(P.deriv(k)(0.0) - dK[k] * eps_B ** k) < 1e-12 * max(1.0, abs(dK[k]))
    assert abs(P(1.0) - math.exp(-0.25 / sigma ** 2)) < 1e-14
    for k in range(1, p):
        assert abs(P.deriv(k)(1.0)) < 1e-9
    # inside the ball K_R is the Gaussian
    r = np.linspace(0, rI, 7)
    assert np.allclose(alg1.K_R(r, sigma, eps_B, p), np.exp(-r ** 2 / sigma ** 2), rtol=1e-15)


def test_box_reading_wide_kernel_two_points():
    # Two points with a kernel much wider than their distance: the box scaling
    # shrinks the cloud so that the periodised kernel's wrap stays below
    # 1e-8; Alg. 1 then reproduces the closed form W = [[0, w], [w, 0]].
    X = np.array([[0.0, 0.0, 0.0], [0.05, 0.0, 0.0]])
    Xs, ss, _, _ = alg1.scale_to_domain(X, 0.1, 0.0, 1e-8)
    w = math.exp(-0.25)
    y = alg1.fastsum_W(Xs, np.array([2.0, -3.0]), alg1.bhat(ss, 16, 3))
    assert np.abs(y - [-3 * w, 2 * w]).max() <= 1e-7


def test_ball_domain_scaling():
    X = workloads.uniform_cube(500, 3, seed=8)
    Xs, ss, c, s = alg1.scale_to_domain(X, 0.1, eps_B=1.0 / 16)
    assert np.sqrt((Xs ** 2).sum(1)).max() <= 0.25 - 1.0 / 32 + 1e-15
    assert abs(ss - 0.1 * s) < 1e-16
    # pairwise distances stay below 1/2 - eps_B
    D = np.sqrt(((Xs[:, None] - Xs[None]) ** 2).sum(-1))
    assert D.max() <= 0.5 - 1.0 / 16 + 1e-14



# ------------------------------------------------------- Laplacian kernel
def _geometric_lattice_degrees(n, h, sigma):
    # sum_{j != i} q^{|i-j|}, q = exp(-h/sigma): two finite geometric series
    q = math.exp(-h / sigma)
    i = np.arange(n)
    return q * (1 - q ** i) / (1 - q) + q * (1 - q ** (n - 1 - i)) / (1 - q)


def test_laplace_lattice_degrees_geometric_series():
    n, h, sigma = 60, 0.3, 0.7
    X = (h * np.arange(n))[:, None]
    deg = graph.degrees(X, sigma, kernel="laplace")
    assert np.allclose(deg, _geometric_lattice_degrees(n, h, sigma), rtol=1e-13, atol=0)


def test_laplace_rotated_line_in_3d():
    # the same lattice along a unit direction: the Euclidean norm gives the same
    # degrees (the l1 norm or the squared norm would not)
    n, h, sigma = 40, 0.25, 0.5
    u = np.array([1.0, 2.0, 2.0]) / 3.0
    X = (h * np.arange(n))[:, None] * u[None, :] + np.array([0.3, -1.0, 2.0])
    deg = graph.degrees(X, sigma, kernel="laplace")
    assert np.allclose(deg, _geometric_lattice_degrees(n, h, sigma), rtol=1e-12, atol=0)
    W = graph.weight_matrix(X, sigma, kernel="laplace")
    assert np.allclose(W.sum(1), deg, rtol=1e-13)


def test_laplace_inner_regulariser_matches_kernel():
    # one-sided finite differences of K_R just inside eps_I against the
    # analytic derivatives (-1/sigma)^k exp(-eps_I/sigma) of the Laplacian,
    # and K_R even and smooth at the origin
    sigma, eps_I, p = 0.05, 0.03, 8
    f = lambda r: alg1.K_R(np.asarray(r, dtype=float), sigma, 1.0 / 8, p, "laplace", eps_I)
    x = eps_I * (1 - 1e-13)
    hh = 1e-4 * eps_I
    f0, f1, f2, f3 = (float(f(x - k * hh)) for k in range(4))
    e = math.exp(-eps_I / sigma)
    assert abs(f0 - e) <= 1e-12
    d1 = (3 * f0 - 4 * f1 + f2) / (2 * hh)
    assert abs(d1 - (-e / sigma)) <= 1e-6 * e / sigma
    d2 = (2 * f0 - 5 * f1 + 4 * f2 - f3) / hh ** 2
    assert abs(d2 - e / sigma ** 2) <= 1e-3 * e / sigma ** 2
    # smooth at 0: K_R(t) - K_R(0) is quadratic in t (a cusp would be linear)
    t = 1e-4
    ratio = (float(f(2 * t)) - float(f(0.0))) / (float(f(t)) - float(f(0.0)))
    assert abs(ratio - 4.0) <= 1e-3
    # outside eps_I it is the kernel itself
    r = np.linspace(eps_I, 0.5 - 1.0 / 8, 50)
    assert np.allclose(f(r), np.exp(-r / sigma), rtol=1e-15)


@pytest.mark.parametrize("d,N,c,tol", [(1, 64, 8, 1e-6), (2, 64, 8, 1e-5), (3, 48, 6, 1e-4)])
def test_laplace_alg1_with_near_field_against_direct_sum(d, N, c, tol):
    rng = np.random.default_rng(20 + d)
    X = rng.normal(size=(220, d))
    sigma, p = 0.8, 8
    eps_I = c / N
    eps_B = max(1.0 / 16, eps_I)
    Xs, ss, _, _ = alg1.scale_to_domain(X, sigma, eps_B=eps_B)
    v = rng.random(220)
    b = alg1.bhat(ss, N, d, eps_B, p, "laplace", eps_I)
    far = alg1.fastsum_W(Xs, v, b)
    near = alg1.near_field(Xs, v, ss, eps_I, p)
    ref = graph.W_apply(X, sigma, v, kernel="laplace")
    l1 = np.abs(v).sum()
    assert np.abs(far + near - ref).max() <= tol * l1
    # the near field carries the cusp: without it the error is orders larger
    assert np.abs(far - ref).max() >= 100 * tol * l1

# ------------------------------------------------------------------ MLP oracle
def test_mlp_gradient_matches_finite_differences():
    from oracle import mlp
    rng = np.random.default_rng(0)
    n_in, h, n_out, B = 5, 7, 2, 11
    npar = h * n_in + h + h * h + h + n_out * h + n_out
    p = rng.normal(0, 0.5, npar)
    X = rng.normal(0, 1, (B, n_in))
    Y = rng.normal(0, 1, (B, n_out))
    norm = (rng.normal(0, 1, n_in), rng.uniform(0.5, 2, n_in), rng.normal(0, 1, n_out), rng.uniform(0.5, 2, n_out))
    loss, g = mlp.loss_grad(p, X, Y, n_in, h, n_out, norm)
    eps = 1e-6
    for i in rng.choice(npar, 25, replace=False):
        e = np.zeros(npar)
        e[i] = eps
        fd = (mlp.loss_grad(p + e, X, Y, n_in, h, n_out, norm)[0] -
              mlp.loss_grad(p - e, X, Y, n_in, h, n_out, norm)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd))
    # the loss is the mean squared error of the standardised outputs
    Z = (mlp.forward(p, X, n_in, h, n_out, norm) - norm[2]) / norm[3]
    assert abs(loss - np.mean((Z - (Y - norm[2]) / norm[3]) ** 2)) < 1e-14


# ---------------------------------------------------------------- Alg. 2
def test_allen_cahn_T_is_gradient_of_potential():
    # Eq. def:T_ij is the gradient of the multi-well potential of
    # Eq. def_multiwell at points where every entry lies in (0, 1)
    from oracle import allen_cahn as ac
    rng = np.random.default_rng(40)
    for m in (2, 3, 4, 5):
        U = rng.dirichlet(np.ones(m) * 3.0, size=20)
        U = np.clip(U, 0.02, 0.98)
        T = ac.T_matrix(U)
        h = 1e-6
        G = np.zeros_like(U)
        for j in range(m):
            E = np.zeros(m)
            E[j] = h
            G[:, j] = (ac.potential(U + E) - ac.potential(U - E)) / (2 * h)
        assert np.abs(T - G).max() <= 1e-7 * max(1.0, np.abs(G).max())


def test_simplex_projection_optimal():
    from oracle import allen_cahn as ac
    rng = np.random.default_rng(41)
    # m = 2: the projection onto the segment has the closed form x1 = clip((y1 - y2 + 1)/2, 0, 1)
    Y = rng.normal(0, 2, (50, 2))
    X = ac.project_simplex(Y)
    x1 = np.clip((Y[:, 0] - Y[:, 1] + 1.0) / 2.0, 0.0, 1.0)
    assert np.abs(X[:, 0] - x1).max() <= 1e-14 and np.abs(X.sum(1) - 1).max() <= 1e-14
    # m = 3..6: on the simplex, and no sampled simplex point is closer
    for m in (3, 4, 6):
        Y = rng.normal(0, 1, (30, m))
        X = ac.project_simplex(Y)
        assert (X >= 0).all() and np.abs(X.sum(1) - 1).max() <= 1e-13
        Z = rng.dirichlet(np.ones(m), size=4000)
        for i in range(len(Y)):
            d_best = np.sum((X[i] - Y[i]) ** 2)
            assert (np.sum((Z - Y[i]) ** 2, axis=1) >= d_best - 1e-12).all()
            # and small moves within the simplex do not get closer
            for _ in range(50):
                D = rng.normal(0, 1e-3, m)
                D -= D.mean()
                Z1 = X[i] + D
                if (Z1 >= 0).all():
                    assert np.sum((Z1 - Y[i]) ** 2) >= d_best - 1e-15


def test_allen_cahn_full_eigenbasis_matches_dense_scheme():
    # with all n eigenpairs the projected iteration of Alg. 2 is the scheme of
    # Eq. U_lp1 solved densely, followed by the simplex projection
    from oracle import allen_cahn as ac
    n, m = 60, 3
    X = workloads.uniform_cube(n, 2, seed=42)
    L = graph.L_sym_dense(X, 0.15)
    lam, Phi = np.linalg.eigh(L)
    labels = -np.ones(n, dtype=int)
    labels[[0, 7, 19, 33, 51]] = [0, 1, 2, 0, 1]
    eps, omega0, dt = 0.05, 1000.0, 0.01
    c = omega0 + 3.0 / eps
    U_alg, it, _ = ac.allen_cahn(Phi, lam, labels, m, eps, omega0, c, dt, tol=0.0, max_iter=6)
    assert it == 6
    B = (1.0 + c * dt) * np.eye(n) + eps * dt * L
    F = np.zeros((n, m))
    F[labels >= 0, labels[labels >= 0]] = 1.0
    omega = np.where(labels >= 0, omega0, 0.0)
    U = ac.initial_scores(labels, m)
    for _ in range(6):
        R = (1.0 + c * dt) * U - dt / (2 * eps) * ac.T_matrix(U) - dt * omega[:, None] * (U - F)
        U = ac.project_simplex(np.linalg.solve(B, R))
    assert np.abs(U_alg - U).max() <= 1e-12
    assert (ac.predict(U_alg)[labels >= 0] == labels[labels >= 0]).all()


def _golden_sbm():
    rows = []
    path = os.path.join(os.path.dirname(__file__), "golden", "sbm_allen_cahn.txt")
    with open(path) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                case, p, err = line.split()
                rows.append((case, float(p), float(err)))
    return rows


def _sbm_error(case, p, graphs, seed):
    from oracle import allen_cahn as ac
    errs = []
    for g in range(graphs):
        noisy = case == "noisy"
        Ws, truth = workloads.block_model_layers([50, 50], [0.7, 0.5 if noisy else 0.7],
                                                 [0.3, 0.5 if noisy else 0.3], seed=seed + g)
        lam, Phi = eigen.power_mean_eigs([graph.L_sym_from_W(W) for W in Ws], p, 2)
        labels = workloads.known_labels(truth, 0.04, seed=seed + 1000 + g)
        eps, omega0 = 0.005, 1000.0
        U, _, _ = ac.allen_cahn(Phi, lam, labels, 2, eps, omega0, omega0 + 3.0 / eps, 0.01, 1e-6, 300)
        errs.append(np.mean(ac.predict(U) != truth))
    return 100.0 * float(np.mean(errs))


def test_sbm_example_of_the_paper():
    # The block-model example of Sec. 9: the paper prints mean classification
    # errors of Alg. 2 on the power mean Laplacian of a two-layer SBM whose
    # second layer is either informative or pure noise.  The sampler's details
    # and the random graphs are not given, so the oracle (its power means for
    # p > 0 and p < 0, eigenpairs and Alg. 2) is held to the outcome the paper
    # reports: every informative case and every negative p stays within
    # 5 percentage points of the printed error, while p = 10 with a noise layer
    # fails (at least half the printed 46.1 %, and far worse than p <= 1).
    got = {}
    for case, p, paper in _golden_sbm():
        err = _sbm_error(case, p, graphs=25, seed=700 if case == "clean" else 800)
        got[(case, p)] = err
        if paper < 10.0:
            assert err <= paper + 5.0, (case, p, err, paper)
        else:
            assert err >= 0.5 * paper, (case, p, err, paper)
    good = max(got[("noisy", 1.0)], got[("noisy", -20.0)], got[("noisy", -30.0)])
    assert got[("noisy", 10.0)] >= 5.0 * good + 10.0, got


# ------------------------------------------------------ comparison helpers
def test_subspace_angle_known_angles():
    # the GPU parity tests bound eigenvector errors by this angle, so it is
    # pinned on subspaces with known principal angles
    rng = np.random.default_rng(21)
    Q, _ = np.linalg.qr(rng.standard_normal((9, 9)))
    for theta in (0.0, 1e-7, 0.3, 1.2):
        u = Q[:, 0]
        v = math.cos(theta) * Q[:, 0] + math.sin(theta) * Q[:, 1]
        assert abs(eigen.subspace_angle(u[:, None], v[:, None]) - theta) <= 1e-9
        # sign and scale of the basis do not matter
        assert abs(eigen.subspace_angle(u[:, None], -3.0 * v[:, None]) - theta) <= 1e-9
    # two planes: principal angles 0.2 and 0.7; the largest is reported
    U = Q[:, :2]
    V = np.stack([math.cos(0.2) * Q[:, 0] + math.sin(0.2) * Q[:, 2],
                  math.cos(0.7) * Q[:, 1] + math.sin(0.7) * Q[:, 3]], axis=1)
    assert abs(eigen.subspace_angle(U, V) - 0.7) <= 1e-9
    # a rotation inside the same plane is angle 0
    R = np.array([[math.cos(0.4), -math.sin(0.4)], [math.sin(0.4), math.cos(0.4)]])
    assert eigen.subspace_angle(U, U @ R) <= 1e-7


def test_eigen_groups_and_sign_convention():
    lam = np.array([0.0, 0.5, 0.5 + 1e-9, 0.5 + 2e-9, 1.0, 2.0 - 1e-8, 2.0])
    assert eigen.eigen_groups(lam, rel_gap=1e-6) == [[0], [1, 2, 3], [4], [5, 6]]
    assert eigen.eigen_groups(lam, rel_gap=1e-12) == [[i] for i in range(7)]
    Phi = np.array([[0.1, -0.9], [-0.8, 0.2], [0.3, 0.1]])
    F = eigen.fix_signs(Phi)
    assert np.array_equal(F[:, 0], -Phi[:, 0]) and np.array_equal(F[:, 1], -Phi[:, 1])
    assert np.all(F[np.argmax(np.abs(F), axis=0), [0, 1]] > 0)


def test_oracle_reproduces_stored_values():
    # values written by tests/golden/make_oracle_golden.py from the oracle alone;
    # a change to the oracle's arithmetic shows here first
    path = os.path.join(os.path.dirname(__file__), "golden", "oracle_single_n2000_d3.txt")
    stored = {"eigenvalue": {}, "degree": {}}
    with open(path) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                kind, i, v = line.split()
                stored[kind][int(i)] = float(v)
    X = workloads.uniform_cube(2000, 3, seed=1)
    lam, _ = eigen.lsym_eigs(X, 0.1, 10)
    deg = graph.degrees(X, 0.1)[:16]
    assert np.allclose(lam, [stored["eigenvalue"][i] for i in range(10)], rtol=0, atol=1e-12)
    assert np.allclose(deg, [stored["degree"][j] for j in range(16)], rtol=1e-13, atol=0)
    assert abs(stored["eigenvalue"][0]) <= 1e-12            # lambda_0 = 0 (connected graph)
