"""Oracle: Alg. 1 (NFFT-based fast summation, Sec. 4) without the NFFT's
approximations (test infrastructure only).

Alg. 1 replaces K by the trigonometric polynomial
    K_RF(y) = sum_{l in I_N} b_l exp(2 pi i l.y),  I_N = {-N/2..N/2-1}^d   (Eq. K_RF)
whose coefficients come from samples of the (regularised) kernel on k/N,
    b_l = N^{-d} sum_{k in I_N} K_R(k/N) exp(-2 pi i l.k/N)   (footnote to Sec. 4)
and evaluates f_RF(x_i) = sum_l b_l v_hat_l exp(2 pi i l.x_i) with
v_hat_l = sum_j v_j exp(-2 pi i l.x_j)  (Eq. nfftWtilde_x:kernel:RF).
Steps 1 and 3 of Alg. 1 (adjoint NFFT, NFFT) are done here as the exact
non-equispaced sums they approximate; the output is real up to the term of
the unpaired frequency -N/2, and the real part is returned.  W v then follows
as f_RF - K(0) v (Sec. 4, W = W~ - K(0) I).

Readings of what the paper leaves open:

* Domain (the node condition of Alg. 1 is garbled).  Alg. 1 wants nodes in [-1/4, 1/4]^d.  W depends only
  on ||x_i - x_j|| / sigma, so each layer is mapped by one isotropic affine
  map x' = s (x - c), sigma' = s sigma, with c the bounding-box centre.
  - eps_B > 0 ("ball"): s = (1/4 - eps_B/2) / max_i ||x_i - c||_2, so every
    pair distance is <= 1/2 - eps_B where K_R = K.
  - eps_B = 0 ("box"): s = a / h with h the largest bounding-box half-extent
    and a = min(1/4, 1 / (2 + (sigma/h) sqrt(ln(2d/eps_wrap)))), which keeps
    the periodisation error 2d exp(-(1-2a)^2/sigma'^2) below eps_wrap.
* Regulariser (deferred by the paper to the NFFT literature).  K_R is the smooth 1-periodic regularised kernel
  of the footnote to Sec. 4.  For eps_B = 0 it is the 1-periodisation of the
  Gaussian, K_R(y) = sum_{r in Z^d} K(y + r), which equals K up to the wrap
  error above for every difference of two nodes.  For eps_B > 0, K_R(r) = K(r) for
  r <= r_I = 1/2 - eps_B; on (r_I, 1/2] it is the two-point Taylor polynomial
  of degree 2p-1 matching K's derivatives 0..p-1 at r_I, with value K(1/2)
  and vanishing derivatives 1..p-1 at r = 1/2; beyond 1/2 (cube corners) it
  stays at K(1/2).

* Laplacian kernel K(r) = exp(-r/sigma) (named in Sec. 4).  Its cusp at r = 0
  makes the Fourier coefficients of K itself decay slowly, so (as in the
  fast summation of non-smooth radial kernels that Sec. 4 refers to) K_R is
  regularised at the origin as well: on r < eps_I it is the even polynomial
  sum_{j<p} c_j r^{2j} matching K's derivatives 0..p-1 at r = eps_I (smooth
  at 0 in every dimension).  Alg. 1 then sums K_R, and the near field
      f_NE(x_i) = sum_{j: ||x_i - x_j|| < eps_I} (K - K_R)(||x_i - x_j||) v_j
  (the pair j = i included, so that W v = f_RF + f_NE - K(0) v) is added by
  direct summation.  The ball domain is required; its outer regulariser
  matches the Laplacian's derivatives (-1/sigma)^k exp(-r/sigma).

Pinned by tests/test_oracle_pins.py: b_l against the closed-form Fourier
coefficients of the periodised Gaussian (Poisson summation); the adjoint
transform on equispaced nodes against numpy's FFT; f_RF - K(0) v against the
direct sum within the Fourier-tail bound, also on the ball domain; the
regulariser's matching conditions, and its smoothness setting the rate at
which the error falls with N (at least N^-p); for the Laplacian, the continuity of K_R and of its first
derivatives across r = eps_I by one-sided finite differences, and
f_RF + f_NE - K(0) v against the direct sum within the kernel approximation
error measured on the same grid.
"""
from __future__ import annotations

import math

import numpy as np


# ----------------------------------------------------------------- domain
def scale_to_domain(X, sigma, eps_B=0.0, eps_wrap=1e-9):
    """Isotropic map of one layer into the Alg. 1 domain (Domain, above).

    Returns (Xs, sigma_s, c, s) with Xs = s (X - c) and sigma_s = s sigma.
    """
    X = np.asarray(X, dtype=np.float64)
    n, d = X.shape
    lo, hi = X.min(axis=0), X.max(axis=0)
    c = 0.5 * (lo + hi)
    if eps_B > 0:
        rmax = float(np.sqrt(((X - c) ** 2).sum(axis=1)).max())
        if rmax <= 0:
            rmax = sigma
        s = (0.25 - 0.5 * eps_B) / rmax
    else:
        h = float(0.5 * (hi - lo).max())
        if h <= 0:
            h = sigma
        a = min(0.25, 1.0 / (2.0 + (sigma / h) * math.sqrt(math.log(2.0 * d / eps_wrap))))
        s = a / h
    return s * (X - c), s * sigma, c, s


# ------------------------------------------------------------ regulariser
def _gauss_derivs(r, sigma, p):
    """K^{(k)}(r) for k = 0..p-1, K(r) = exp(-r^2/sigma^2).

    With z = r/sigma, d^k/dr^k exp(-z^2) = (-1)^k sigma^-k H_k(z) exp(-z^2),
    H_k the physicists' Hermite polynomials (H_{k+1} = 2z H_k - 2k H_{k-1}).
    """
    z = r / sigma
    H = [1.0, 2.0 * z]
    for k in range(1, p):
        H.append(2.0 * z * H[k] - 2.0 * k * H[k - 1])
    e = math.exp(-z * z)
    return [((-1.0) ** k) * (sigma ** -k) * H[k] * e for k in range(p)]


def _laplace_derivs(r, sigma, p):
    """K^{(k)}(r) for k = 0..p-1, K(r) = exp(-r/sigma): (-1/sigma)^k exp(-r/sigma)."""
    e = math.exp(-r / sigma)
    return [((-1.0 / sigma) ** k) * e for k in range(p)]


def _radial(r, sigma, kernel):
    r = np.asarray(r, dtype=np.float64)
    return np.exp(-(r * r) / (sigma * sigma)) if kernel == "gauss" else np.exp(-r / sigma)


def regulariser_poly(sigma, eps_B, p, kernel="gauss"):
    """Monomial coefficients q_0..q_{2p-1} of the two-point Taylor polynomial
    in t = (r - r_I)/eps_B on [0, 1] (Regulariser, above)."""
    rI = 0.5 - eps_B
    dK = (_gauss_derivs if kernel == "gauss" else _laplace_derivs)(rI, sigma, p)
    n = 2 * p
    A = np.zeros((n, n))
    rhs = np.zeros(n)
    # derivative k of t^j at t: j!/(j-k)! t^(j-k)
    for k in range(p):
        for j in range(k, n):
            A[k, j] = math.factorial(j) / math.factorial(j - k) * (0.0 ** (j - k))
            A[p + k, j] = math.factorial(j) / math.factorial(j - k)
        rhs[k] = dK[k] * eps_B ** k
        rhs[p + k] = float(_radial(0.5, sigma, kernel)) if k == 0 else 0.0
    return np.linalg.solve(A, rhs)


def inner_poly(sigma, eps_I, p):
    """Coefficients c_0..c_{p-1} of the inner regulariser of the Laplacian,
    P(r) = sum_j c_j r^{2j}, with P^{(k)}(eps_I) = K^{(k)}(eps_I), k < p
    (Laplacian kernel, above).  The k-th derivative of r^{2j} is (2j)!/(2j-k)! r^{2j-k}."""
    dK = _laplace_derivs(eps_I, sigma, p)
    A = np.zeros((p, p))
    for k in range(p):
        for j in range(p):
            e = 2 * j
            if e >= k:
                A[k, j] = math.factorial(e) / math.factorial(e - k) * eps_I ** (e - k)
    return np.linalg.solve(A, np.array(dK))


def K_R(r, sigma, eps_B=0.0, p=0, kernel="gauss", eps_I=0.0):
    """Regularised radial kernel of the ball domain (Regulariser, above; the
    Laplacian kernel, above, for its inner part); the plain Gaussian when eps_B = 0 (the box
    domain samples its periodisation instead, see kernel_samples)."""
    r = np.asarray(r, dtype=np.float64)
    K = _radial(r, sigma, kernel)
    if eps_B <= 0:
        if kernel != "gauss":
            raise ValueError("the Laplacian kernel needs the ball domain (eps_B > 0)")
        return K
    q = regulariser_poly(sigma, eps_B, p, kernel)
    rI = 0.5 - eps_B
    t = np.clip((r - rI) / eps_B, 0.0, 1.0)
    P = np.polyval(q[::-1], t)
    out = np.where(r <= rI, K, P)
    if kernel == "laplace":
        c = inner_poly(sigma, eps_I, p)
        Pin = np.polyval(c[::-1], r * r)
        out = np.where(r < eps_I, Pin, out)
    return out


def periodised_gaussian_1d(y, sigma, images=None):
    """sum_{r in Z} exp(-(y + r)^2 / sigma^2), truncated where the terms vanish."""
    y = np.asarray(y, dtype=np.float64)
    R = images if images is not None else 2 + int(math.ceil(8.0 * sigma))
    return sum(np.exp(-((y + r) ** 2) / (sigma * sigma)) for r in range(-R, R + 1))


# ------------------------------------------------------- Fourier coefficients
def kernel_samples(sigma_s, N, d, eps_B=0.0, p=0, kernel="gauss", eps_I=0.0):
    """K_R on the grid k/N, k in I_N^d (Regulariser, above), shape (N,)*d indexed by k + N/2."""
    k = np.arange(-N // 2, N // 2) / N
    if eps_B <= 0 and kernel == "gauss":
        g1 = periodised_gaussian_1d(k, sigma_s)
        out = g1
        for _ in range(d - 1):
            out = np.multiply.outer(out, g1)
        return out
    grids = np.meshgrid(*([k] * d), indexing="ij")
    r = np.sqrt(sum(g * g for g in grids))
    return K_R(r, sigma_s, eps_B, p, kernel, eps_I)


def bhat(sigma_s, N, d, eps_B=0.0, p=0, kernel="gauss", eps_I=0.0):
    """b_l, l in I_N^d, from N^d samples of K_R on k/N and a d-dim FFT.

    Returned as a real array of shape (N,)*d indexed by l + N/2 on every axis.
    """
    samples = kernel_samples(sigma_s, N, d, eps_B, p, kernel, eps_I)
    # FFT wants index 0 at k = 0: shift, transform, shift back to l + N/2 order.
    F = np.fft.fftn(np.fft.ifftshift(samples)) / float(N) ** d
    return np.real(np.fft.fftshift(F))


# ------------------------------------------------------------- Alg. 1
def _exp_factors(Xs, N, sign):
    l = np.arange(-N // 2, N // 2)
    return [np.exp(sign * 2j * np.pi * np.outer(Xs[:, a], l)) for a in range(Xs.shape[1])]


def adjoint_ndft(Xs, v, N):
    """Step 1 of Alg. 1 done exactly: v_hat_l = sum_j v_j exp(-2 pi i l.x_j)."""
    E = _exp_factors(Xs, N, -1.0)
    v = np.asarray(v, dtype=np.float64)
    d = Xs.shape[1]
    if d == 1:
        return v @ E[0]
    if d == 2:
        return np.einsum("j,ja,jb->ab", v, E[0], E[1], optimize=True)
    return np.einsum("j,ja,jb,jc->abc", v, E[0], E[1], E[2], optimize=True)


def ndft(Xs, fhat, N):
    """Step 3 of Alg. 1 done exactly: f(x_i) = sum_l fhat_l exp(2 pi i l.x_i)."""
    E = _exp_factors(Xs, N, +1.0)
    d = Xs.shape[1]
    if d == 1:
        return E[0] @ fhat
    if d == 2:
        return np.einsum("ab,ia,ib->i", fhat, E[0], E[1], optimize=True)
    return np.einsum("abc,ia,ib,ic->i", fhat, E[0], E[1], E[2], optimize=True)


def fastsum_Wtilde(Xs, v, b):
    """Alg. 1: f_RF(x_i) ~ (W~ v)_i with exact non-equispaced sums (real part)."""
    N = b.shape[0]
    vhat = adjoint_ndft(Xs, v, N)          # step 1
    fhat = b * vhat                        # step 2
    return np.real(ndft(Xs, fhat, N))      # step 3


def fastsum_W(Xs, v, b, K0=1.0):
    """W v = W~ v - K(0) v  (Sec. 4)."""
    v = np.asarray(v, dtype=np.float64)
    return fastsum_Wtilde(Xs, v, b) - K0 * v


def near_field(Xs, v, sigma_s, eps_I, p):
    """f_NE(x_i) = sum_{j: ||x_i - x_j|| < eps_I} (K - K_R)(||x_i - x_j||) v_j for the
    Laplacian, the pair j = i included (Laplacian kernel, above).  Direct O(n^2) sum."""
    Xs = np.asarray(Xs, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    c = inner_poly(sigma_s, eps_I, p)
    out = np.zeros(Xs.shape[0])
    for i in range(Xs.shape[0]):
        r = np.sqrt(((Xs - Xs[i]) ** 2).sum(axis=1))
        near = r < eps_I
        rn = r[near]
        out[i] = np.dot(np.exp(-rn / sigma_s) - np.polyval(c[::-1], rn * rn), v[near])
    return out
