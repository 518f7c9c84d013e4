"""Oracle: eigenpairs of the graph operators (test infrastructure only).

* `smallest_eigs(L, k)`: k smallest eigenpairs of a dense symmetric matrix,
  numpy's eigh as the library step.  Ascending eigenvalues; each eigenvector's
  sign fixed so that its largest-magnitude entry is positive.
* `lsym_eigs`, `L1_eigs`, `Lp_eigs`: the k smallest eigenpairs of L_sym,
  of L_1 = (1/T) sum_t L_sym^(t) (Sec. 3: the k largest of I - L_1, lambda =
  1 - theta), and of L_{p,delta} for p < 0 (Sec. 3: the k largest mu of
  L_{p,delta}^p map to lambda = mu^(1/p) because lambda -> lambda^p reverses
  the order).
* `power_mean_eigs(Ls, p, k)`: the same for given layer Laplacians (weight
  matrices given directly, e.g. a stochastic block model) and any p != 0,
  including p > 0 (delta = 0, the k smallest mu).
* `jacobi_eigh(A)`: textbook cyclic Jacobi rotations (Golub & Van Loan,
  Matrix Computations, Sec. 8.5), a second opinion independent of LAPACK;
  small n only.

Pinned by tests/test_oracle_pins.py: Jacobi against eigh, the equilateral
closed form {0, n/(n-1)}, the spectrum bounds [0, 2], sum(lambda) = n,
lambda_0 = 0, the p-mapping on identical layers, the power means of commuting
layers against the scalar power means of their eigenvalues, subspace_angle on
subspaces with known principal angles (0 to 1.2, 1e-7 included),
eigen_groups and the sign rule on crafted inputs; with the Allen-Cahn oracle,
the stochastic-block-model example of Sec. 9 (classification errors of
p = 10, 1, -20, -30 on a clean and a noisy second layer, within bands around
the paper's printed values, tests/golden/sbm_allen_cahn.txt).
"""
from __future__ import annotations

import numpy as np

from . import graph


def fix_signs(Phi):
    """Flip each column so that its largest-magnitude entry is positive."""
    Phi = np.array(Phi, dtype=np.float64, copy=True)
    idx = np.argmax(np.abs(Phi), axis=0)
    sgn = np.sign(Phi[idx, np.arange(Phi.shape[1])])
    sgn[sgn == 0] = 1.0
    return Phi * sgn[None, :]


def smallest_eigs(L, k):
    lam, Phi = np.linalg.eigh(0.5 * (L + L.T))
    return lam[:k].copy(), fix_signs(Phi[:, :k])


def largest_eigs(M, k):
    lam, Phi = np.linalg.eigh(0.5 * (M + M.T))
    order = np.argsort(lam)[::-1][:k]
    return lam[order].copy(), fix_signs(Phi[:, order])


def lsym_eigs(X, sigma, k, kernel="gauss"):
    return smallest_eigs(graph.L_sym_dense(X, sigma, kernel), k)


def L1_eigs(layers, sigmas, k, kernel="gauss"):
    """k smallest eigenpairs of L_1 via the k largest theta of I - L_1 (Sec. 3)."""
    T = len(layers)
    n = layers[0].shape[0]
    IL1 = np.zeros((n, n))
    for t in range(T):
        IL1 += np.eye(n) - graph.L_sym_dense(layers[t], sigmas[t], kernel)
    IL1 /= T
    theta, Phi = largest_eigs(IL1, k)
    return 1.0 - theta, Phi


def Lp_eigs(layers, sigmas, p, k, kernel="gauss"):
    """k smallest eigenpairs of L_{p,delta} for p < 0 (Sec. 3)."""
    if p >= 0:
        raise ValueError("use L1_eigs for p = 1")
    M = graph.power_mean_p_dense(layers, sigmas, p, kernel)
    mu, Phi = largest_eigs(M, k)
    return mu ** (1.0 / p), Phi


def power_mean_eigs(Ls, p, k):
    """k smallest eigenpairs of the power mean L_{p,delta} = M^(1/p),
    M = (1/T) sum_t (L_t + delta I)^p, of given layer Laplacians (Eq.
    power_mean_laplacian_shifted; delta = 0 for p > 0, Sec. 2).  lambda ->
    lambda^(1/p) is increasing for p > 0 and decreasing for p < 0, so the k
    smallest lambda come from the k smallest mu for p > 0 and from the k
    largest for p < 0.  p = 1 is the plain mean of the L_t."""
    if p == 1:
        return smallest_eigs(sum(np.asarray(L, dtype=np.float64) for L in Ls) / len(Ls), k)
    M = graph.power_mean_of_laplacians(Ls, p)
    mu, Phi = largest_eigs(M, k) if p < 0 else smallest_eigs(M, k)
    return np.maximum(mu, 0.0) ** (1.0 / p), Phi


def jacobi_eigh(A, tol=1e-14, max_sweeps=60):
    """Cyclic Jacobi eigenvalue algorithm for a symmetric matrix.

    Each rotation annihilates A[p, q] with the stable choice of tan(theta)
    (the smaller root), applied to rows/columns p, q and accumulated in V.
    Returns (ascending eigenvalues, eigenvectors as columns).
    """
    A = np.array(A, dtype=np.float64, copy=True)
    n = A.shape[0]
    V = np.eye(n)
    for _ in range(max_sweeps):
        off = np.sqrt(np.sum(np.tril(A, -1) ** 2))
        if off <= tol * np.sqrt(np.sum(A * A)):
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                apq = A[p, q]
                if apq == 0.0:
                    continue
                tau = (A[q, q] - A[p, p]) / (2.0 * apq)
                t = np.sign(tau) / (abs(tau) + np.sqrt(1.0 + tau * tau)) if tau != 0 else 1.0
                c = 1.0 / np.sqrt(1.0 + t * t)
                s = t * c
                Ap = A[:, p].copy()
                Aq = A[:, q].copy()
                A[:, p] = c * Ap - s * Aq
                A[:, q] = s * Ap + c * Aq
                Ap = A[p, :].copy()
                Aq = A[q, :].copy()
                A[p, :] = c * Ap - s * Aq
                A[q, :] = s * Ap + c * Aq
                Vp = V[:, p].copy()
                Vq = V[:, q].copy()
                V[:, p] = c * Vp - s * Vq
                V[:, q] = s * Vp + c * Vq
    lam = np.diag(A).copy()
    order = np.argsort(lam)
    return lam[order], V[:, order]


def subspace_angle(U, V):
    """Largest principal angle between span(U) and span(V) of equal dimension
    (radians), Bjorck & Golub (1973): its cosine is the smallest singular value
    of Qu^T Qv, its sine the largest of (I - Qu Qu^T) Qv; atan2 of the two is
    accurate at every angle (the cosine alone cannot resolve angles below
    about 1e-8)."""
    Qu, _ = np.linalg.qr(U)
    Qv, _ = np.linalg.qr(V)
    c = np.linalg.svd(Qu.T @ Qv, compute_uv=False).min()
    s = np.linalg.svd(Qv - Qu @ (Qu.T @ Qv), compute_uv=False).max()
    return float(np.arctan2(s, c))


def eigen_groups(lam, rel_gap=1e-6):
    """Group indices of (sorted) eigenvalues whose neighbours are closer than
    rel_gap times the spectrum width (near-degenerate clusters)."""
    lam = np.asarray(lam)
    width = max(float(lam.max() - lam.min()), 1e-300)
    groups, cur = [], [0]
    for i in range(1, len(lam)):
        if lam[i] - lam[i - 1] < rel_gap * width:
            cur.append(i)
        else:
            groups.append(cur)
            cur = [i]
    groups.append(cur)
    return groups
