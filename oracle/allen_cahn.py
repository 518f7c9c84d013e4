"""Oracle: the multiclass multilayer graph Allen-Cahn scheme (Alg. 2, Sec. 6
and Sec. 7) in FP64 (test infrastructure only).

Written from the definitions, in the order of Alg. 2:

* `potential(U)`      psi(u_i) = prod_{q=1..m} (1/4) ||u_i - e_q||_1^2
                      (Eq. def_multiwell, with the sum over the m classes).
* `T_matrix(U)`       T_ij = sum_q (1/2)(1 - 2 delta_jq) ||u_i - e_q||_1
                             prod_{p != q} (1/4) ||u_i - e_p||_1^2  (Eq. def:T_ij)
* `project_simplex(Y)` row-wise Euclidean projection onto the Gibbs simplex
                      (Eq. gibbssimplex) by the sort-and-threshold method of
                      Chen & Ye (2011): sort y ascending, the threshold t is the
                      first (from the top) t_i = (sum_{j>i} y_(j) - 1)/(m - i)
                      with t_i >= y_(i), else (sum y - 1)/m; x = max(y - t, 0).
* `allen_cahn(...)`   steps 2-4 of Alg. 2 from given eigenpairs (Phi_k,
                      Lambda_k): Z = [(1 + c dt) I + eps dt Lambda_k]^{-1} Phi_k^T,
                      U^0 (labelled rows e_j, others 1/m), then per iteration
                      T^l, V^{l+1} = Z((1 + c dt) U^l - dt/(2 eps) T^l
                      - dt omega (U^l - F)), U^{l+1} = projection of Phi_k V^{l+1},
                      relative_change = max_i ||u_i^{l+1} - u_i^l||^2 /
                      max_i ||u_i^{l+1}||^2, stop when <= tol or after max_iter.
* `predict(U)`        row-wise argmax, ties to the lowest class id (Sec. 7).

Reading: Eq. def_multiwell writes the inner l1 sum with the index range 1..n;
it runs over the m entries of u_i (the paper's own inline form of the norm).

Pinned by tests/test_oracle_pins.py: T against central finite differences of
the potential at interior simplex points; the projection against its
optimality conditions and a brute-force search for m = 3; Alg. 2 with k = n
(all eigenpairs) against a dense solve of the un-projected scheme
Eq. U_lp1 followed by the projection.
"""
from __future__ import annotations

import numpy as np


def l1_to_corners(U):
    """a[i, q] = ||u_i - e_q||_1."""
    n, m = U.shape
    a = np.empty((n, m))
    for q in range(m):
        E = np.zeros(m)
        E[q] = 1.0
        a[:, q] = np.abs(U - E[None, :]).sum(axis=1)
    return a


def potential(U):
    a = l1_to_corners(U)
    return np.prod(0.25 * a * a, axis=1)


def T_matrix(U):
    n, m = U.shape
    a = l1_to_corners(U)
    T = np.zeros((n, m))
    for j in range(m):
        for q in range(m):
            sgn = 1.0 - 2.0 * (1.0 if j == q else 0.0)
            prod = np.ones(n)
            for p in range(m):
                if p != q:
                    prod *= 0.25 * a[:, p] ** 2
            T[:, j] += 0.5 * sgn * a[:, q] * prod
    return T


def project_simplex(Y):
    Y = np.asarray(Y, dtype=np.float64)
    n, m = Y.shape
    X = np.empty_like(Y)
    for i in range(n):
        y = Y[i]
        s = np.sort(y)
        t = (y.sum() - 1.0) / m
        for k in range(m - 1, 0, -1):           # k = m-1 .. 1 (1-based i of the method)
            ti = (s[k:].sum() - 1.0) / (m - k)
            if ti >= s[k - 1]:
                t = ti
                break
        X[i] = np.maximum(y - t, 0.0)
    return X


def initial_scores(labels, m):
    n = len(labels)
    U = np.full((n, m), 1.0 / m)
    lab = labels >= 0
    U[lab] = 0.0
    U[np.nonzero(lab)[0], labels[lab]] = 1.0
    return U


def allen_cahn(Phi, lam, labels, m, eps, omega0, c, dt, tol, max_iter):
    """Alg. 2 steps 2-4.  Phi n x k, lam k, labels n (class id or -1).
    Returns (U, iterations, relative changes per iteration)."""
    Phi = np.asarray(Phi, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    labels = np.asarray(labels)
    n, k = Phi.shape
    Z = (1.0 / ((1.0 + c * dt) + eps * dt * lam))[:, None] * Phi.T
    F = np.zeros((n, m))
    lab = labels >= 0
    F[np.nonzero(lab)[0], labels[lab]] = 1.0
    omega = np.where(lab, omega0, 0.0)
    U = initial_scores(labels, m)
    changes = []
    it = 0
    while True:
        T = T_matrix(U)
        R = (1.0 + c * dt) * U - dt / (2.0 * eps) * T - dt * omega[:, None] * (U - F)
        V = Z @ R
        Unew = project_simplex(Phi @ V)
        change = np.max(np.sum((Unew - U) ** 2, axis=1)) / np.max(np.sum(Unew ** 2, axis=1))
        U = Unew
        it += 1
        changes.append(float(change))
        if not (change > tol) or it >= max_iter:
            break
    return U, it, changes


def predict(U):
    return np.argmax(U, axis=1)      # numpy's argmax returns the first maximum
