"""Oracle: graph definitions of Sec. 2-3 in FP64 (test infrastructure only).

Definitions followed, each written out directly:

* weight function  w(x_i, x_j) = K(x_i - x_j) for i != j, w(x_i, x_i) = 0
  (Sec. 2: no self-edges) with one of the radial kernels of Sec. 4:
  the Gaussian K(y) = exp(-||y||^2 / sigma^2) (kernel="gauss", the default)
  or the Laplacian K(y) = exp(-||y|| / sigma) (kernel="laplace").
* degree           deg(x_i) = sum_j w(x_i, x_j),  D = diag(W 1)      (Sec. 2)
* normalised       L_sym = I - D^{-1/2} W D^{-1/2}                   (Sec. 2)
* multilayer p=1   I - L_1 = (1/T) sum_t D_t^{-1/2} W_t D_t^{-1/2}    (Eq. I-L_1)
* shifted power    L_{p,delta}^p = (1/T) sum_t (L_sym^(t) + delta I)^p,
                   delta = log(1+|p|) for p<0, 0 for p>0             (Sec. 2,
                   Eq. power_mean_laplacian_shifted, Eq. L_p_delta_power_p)

Pinned by tests/test_oracle_pins.py: two-point and equilateral closed forms,
the Poisson-summation value of a lattice degree, the sigma -> infinity limit,
and the invariants A D^{1/2} 1 = D^{1/2} 1, trace A = 0; for the Laplacian,
the geometric-series degrees of an equispaced 1-d lattice, and the same
lattice laid along a rotated line in 3-d (the Euclidean norm, not its square
nor the l1 norm).  The layer means multilayer_A_apply / multilayer_W_apply:
two-point layers (the normalised mean swaps v exactly; the raw mean scales the
swap by the mean weight), a three-point line plus an equilateral triangle in
closed form, T identical layers against the single layer, invariance under the
layer order, W 1 = the mean degrees, and the identity's image against the
dense I - L_1 of numpy weight matrices (symmetric, zero trace, spectrum in
[-1, 1], eigenvalues of eigen.L1_eigs).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_LIB = None


def _lib():
    """The compiled C direct sum, or None when it is not built."""
    global _LIB
    if _LIB is None:
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "liboracle_direct.so")
        if not os.path.exists(path):
            try:
                from . import build_oracle
                build_oracle.build()
            except Exception:
                return None
        lib = ctypes.CDLL(path)
        lib.oracle_gauss_rows.restype = ctypes.c_int
        lib.oracle_gauss_rows.argtypes = [
            ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
            ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int]
        lib.oracle_kernel_rows.restype = ctypes.c_int
        lib.oracle_kernel_rows.argtypes = [
            ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
            ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int]
        lib.oracle_num_threads.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def num_threads() -> int:
    lib = _lib()
    return int(lib.oracle_num_threads()) if lib is not None else 1


def gaussian(r2, sigma):
    """K as a function of the squared distance: exp(-r^2 / sigma^2) (Sec. 4)."""
    return np.exp(-np.asarray(r2, dtype=np.float64) / (sigma * sigma))


KERNELS = {"gauss": 0, "laplace": 1}


def kernel_of_r2(r2, sigma, kernel="gauss"):
    """K as a function of the squared distance for either kernel of Sec. 4."""
    r2 = np.asarray(r2, dtype=np.float64)
    if kernel == "gauss":
        return gaussian(r2, sigma)
    if kernel == "laplace":
        return np.exp(-np.sqrt(r2) / sigma)
    raise ValueError(f"unknown kernel {kernel!r}")


def weight_matrix(X, sigma, kernel="gauss"):
    """Dense W (n x n) with zero diagonal, squared distances summed from the
    coordinate differences (blocks of rows, any dimension).  Small n only."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    W = np.empty((n, n))
    step = max(1, int(2 ** 24 // max(1, n * X.shape[1])))
    for i0 in range(0, n, step):
        diff = X[i0:i0 + step, None, :] - X[None, :, :]
        W[i0:i0 + step] = kernel_of_r2(np.einsum("ijk,ijk->ij", diff, diff), sigma, kernel)
    np.fill_diagonal(W, 0.0)
    return W


def W_apply(X, sigma, V, rows=None, nthreads=0, kernel="gauss"):
    """(W V)[rows] by direct summation over all n points (FP64).

    X: (n, d) points, V: (n,) or (n, b).  rows: None (all) or an index array.
    Uses the C implementation; falls back to blocked numpy when it is absent.
    """
    X = np.ascontiguousarray(X, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    squeeze = V.ndim == 1
    V2 = np.ascontiguousarray(V.reshape(V.shape[0], -1))
    n, d = X.shape
    b = V2.shape[1]
    r = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    nrows = n if r is None else r.shape[0]
    out = np.empty((nrows, b), dtype=np.float64)
    lib = _lib()
    if lib is not None:
        rc = lib.oracle_kernel_rows(X.ctypes.data, n, d, float(sigma), KERNELS[kernel], V2.ctypes.data, b,
                                    None if r is None else r.ctypes.data, nrows,
                                    out.ctypes.data, int(nthreads))
        if rc != 0:
            raise ValueError("oracle_kernel_rows rejected its arguments")
    else:
        idx = np.arange(n) if r is None else r
        for s in range(0, nrows, 256):
            ii = idx[s:s + 256]
            diff = X[ii, None, :] - X[None, :, :]
            K = kernel_of_r2(np.einsum("ijk,ijk->ij", diff, diff), sigma, kernel)
            K[np.arange(len(ii)), ii] = 0.0
            out[s:s + 256] = K @ V2
    return out[:, 0] if squeeze else out


def degrees(X, sigma, rows=None, nthreads=0, kernel="gauss"):
    """deg(x_i) = sum_{j != i} K(x_i - x_j)  (Sec. 2, D = diag(W 1))."""
    n = np.asarray(X).shape[0]
    return W_apply(X, sigma, np.ones(n), rows=rows, nthreads=nthreads, kernel=kernel)


def A_apply(X, sigma, V, deg=None, nthreads=0, kernel="gauss"):
    """D^{-1/2} W D^{-1/2} V, the matrix I - L_sym of one layer (Sec. 2)."""
    if deg is None:
        deg = degrees(X, sigma, nthreads=nthreads, kernel=kernel)
    s = 1.0 / np.sqrt(deg)
    V = np.asarray(V, dtype=np.float64)
    sv = s[:, None] * V.reshape(V.shape[0], -1)
    out = s[:, None] * W_apply(X, sigma, sv, nthreads=nthreads, kernel=kernel)
    return out[:, 0] if V.ndim == 1 else out


def multilayer_A_apply(layers, sigmas, V, degs=None, nthreads=0, kernel="gauss"):
    """(1/T) sum_t D_t^{-1/2} W_t D_t^{-1/2} V  =  (I - L_1) V   (Eq. I-L_1)."""
    T = len(layers)
    acc = None
    for t in range(T):
        y = A_apply(layers[t], sigmas[t], V, None if degs is None else degs[t], nthreads, kernel)
        acc = y if acc is None else acc + y
    return acc / T


def multilayer_W_apply(layers, sigmas, V, nthreads=0, kernel="gauss"):
    """(1/T) sum_t W_t V  (the raw multilayer weight product)."""
    T = len(layers)
    acc = None
    for t in range(T):
        y = W_apply(layers[t], sigmas[t], V, nthreads=nthreads, kernel=kernel)
        acc = y if acc is None else acc + y
    return acc / T


def L_sym_from_W(W):
    """L_sym = I - D^{-1/2} W D^{-1/2}, D = diag(W 1) (Sec. 2), for a given
    symmetric weight matrix with zero diagonal."""
    W = np.asarray(W, dtype=np.float64)
    s = 1.0 / np.sqrt(W.sum(axis=1))
    return np.eye(W.shape[0]) - (s[:, None] * W) * s[None, :]


def L_sym_dense(X, sigma, kernel="gauss"):
    """Dense L_sym = I - D^{-1/2} W D^{-1/2} (Sec. 2).  Small n only."""
    return L_sym_from_W(weight_matrix(X, sigma, kernel))


def shift_delta(p):
    """delta = log(1+|p|) for p < 0 and 0 for p > 0 (Sec. 2, footnote on the shift)."""
    if p == 0:
        raise ValueError("p = 0 is not covered by the power mean definition used here")
    return float(np.log1p(abs(p))) if p < 0 else 0.0


def power_mean_p_dense(layers, sigmas, p, kernel="gauss"):
    """L_{p,delta}^p = (1/T) sum_t (L_sym^(t) + delta I)^p  (Eq. L_p_delta_power_p).

    The matrix power of each symmetric layer term is formed through its
    eigendecomposition, f(A) = Phi f(Lambda) Phi^T (Sec. 2).  `kernel` is one
    kernel name for every layer or a list with one per layer.
    """
    T = len(layers)
    kernels = [kernel] * T if isinstance(kernel, str) else list(kernel)
    return power_mean_of_laplacians([L_sym_dense(layers[t], sigmas[t], kernels[t]) for t in range(T)], p)


def power_mean_of_laplacians(Ls, p):
    """(1/T) sum_t (L_t + delta I)^p for given symmetric layer Laplacians L_t
    (Eq. L_p_delta_power_p; delta = log(1+|p|) for p < 0, 0 for p > 0, Sec. 2),
    each power through the layer's eigendecomposition.  For p > 0 the
    eigenvalues of the positive semi-definite L_t are clipped at 0 against
    rounding."""
    delta = shift_delta(p)
    M = None
    for L in Ls:
        lam, Phi = np.linalg.eigh(np.asarray(L, dtype=np.float64) + delta * np.eye(L.shape[0]))
        if p < 0 and lam.min() <= 0:
            raise ValueError("shifted Laplacian is not positive definite")
        lam = np.maximum(lam, 0.0) if p > 0 else lam
        F = (Phi * lam ** p) @ Phi.T
        M = F if M is None else M + F
    return 0.5 * (M + M.T) / len(Ls)
