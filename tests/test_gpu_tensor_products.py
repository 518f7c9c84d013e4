"""The eigensolvers' dense products on the fp16 tensor cores (tcgen05),
FP64-exact through 8-bit slices of the operands (the error-free splitting of
Ozaki, Ogita, Oishi and Rump): the Gram A^T B and the update Y -= A M against
references in extended precision, entry by entry within a few units of 2^-53
times sum_i |a_i||b_i| (the accuracy of an FP64 product) plus the resolution
of A's fixed scale (64-bit fixed point below 2: 2^-62 per unit of the other
factor), and the eigensolvers' results with the products on the tensor
cores and in double-word FP32 against the same solves on the FP64 pipe."""
import numpy as np
import pytest
import torch

from paper_2007_05239_gb300 import _lib as ml
from paper_2007_05239_gb300 import workloads

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def orthonormal(n, r, seed):
    Q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((n, r)))
    return Q


@pytest.mark.parametrize("n,rc,cb", [(1000, 1, 1), (70_001, 40, 8), (300_000, 21, 1), (4097, 48, 5), (129, 17, 3)])
def test_block_gram_is_fp64_accurate(n, rc, cb):
    rng = np.random.default_rng(rc * 1000 + cb)
    A = orthonormal(n, rc, rc)
    B = rng.uniform(-1.5, 1.5, (n, cb)) * rng.uniform(0, 1, (1, cb))
    B[:, 0] *= 1e-9                                   # a tiny column: absolute accuracy still holds
    G = ml.ml_block_gram(dev(A), dev(B)).cpu().numpy()
    ref = (A.astype(np.longdouble).T @ B.astype(np.longdouble)).astype(np.float64)
    bound = 4 * U * (np.abs(A).T @ np.abs(B)) + 2.0 ** -62 * np.abs(B).sum(0)[None, :]
    err = np.abs(G - ref)
    assert (err <= bound).all(), float((err / bound).max())
    # no worse than a plain FP64 product, column by column
    f64 = np.abs(A.T @ B - ref)
    assert (err.max(0) <= 4 * np.maximum(f64.max(0), U * (np.abs(A).T @ np.abs(B)).max(0))).all()


def test_block_gram_on_strided_rows():
    # the point-major basis of the block solver: rows of ld = ncv + b doubles
    n, ld, rc, cb = 50_000, 40, 32, 8
    X = np.random.default_rng(3).uniform(-1, 1, (n, ld))
    Xd = dev(X)
    G = ml.ml_block_gram(Xd[:, :rc], Xd[:, rc:rc + cb]).cpu().numpy()
    ref = (X[:, :rc].astype(np.longdouble).T @ X[:, rc:rc + cb].astype(np.longdouble)).astype(np.float64)
    bound = 4 * U * (np.abs(X[:, :rc]).T @ np.abs(X[:, rc:rc + cb])) + 2.0 ** -62 * np.abs(X[:, rc:rc + cb]).sum(0)
    assert (np.abs(G - ref) <= bound).all()


@pytest.mark.parametrize("sub", [False, True])
@pytest.mark.parametrize("n,rc,cb", [(100_003, 40, 8), (1000, 1, 1), (7777, 21, 27), (128, 48, 3)])
def test_block_update_is_fp64_accurate(n, rc, cb, sub):
    rng = np.random.default_rng(n + rc)
    A = orthonormal(n, rc, n % 97)
    M = rng.standard_normal((rc, cb)) * 10.0 ** rng.uniform(-9, 3, (1, cb))   # columns of any magnitude
    Y0 = rng.standard_normal((n, cb))
    Y = dev(Y0)
    ml.ml_block_update(dev(A), dev(M), Y, sub=sub)
    got = Y.cpu().numpy()
    prod = (A.astype(np.longdouble) @ M.astype(np.longdouble))
    ref = ((Y0.astype(np.longdouble) - prod) if sub else prod).astype(np.float64)
    bound = 4 * U * (np.abs(A) @ np.abs(M) + (np.abs(Y0) if sub else 0)) + 2.0 ** -62 * np.abs(M).sum(0)[None, :]
    err = np.abs(got - ref)
    assert (err <= bound).all(), float((err / bound).max())


def test_block_update_in_place_other_columns():
    # Y = A itself, writing columns that are not read (the Ritz step writes a
    # second basis; the block step updates the block that follows the basis)
    n, rc, cb = 20_000, 16, 4
    X = np.random.default_rng(9).uniform(-1, 1, (n, rc + cb))
    M = np.random.default_rng(10).standard_normal((rc, cb))
    Xd = dev(X)
    ml.ml_block_update(Xd[:, :rc], dev(M), Xd[:, rc:], sub=True)
    ref = (X[:, rc:].astype(np.longdouble) - X[:, :rc].astype(np.longdouble) @ M.astype(np.longdouble))
    assert np.abs(Xd.cpu().numpy()[:, rc:] - ref.astype(np.float64)).max() <= 1e-14
    assert np.array_equal(Xd.cpu().numpy()[:, :rc], X[:, :rc])


def test_operand_beyond_the_fixed_scale_is_refused():
    A = dev(np.full((1000, 4), 3.0))
    B = dev(np.ones((1000, 2)))
    with pytest.raises(ml.MLError) as e:
        ml.ml_block_gram(A, B)
    assert e.value.status == ml.ML_ERR_DOMAIN
    with pytest.raises(ml.MLError):
        ml.ml_block_gram(dev(np.ones((100, 49))), B[:100])   # rc beyond 48


def _solve_kinds(fn):
    out = {}
    for kind in ("fp64", "dword", "tensor"):
        ml.ml_set_dense_products(kind)
        try:
            out[kind] = fn()
        finally:
            ml.ml_set_dense_products("dword")
    return out


def test_eigensolvers_same_results_for_every_kind_of_product():
    # the basis products on the FP64 pipe, in double-word FP32 (the default)
    # and on the tensor cores: the same eigenpairs to well within the
    # eigensolver's tolerance
    n = 6000
    layers = [workloads.uniform_cube(n, 3, seed=500), workloads.uniform_cube(n, 2, seed=501)]
    plans = [ml.ml_fastsum_plan(dev(L), s, prec="f64", target_rel_err=1e-12) for L, s in zip(layers, [0.1, 0.08])]
    k = 8

    def combined():
        V = torch.empty(n * k, dtype=torch.float64, device="cuda")
        lam, nconv, st = ml.ml_lanczos_eigs(plans, k, p=1.0, tol=1e-11, seed=4, evecs=V)
        return lam, V.cpu().numpy().reshape(k, n), st

    def per_layer():
        V = torch.empty(2 * n * k, dtype=torch.float64, device="cuda")
        lam, nconv, st = ml.ml_lanczos_eigs_layers(plans, k, block=8, tol=1e-11, seed=4, evecs=V)
        return lam, V.cpu().numpy().reshape(2, k, n), st

    for fn in (combined, per_layer):
        res = _solve_kinds(fn)
        l0, v0, s0 = res["fp64"]
        assert s0 == ml.ML_OK
        for kind in ("dword", "tensor"):
            l1, v1, s1 = res[kind]
            assert s1 == ml.ML_OK
            assert np.abs(l1 - l0).max() <= 1e-12, (kind, l1, l0)
            # the same Krylov process up to rounding: the vectors agree closely
            assert np.abs(np.abs((v1 * v0).sum(-1)) - 1).max() <= 1e-9, kind
