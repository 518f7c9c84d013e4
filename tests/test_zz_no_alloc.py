"""ml_fastsum_apply_noalloc: the product without any device allocation.

Some callers cannot call cudaMalloc while they run the product (a framework
allocator that owns the device, latency-bound loops, builds that forbid
allocation after start-up).  This entry point takes all its scratch from a
fixed 32 MiB device array inside the library; these tests check, through the
C ABI, that its output equals the allocating entry point's on two calls in a
row, that on fresh plans it runs first without changing the plans' or the
device's memory, and that oversized requests and host buffers are rejected.  The file is
named so that pytest collects it last.
"""
import numpy as np
import pytest
import torch

from paper_2007_05239_gb300 import _lib as ml
from paper_2007_05239_gb300 import workloads

pytestmark = pytest.mark.gpu


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_noalloc_matches_apply_two_calls(prec):
    n = 6000
    rng = np.random.default_rng(3)
    layers = [workloads.uniform_cube(n, 3, seed=200), rng.uniform(0, 1, (n, 2))]
    plans = [ml.ml_fastsum_plan(dev(L), s, prec=prec) for L, s in zip(layers, [0.1, 0.15])]
    for call in range(2):
        X = dev(rng.uniform(-1, 1, (n, 5)))   # passes of 4 + 1 vectors
        ref = torch.empty_like(X)
        got = torch.full_like(X, np.nan)
        ml.ml_fastsum_apply(plans, X, ref, mode="normalized")
        ml.ml_fastsum_apply_noalloc(plans, X, got, mode="normalized")
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.isfinite(g).all()
        # the same kernels on the same inputs: equal up to FP64 rounding
        assert np.abs(g - r).max() <= 1e-13 * np.abs(r).max(), f"call {call}"


def test_noalloc_first_on_fresh_plans_allocates_nothing():
    # Fresh plans whose workspace was never grown: the no-alloc product runs
    # first, and neither the plans' device memory nor the device's free memory
    # changes across the call (with the device synchronised on both sides).
    # The allocating product afterwards gives the same values.
    n = 5000
    rng = np.random.default_rng(8)
    X = dev(rng.uniform(0, 1, (n, 3)))
    got = torch.full_like(X, np.nan)
    ref = torch.empty_like(X)
    # one call on other plans of the same shapes first: the CUDA runtime loads
    # kernels (and the library's static array) lazily, on first use, and that
    # loading takes device memory once per process
    warm = [ml.ml_fastsum_plan(dev(workloads.uniform_cube(n, dd, seed=230 + dd)), s, prec="f64")
            for dd, s in ((3, 0.1), (2, 0.12))]
    ml.ml_fastsum_apply_noalloc(warm, X, got, mode="normalized")
    for pl in warm:
        pl.destroy()
    layers = [workloads.uniform_cube(n, 3, seed=220), workloads.uniform_cube(n, 2, seed=221)]
    plans = [ml.ml_fastsum_plan(dev(L), s, prec="f64") for L, s in zip(layers, [0.1, 0.12])]
    got.fill_(np.nan)
    torch.cuda.synchronize()
    owned = [pl.info["device_bytes"] for pl in plans]
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        ml.ml_fastsum_apply_noalloc(plans, X, got, mode="normalized")
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert [pl.info["device_bytes"] for pl in plans] == owned
    assert free1 == free0
    ml.ml_fastsum_apply(plans, X, ref, mode="normalized")
    torch.cuda.synchronize()
    r, g = ref.cpu().numpy(), got.cpu().numpy()
    assert np.isfinite(g).all()
    assert np.abs(g - r).max() <= 1e-13 * np.abs(r).max()


def test_noalloc_per_layer_and_raw():
    n = 3000
    L = [workloads.uniform_cube(n, 2, seed=210 + t) for t in range(2)]
    plans = [ml.ml_fastsum_plan(dev(x), 0.1, prec="f64") for x in L]
    X = dev(np.random.default_rng(4).uniform(0, 1, (2, n, 1)))
    ref, got = torch.empty_like(X), torch.empty_like(X)
    ml.ml_fastsum_apply(plans, X, ref, mode="raw", per_layer=True)
    ml.ml_fastsum_apply_noalloc(plans, X, got, mode="raw", per_layer=True)
    assert torch.allclose(got, ref, rtol=1e-13, atol=0)


def test_noalloc_rejects_oversize_and_host_buffers():
    # 3e6 FP64 points need ~3000 subproblem tiles: far more than 32 MiB
    n = 3_000_000
    big = np.random.default_rng(5).uniform(0, 1, (n, 3))
    plan = ml.ml_fastsum_plan(dev(big), 0.05, prec="f64")
    X = dev(np.ones((n, 1)))
    Y = torch.empty_like(X)
    with pytest.raises(ml.MLError) as e:
        ml.ml_fastsum_apply_noalloc([plan], X, Y)
    assert e.value.status == ml.ML_ERR_ARG and "static limit" in str(e.value)
    small = ml.ml_fastsum_plan(dev(workloads.uniform_cube(500, 3, seed=6)), 0.1, prec="f64")
    xh = np.ones((500, 1))
    with pytest.raises(ml.MLError):
        ml.ml_fastsum_apply_noalloc([small], xh, np.empty((500, 1)))
