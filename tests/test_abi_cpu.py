"""The C-ABI library builds, loads and exports every symbol include/ml_fastsum.h
declares; argument checks answer without touching a GPU."""
import ctypes
import os
import re

import pytest

from paper_2007_05239_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ml_fastsum.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ml_[a-z_]+)\s*\(", src)))


def test_header_and_binding_agree():
    assert _declared() == sorted(_lib.EXPORTS)


def test_library_exports_every_symbol():
    lib = _lib.load()
    for name in _declared():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_argument_errors_without_gpu():
    lib = _lib.load()
    h = ctypes.c_void_p()
    assert lib.ml_fastsum_plan(ctypes.byref(h), None, 10, 3, 0.1, 0, 0, 0.0, 0, 1, 0.0, None) == _lib.ML_ERR_ARG
    assert b"null" in lib.ml_last_error()
    dummy = ctypes.c_double(0.0)
    p = ctypes.addressof(dummy)
    assert lib.ml_fastsum_plan(ctypes.byref(h), p, 10, 4, 0.1, 0, 0, 0.0, 0, 1, 0.0, None) == _lib.ML_ERR_ARG
    assert lib.ml_fastsum_plan(ctypes.byref(h), p, 10, 3, -1.0, 0, 0, 0.0, 0, 1, 0.0, None) == _lib.ML_ERR_ARG
    assert lib.ml_fastsum_plan(ctypes.byref(h), p, 10, 3, 0.1, 7, 0, 0.0, 0, 1, 0.0, None) == _lib.ML_ERR_ARG
    assert lib.ml_fastsum_plan(ctypes.byref(h), p, 10, 3, 0.1, 0, 9, 0.0, 0, 1, 0.0, None) == _lib.ML_ERR_ARG
    assert lib.ml_fastsum_plan(ctypes.byref(h), p, 10, 3, 0.1, 0, 0, 0.25, 0, 1, 0.0, None) == _lib.ML_ERR_ARG
    assert lib.ml_fastsum_apply(None, 1, None, 1, None, 0, None) == _lib.ML_ERR_ARG
    ev = (ctypes.c_double * 4)()
    assert lib.ml_lanczos_eigs(None, 1, 2, 1.0, 0.0, 0, 1, 0, ev, None, None, None) == _lib.ML_ERR_ARG
    assert lib.ml_plan_destroy(None) == _lib.ML_OK


@pytest.mark.skipif(os.environ.get("CUDA_VISIBLE_DEVICES", None) not in (None, ""), reason="GPU may be visible")
def test_no_cpu_fallback():
    # Without a usable GPU a well-formed call fails with ML_ERR_CUDA instead of
    # computing anything on the CPU.
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    lib = _lib.load()
    h = ctypes.c_void_p()
    pts = (ctypes.c_double * 30)(*([0.1 * i for i in range(30)]))
    st = lib.ml_fastsum_plan(ctypes.byref(h), ctypes.addressof(pts), 10, 3, 0.1, 0, 0, 0.0, 0, 1, 0.0, None)
    assert st == _lib.ML_ERR_CUDA
