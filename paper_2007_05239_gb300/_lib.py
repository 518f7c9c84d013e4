"""Thin Python binding of the C ABI in include/ml_fastsum.h.

Argument marshalling only: every step of the fast summation and of the
eigensolver runs in the CUDA library libmlfastsum.so.  There is no CPU
fallback; without the built library every call raises.
"""
from __future__ import annotations

import ctypes
import os
import warnings

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmlfastsum.so")

ML_OK, ML_ERR_ARG, ML_ERR_CUDA, ML_ERR_OOM, ML_ERR_DOMAIN, ML_ERR_DEGREE, ML_ERR_BREAKDOWN, \
    ML_ERR_TIMEOUT, ML_WARN_NOT_CONVERGED = range(9)
STATUS_NAMES = ["ML_OK", "ML_ERR_ARG", "ML_ERR_CUDA", "ML_ERR_OOM", "ML_ERR_DOMAIN", "ML_ERR_DEGREE",
                "ML_ERR_BREAKDOWN", "ML_ERR_TIMEOUT", "ML_WARN_NOT_CONVERGED"]
ML_F32, ML_F64 = 0, 1
ML_KERNEL_GAUSS, ML_KERNEL_LAPLACE = 0, 1
ML_RAW_W, ML_NORMALIZED_A, ML_DEGREE, ML_PER_LAYER = 0, 1, 2, 16
MODES = {"raw": ML_RAW_W, "normalized": ML_NORMALIZED_A, "degree": ML_DEGREE}

# every symbol the header declares
EXPORTS = ["ml_fastsum_plan", "ml_fastsum_plan_ex", "ml_fastsum_plan_autotune", "ml_fastsum_plan_learned",
           "ml_fastsum_plan_many", "ml_dense_plan", "ml_dense_plan_matrix",
           "ml_fastsum_apply",
           "ml_fastsum_apply_noalloc", "ml_direct_sum_rows", "ml_cloud_features", "ml_mlp_create",
           "ml_mlp_param_count", "ml_mlp_get_params", "ml_mlp_set_params", "ml_mlp_set_norm", "ml_mlp_forward",
           "ml_mlp_loss_grad", "ml_mlp_train", "ml_mlp_set_margins", "ml_mlp_destroy", "ml_lanczos_eigs", "ml_lanczos_eigs_layers", "ml_allen_cahn",
           "ml_plan_get_info",
           "ml_plan_copy_table", "ml_plan_destroy", "ml_last_error", "ml_version", "ml_profile_enable",
           "ml_profile_reset", "ml_profile_read", "ml_graph_replays", "ml_measure_peak", "ml_block_gram",
           "ml_block_update", "ml_set_dense_products", "ml_release_cached_memory"]


class MLError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


ML_FEATURES = 9


class PlanParams(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("taps", ctypes.c_int), ("oversampling", ctypes.c_double),
                ("eps_B", ctypes.c_double), ("p_reg", ctypes.c_int), ("prec", ctypes.c_int),
                ("target_rel_err", ctypes.c_double), ("bin", ctypes.c_int), ("kernel", ctypes.c_int),
                ("eps_I", ctypes.c_double)]


class AcParams(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("omega0", ctypes.c_double), ("c", ctypes.c_double),
                ("dt", ctypes.c_double), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("d", ctypes.c_int), ("N", ctypes.c_int), ("m", ctypes.c_int),
                ("n_os", ctypes.c_int), ("L", ctypes.c_int * 3), ("bin", ctypes.c_int), ("nbins", ctypes.c_int),
                ("nsub", ctypes.c_int), ("prec", ctypes.c_int), ("domain", ctypes.c_int), ("p_reg", ctypes.c_int),
                ("eps_B", ctypes.c_double), ("sigma", ctypes.c_double), ("sigma_s", ctypes.c_double),
                ("scale", ctypes.c_double), ("center", ctypes.c_double * 3), ("target_rel_err", ctypes.c_double),
                ("deg_min", ctypes.c_double), ("deg_max", ctypes.c_double), ("device_bytes", ctypes.c_int64),
                ("applied_vectors", ctypes.c_int64), ("taps", ctypes.c_int), ("dense", ctypes.c_int),
                ("kernel", ctypes.c_int), ("eps_I", ctypes.c_double), ("kernel_err", ctypes.c_double),
                ("near_pairs", ctypes.c_int64)]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if isinstance(v, ctypes.Array) else v
        return out


_LIB = None


def load():
    """Load libmlfastsum.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run paper_2007_05239_gb300.build.build() first")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    lib.ml_fastsum_plan.restype = ctypes.c_int
    lib.ml_fastsum_plan.argtypes = [ctypes.POINTER(P), P, ctypes.c_int64, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_double, P]
    lib.ml_fastsum_apply.restype = ctypes.c_int
    lib.ml_fastsum_apply.argtypes = [P, ctypes.c_int, P, ctypes.c_int, P, ctypes.c_int, P]
    lib.ml_fastsum_apply_noalloc.restype = ctypes.c_int
    lib.ml_fastsum_apply_noalloc.argtypes = [P, ctypes.c_int, P, ctypes.c_int, P, ctypes.c_int, P]
    lib.ml_lanczos_eigs.restype = ctypes.c_int
    lib.ml_lanczos_eigs.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_uint64, P, P, P, P]
    lib.ml_lanczos_eigs_layers.restype = ctypes.c_int
    lib.ml_lanczos_eigs_layers.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_uint64, P, P, P, P]
    lib.ml_allen_cahn.restype = ctypes.c_int
    lib.ml_allen_cahn.argtypes = [P, P, ctypes.c_int64, ctypes.c_int, P, ctypes.c_int, P, P, P, P, P, P]
    lib.ml_plan_get_info.restype = ctypes.c_int
    lib.ml_plan_get_info.argtypes = [P, ctypes.POINTER(PlanInfo)]
    lib.ml_plan_copy_table.restype = ctypes.c_int
    lib.ml_plan_copy_table.argtypes = [P, ctypes.c_int, P, ctypes.c_int64]
    lib.ml_plan_destroy.restype = ctypes.c_int
    lib.ml_plan_destroy.argtypes = [P]
    lib.ml_last_error.restype = ctypes.c_char_p
    lib.ml_last_error.argtypes = []
    lib.ml_version.restype = ctypes.c_char_p
    lib.ml_version.argtypes = []
    lib.ml_fastsum_plan_ex.restype = ctypes.c_int
    lib.ml_fastsum_plan_ex.argtypes = [ctypes.POINTER(P), P, ctypes.c_int64, ctypes.c_int, ctypes.c_double,
                                       ctypes.POINTER(PlanParams), P]
    lib.ml_fastsum_plan_many.restype = ctypes.c_int
    lib.ml_fastsum_plan_many.argtypes = [P, P, ctypes.c_int64, P, P, P, ctypes.c_int, P]
    lib.ml_dense_plan.restype = ctypes.c_int
    lib.ml_dense_plan.argtypes = [ctypes.POINTER(P), P, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                  P]
    lib.ml_dense_plan_matrix.restype = ctypes.c_int
    lib.ml_dense_plan_matrix.argtypes = [ctypes.POINTER(P), P, ctypes.c_int64, ctypes.c_int, P]
    lib.ml_fastsum_plan_autotune.restype = ctypes.c_int
    lib.ml_fastsum_plan_autotune.argtypes = [ctypes.POINTER(P), P, ctypes.c_int64, ctypes.c_int, ctypes.c_double, P,
                                             ctypes.c_int, P, P]
    lib.ml_fastsum_plan_learned.restype = ctypes.c_int
    lib.ml_fastsum_plan_learned.argtypes = [ctypes.POINTER(P), P, ctypes.c_int64, ctypes.c_int, ctypes.c_double,
                                            ctypes.c_int, ctypes.c_double, P, ctypes.c_double, P, P]
    lib.ml_direct_sum_rows.restype = ctypes.c_int
    lib.ml_direct_sum_rows.argtypes = [P, ctypes.c_int64, ctypes.c_int, ctypes.c_double, P, P, ctypes.c_int64, P, P]
    lib.ml_cloud_features.restype = ctypes.c_int
    lib.ml_cloud_features.argtypes = [P, ctypes.c_int64, ctypes.c_int, ctypes.c_double, P, P]
    lib.ml_mlp_create.restype = ctypes.c_int
    lib.ml_mlp_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64]
    lib.ml_mlp_param_count.restype = ctypes.c_int64
    lib.ml_mlp_param_count.argtypes = [P]
    for nm in ("ml_mlp_get_params", "ml_mlp_set_params"):
        getattr(lib, nm).restype = ctypes.c_int
        getattr(lib, nm).argtypes = [P, P, ctypes.c_int64]
    lib.ml_mlp_set_norm.restype = ctypes.c_int
    lib.ml_mlp_set_norm.argtypes = [P, P, P, P, P]
    lib.ml_mlp_forward.restype = ctypes.c_int
    lib.ml_mlp_forward.argtypes = [P, P, ctypes.c_int, P]
    lib.ml_mlp_loss_grad.restype = ctypes.c_int
    lib.ml_mlp_loss_grad.argtypes = [P, P, P, ctypes.c_int, P, P]
    lib.ml_mlp_train.restype = ctypes.c_int
    lib.ml_mlp_train.argtypes = [P, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_float, P]
    lib.ml_mlp_set_margins.restype = ctypes.c_int
    lib.ml_mlp_set_margins.argtypes = [P, P, ctypes.c_int]
    lib.ml_mlp_destroy.restype = ctypes.c_int
    lib.ml_mlp_destroy.argtypes = [P]
    lib.ml_graph_replays.restype = ctypes.c_int64
    lib.ml_graph_replays.argtypes = []
    lib.ml_measure_peak.restype = ctypes.c_int
    lib.ml_block_gram.restype = ctypes.c_int
    lib.ml_block_gram.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p,
                                  ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    lib.ml_block_update.restype = ctypes.c_int
    lib.ml_block_update.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p,
                                    ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p]
    lib.ml_release_cached_memory.restype = ctypes.c_int
    lib.ml_release_cached_memory.argtypes = []
    lib.ml_set_dense_products.restype = ctypes.c_int
    lib.ml_set_dense_products.argtypes = [ctypes.c_int]
    lib.ml_measure_peak.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    lib.ml_profile_enable.restype = ctypes.c_int
    lib.ml_profile_enable.argtypes = [ctypes.c_int]
    lib.ml_profile_reset.restype = ctypes.c_int
    lib.ml_profile_reset.argtypes = []
    lib.ml_profile_read.restype = ctypes.c_int
    lib.ml_profile_read.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_int64),
                                    ctypes.POINTER(ctypes.c_double)]
    _LIB = lib
    return lib


def _check(st):
    if st == ML_OK:
        return st
    msg = load().ml_last_error().decode()
    if st == ML_WARN_NOT_CONVERGED:
        warnings.warn(f"ML_WARN_NOT_CONVERGED: {msg}")
        return st
    raise MLError(st, msg)


def _ptr(a):
    """Raw address of a torch tensor or numpy array (contiguous float64)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise ValueError("numpy arrays must be C-contiguous float64")
        return a.ctypes.data
    if a.dtype.__str__() != "torch.float64" or not a.is_contiguous():
        raise ValueError("tensors must be contiguous float64")
    return a.data_ptr()


def _ptr_i32(a):
    """Raw address of a contiguous int32 torch tensor (or None)."""
    if a is None:
        return None
    if a.dtype.__str__() != "torch.int32" or not a.is_contiguous():
        raise ValueError("tensors must be contiguous int32")
    return a.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


class Plan:
    """One layer's plan (owns library memory until destroy())."""

    def __init__(self, handle, n, d):
        self.handle = ctypes.c_void_p(handle)
        self.n = n
        self.d = d

    @property
    def info(self):
        inf = PlanInfo()
        _check(load().ml_plan_get_info(self.handle, ctypes.byref(inf)))
        return inf.as_dict()

    def table(self, which):
        inf = self.info
        H = inf["N"] // 2 + 1
        size = {0: H ** inf["d"], 1: H, 2: inf["n"]}[which]
        out = np.empty(size, dtype=np.float64)
        _check(load().ml_plan_copy_table(self.handle, which, out.ctypes.data, size))
        return out

    def destroy(self):
        if self.handle is not None and self.handle.value:
            load().ml_plan_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def ml_fastsum_plan(points, sigma, N=0, m=0, eps_B=0.0, p_reg=0, prec="f64", target_rel_err=0.0, stream=None):
    """Plan one layer.  `points`: float64 (n, d), a CUDA tensor, or host
    memory (numpy array or CPU tensor) that the library copies to the device."""
    lib = load()
    n, d = int(points.shape[0]), int(points.shape[1])
    h = ctypes.c_void_p()
    pr = {"f32": ML_F32, "f64": ML_F64}[prec] if isinstance(prec, str) else int(prec)
    _check(lib.ml_fastsum_plan(ctypes.byref(h), _ptr(points), n, d, float(sigma), int(N), int(m), float(eps_B),
                               int(p_reg), pr, float(target_rel_err), _stream(stream)))
    return Plan(h.value, n, d)


KERNELS = {"gauss": ML_KERNEL_GAUSS, "laplace": ML_KERNEL_LAPLACE}


def _params(N, taps, oversampling, eps_B, p_reg, prec, target_rel_err, bin, kernel="gauss", eps_I=0.0):
    return PlanParams(int(N), int(taps), float(oversampling), float(eps_B), int(p_reg),
                      {"f32": ML_F32, "f64": ML_F64}[prec] if isinstance(prec, str) else int(prec),
                      float(target_rel_err), int(bin),
                      KERNELS[kernel] if isinstance(kernel, str) else int(kernel), float(eps_I))


def ml_fastsum_plan_ex(points, sigma, N=0, taps=0, oversampling=0.0, eps_B=0.0, p_reg=0, prec="f64",
                       target_rel_err=0.0, bin=0, kernel="gauss", eps_I=0.0, stream=None):
    """Plan one layer with explicit window width / oversampling / bin edge (0 = automatic);
    kernel "gauss" (exp(-r^2/sigma^2)) or "laplace" (exp(-r/sigma), with its near-field radius eps_I)."""
    lib = load()
    n, d = int(points.shape[0]), int(points.shape[1])
    prm = _params(N, taps, oversampling, eps_B, p_reg, prec, target_rel_err, bin, kernel, eps_I)
    h = ctypes.c_void_p()
    _check(lib.ml_fastsum_plan_ex(ctypes.byref(h), _ptr(points), n, d, float(sigma), ctypes.byref(prm),
                                  _stream(stream)))
    return Plan(h.value, n, d)


def ml_fastsum_plan_many(points, sigmas, N=0, taps=0, oversampling=0.0, eps_B=0.0, p_reg=0, prec="f64",
                         target_rel_err=0.0, kernel="gauss", eps_I=0.0, stream=None):
    """Plans of several layers (point tensors or arrays sharing n, device or
    host memory; host points are copied by the library), built concurrently."""
    lib = load()
    T = len(points)
    n = int(points[0].shape[0])
    prm = _params(N, taps, oversampling, eps_B, p_reg, prec, target_rel_err, 0, kernel, eps_I)
    handles = (ctypes.c_void_p * T)()
    ptrs = (ctypes.c_void_p * T)(*[_ptr(x) for x in points])
    dims = (ctypes.c_int * T)(*[int(x.shape[1]) for x in points])
    sig = (ctypes.c_double * T)(*[float(s) for s in sigmas])
    _check(lib.ml_fastsum_plan_many(handles, ptrs, n, dims, sig, ctypes.byref(prm), T, _stream(stream)))
    return [Plan(handles[t], n, dims[t]) for t in range(T)]


def ml_dense_plan(points, sigma, prec="f64", stream=None):
    """Dense layer (W stored, any feature dimension) from device points (n, d)."""
    lib = load()
    n, d = int(points.shape[0]), int(points.shape[1])
    h = ctypes.c_void_p()
    _check(lib.ml_dense_plan(ctypes.byref(h), _ptr(points), n, d, float(sigma),
                             {"f32": ML_F32, "f64": ML_F64}[prec], _stream(stream)))
    return Plan(h.value, n, d)


def ml_dense_plan_matrix(W, prec="f64", stream=None):
    """Dense layer from a given symmetric device weight matrix (n, n) float64."""
    lib = load()
    n = int(W.shape[0])
    h = ctypes.c_void_p()
    _check(lib.ml_dense_plan_matrix(ctypes.byref(h), _ptr(W), n, {"f32": ML_F32, "f64": ML_F64}[prec],
                                    _stream(stream)))
    return Plan(h.value, n, 0)


def ml_fastsum_plan_autotune(points, sigma, nv=1, N=0, taps=0, oversampling=0.0, eps_B=0.0, p_reg=0, prec="f64",
                             target_rel_err=0.0, stream=None):
    """Plan one layer with the bin edge chosen by timing nv-vector products.
    Returns (plan, chosen bin edge)."""
    lib = load()
    n, d = int(points.shape[0]), int(points.shape[1])
    prm = _params(N, taps, oversampling, eps_B, p_reg, prec, target_rel_err, 0)
    h = ctypes.c_void_p()
    chosen = ctypes.c_int(0)
    _check(lib.ml_fastsum_plan_autotune(ctypes.byref(h), _ptr(points), n, d, float(sigma), ctypes.byref(prm),
                                        int(nv), ctypes.byref(chosen), _stream(stream)))
    return Plan(h.value, n, d), chosen.value


def ml_fastsum_plan_learned(points, sigma, model=None, prec="f32", target_rel_err=0.0, margin=2.0, stream=None):
    """Plan with parameters chosen by a trained Mlp (None: the automatic rule).
    Returns (plan, chosen) with chosen = (bandwidth factor, taps, oversampling) or zeros."""
    lib = load()
    n, d = int(points.shape[0]), int(points.shape[1])
    h = ctypes.c_void_p()
    ch = np.zeros(3)
    pr = {"f32": ML_F32, "f64": ML_F64}[prec] if isinstance(prec, str) else int(prec)
    _check(lib.ml_fastsum_plan_learned(ctypes.byref(h), _ptr(points), n, d, float(sigma), pr, float(target_rel_err),
                                       None if model is None else model.handle, float(margin), ch.ctypes.data,
                                       _stream(stream)))
    return Plan(h.value, n, d), tuple(ch)


def ml_direct_sum_rows(points, sigma, v, rows, out=None, stream=None):
    """Exact (W v)[rows] on the GPU.  points (n, d), v (n,) float64 CUDA; rows int64 CUDA."""
    import torch
    lib = load()
    n, d = int(points.shape[0]), int(points.shape[1])
    if out is None:
        out = torch.empty(int(rows.shape[0]), dtype=torch.float64, device=points.device)
    _check(lib.ml_direct_sum_rows(_ptr(points), n, d, float(sigma), _ptr(v), rows.data_ptr(), int(rows.shape[0]),
                                  _ptr(out), _stream(stream)))
    return out


def ml_cloud_features(points, sigma, stream=None):
    lib = load()
    f = np.zeros(ML_FEATURES, dtype=np.float32)
    _check(lib.ml_cloud_features(_ptr(points), int(points.shape[0]), int(points.shape[1]), float(sigma),
                                 f.ctypes.data, _stream(stream)))
    return f


class Mlp:
    """The library's FP32 MLP (n_in -> h -> h -> n_out, tanh), on the GPU."""

    def __init__(self, n_in, hidden, n_out, seed=0):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.ml_mlp_create(ctypes.byref(h), int(n_in), int(hidden), int(n_out), ctypes.c_uint64(seed)))
        self.handle = h
        self.n_in, self.hidden, self.n_out = n_in, hidden, n_out

    @property
    def nparam(self):
        return int(load().ml_mlp_param_count(self.handle))

    def get_params(self):
        p = np.empty(self.nparam, dtype=np.float32)
        _check(load().ml_mlp_get_params(self.handle, p.ctypes.data, p.size))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(load().ml_mlp_set_params(self.handle, p.ctypes.data, p.size))

    def set_norm(self, in_mean, in_std, out_mean, out_std):
        arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (in_mean, in_std, out_mean, out_std)]
        _check(load().ml_mlp_set_norm(self.handle, *[a.ctypes.data for a in arrs]))
        self._norm = arrs

    def forward(self, X):
        X = np.ascontiguousarray(X, dtype=np.float32)
        Y = np.empty((X.shape[0], self.n_out), dtype=np.float32)
        _check(load().ml_mlp_forward(self.handle, X.ctypes.data, X.shape[0], Y.ctypes.data))
        return Y

    def loss_grad(self, X, Y):
        X = np.ascontiguousarray(X, dtype=np.float32)
        Y = np.ascontiguousarray(Y, dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        g = np.empty(self.nparam, dtype=np.float32)
        _check(load().ml_mlp_loss_grad(self.handle, X.ctypes.data, Y.ctypes.data, X.shape[0], loss.ctypes.data,
                                       g.ctypes.data))
        return float(loss[0]), g

    def train(self, X, Y, epochs, lr=1e-3):
        X = np.ascontiguousarray(X, dtype=np.float32)
        Y = np.ascontiguousarray(Y, dtype=np.float32)
        losses = np.empty(epochs, dtype=np.float32)
        _check(load().ml_mlp_train(self.handle, X.ctypes.data, Y.ctypes.data, X.shape[0], int(epochs), float(lr),
                                   losses.ctypes.data))
        return losses

    def set_margins(self, margins):
        """Per-bandwidth-factor safety margins of the learned planner (3 values)."""
        m = np.ascontiguousarray(margins, dtype=np.float64)
        _check(load().ml_mlp_set_margins(self.handle, m.ctypes.data, int(m.size)))

    def destroy(self):
        if self.handle is not None and self.handle.value:
            load().ml_mlp_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def _handles(layers):
    arr = (ctypes.c_void_p * len(layers))(*[p.handle.value for p in layers])
    return arr


def ml_fastsum_apply(layers, X, Y, mode="normalized", per_layer=False, stream=None):
    """Y <- operator(X).  X, Y: float64 torch tensors (CUDA or CPU) or numpy arrays, shape (n, b)
    or (T, n, b) with per_layer.  Y is overwritten."""
    lib = load()
    md = MODES[mode] if isinstance(mode, str) else int(mode)
    if per_layer:
        md |= ML_PER_LAYER
    b = 1 if len(Y.shape) == (2 if per_layer else 1) else int(Y.shape[-1])
    arr = _handles(layers)
    _check(lib.ml_fastsum_apply(arr, len(layers), _ptr(X), b, _ptr(Y), md, _stream(stream)))
    return Y


def ml_fastsum_apply_noalloc(layers, X, Y, mode="normalized", per_layer=False, stream=None):
    """As ml_fastsum_apply, without device allocation (static scratch; device X and Y only)."""
    lib = load()
    md = MODES[mode] if isinstance(mode, str) else int(mode)
    if per_layer:
        md |= ML_PER_LAYER
    b = 1 if len(Y.shape) == (2 if per_layer else 1) else int(Y.shape[-1])
    arr = _handles(layers)
    _check(lib.ml_fastsum_apply_noalloc(arr, len(layers), _ptr(X), b, _ptr(Y), md, _stream(stream)))
    return Y


def ml_lanczos_eigs(layers, k, p=1.0, tol=0.0, maxit=0, seed=0, evecs=None, stream=None, block=1):
    """k smallest eigenpairs of L_1 (p=1) or L_{p,delta} (p < 0, e.g. -1 or -10).

    evecs: None, or a float64 buffer with n*k elements (CUDA or CPU) that
    receives the eigenvectors column-major.  Returns (evals, nconv, status)."""
    lib = load()
    ev = np.empty(k, dtype=np.float64)
    nconv = ctypes.c_int(0)
    arr = _handles(layers)
    st = lib.ml_lanczos_eigs(arr, len(layers), int(k), float(p), float(tol), int(maxit), int(block),
                             ctypes.c_uint64(seed), ev.ctypes.data, _ptr(evecs), ctypes.byref(nconv),
                             _stream(stream))
    _check(st)
    return ev, nconv.value, st


def ml_lanczos_eigs_layers(layers, k, block=8, tol=0.0, maxit=0, seed=0, evecs=None, stream=None, ncv=0):
    """For every layer separately, the k smallest eigenpairs of its L_sym,
    all layers advancing together by block Lanczos with `block` vectors.

    evecs: None, or a float64 buffer with T*n*k elements (CUDA or CPU): block
    t holds layer t's eigenvectors column-major.  Returns (evals (T x k),
    nconv (T), status)."""
    lib = load()
    T = len(layers)
    ev = np.empty((T, k), dtype=np.float64)
    nconv = np.zeros(T, dtype=np.int32)
    arr = _handles(layers)
    st = lib.ml_lanczos_eigs_layers(arr, T, int(k), float(tol), int(maxit), int(block), int(ncv), ctypes.c_uint64(seed),
                                    ev.ctypes.data, _ptr(evecs), nconv.ctypes.data, _stream(stream))
    _check(st)
    return ev, nconv, st


def ml_allen_cahn(Phi, lam, labels, m, eps=0.005, omega0=1000.0, c=0.0, dt=0.01, tol=1e-6, max_iter=500, U=None,
                  pred=None, stream=None):
    """Class scores by the graph Allen-Cahn scheme (Alg. 2) from eigenpairs.

    Phi: CUDA float64 buffer of n*k (column-major n x k); lam: k eigenvalues;
    labels: CUDA int32 n (class or -1).  Returns (U (n x m CUDA float64),
    pred (n CUDA int32 or the given buffer), iterations, last relative change)."""
    import torch
    lib = load()
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    k = int(lam.size)
    n = int(labels.numel())
    if U is None:
        U = torch.empty(n * m, dtype=torch.float64, device=labels.device)
    if pred is None:
        pred = torch.empty(n, dtype=torch.int32, device=labels.device)
    prm = AcParams(float(eps), float(omega0), float(c), float(dt), float(tol), int(max_iter))
    iters = ctypes.c_int(0)
    chg = ctypes.c_double(0.0)
    _check(lib.ml_allen_cahn(_ptr(Phi), lam.ctypes.data, n, k, _ptr_i32(labels), int(m), ctypes.byref(prm), _ptr(U),
                             _ptr_i32(pred), ctypes.byref(iters), ctypes.byref(chg), _stream(stream)))
    return U, pred, iters.value, chg.value


def ml_graph_replays():
    """CUDA-graph replays of captured solver iterations since the library was loaded."""
    return int(load().ml_graph_replays())


def _ptr_rows(a):
    """Address of a float64 CUDA tensor whose rows may be strided (unit column stride)."""
    if str(a.dtype) != "torch.float64" or a.dim() != 2 or (a.shape[1] > 1 and a.stride(1) != 1):
        raise ValueError("tensors must be 2-d float64 with unit column stride")
    return a.data_ptr()


def ml_block_gram(A, B, stream=None):
    """G = A^T B on the tensor cores (FP64-exact slices): A (n, rc), B (n, cb)
    float64 CUDA tensors with unit column stride; returns G (rc, cb)."""
    import torch
    n, rc = int(A.shape[0]), int(A.shape[1])
    cb = int(B.shape[1])
    G = torch.empty(rc, cb, dtype=torch.float64, device=A.device)
    _check(load().ml_block_gram(_ptr_rows(A), n, rc, int(A.stride(0)), _ptr_rows(B), cb, int(B.stride(0)),
                                _ptr(G), _stream(stream)))
    return G


def ml_block_update(A, M, Y, sub=False, stream=None):
    """Y = A M (or Y -= A M) on the tensor cores: A (n, rc), M (rc, cb), Y (n, cb)."""
    n, rc = int(A.shape[0]), int(A.shape[1])
    cb = int(M.shape[1])
    _check(load().ml_block_update(_ptr_rows(A), n, rc, int(A.stride(0)), _ptr(M), cb, _ptr_rows(Y),
                                  int(Y.stride(0)), 1 if sub else 0, _stream(stream)))
    return Y


def ml_release_cached_memory():
    """Return the library's cached device blocks of the current device to the driver."""
    _check(load().ml_release_cached_memory())


DENSE = {"fp64": 0, "dword": 1, "tensor": 2}


def ml_set_dense_products(kind="dword"):
    """The eigensolvers' basis products: "fp64", "dword" (default) or "tensor"."""
    _check(load().ml_set_dense_products(DENSE[kind] if isinstance(kind, str) else int(kind)))


PEAKS = {"fp32": 0, "fp64": 1, "smem_atomic": 2}


def ml_measure_peak(what, stream=None):
    """Measured throughput of one resource: "fp32" / "fp64" FMA pipes in
    TFLOP/s, "smem_atomic" conflict-free 32-bit shared atomics in 1e12/s."""
    rate = ctypes.c_double()
    _check(load().ml_measure_peak(PEAKS[what], ctypes.byref(rate), _stream(stream)))
    return rate.value


def ml_profile_enable(on=True):
    _check(load().ml_profile_enable(1 if on else 0))


def ml_profile_reset():
    _check(load().ml_profile_reset())


def ml_profile_read():
    """{kernel family: (launches, total ms)} recorded since the last reset."""
    lib = load()
    out, i = {}, 0
    name = ctypes.c_char_p()
    launches = ctypes.c_int64()
    ms = ctypes.c_double()
    while lib.ml_profile_read(i, ctypes.byref(name), ctypes.byref(launches), ctypes.byref(ms)) == ML_OK:
        out[name.value.decode()] = (launches.value, ms.value)
        i += 1
    return out


def version():
    return load().ml_version().decode()
