"""Thin ctypes binding of the C ABI in ``include/stencil.h``.

Argument marshalling only: every step of a stencil run happens in the CUDA
library.  Device arrays are torch tensors (their ``data_ptr()`` is passed) and
streams are torch streams (their ``cuda_stream`` handle is passed); host
arrays are numpy arrays.  Loading fails loudly when the library has not been
built: there is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libstencil_gb300.so")

F32, F64 = 0, 1
PREC_FP32, PREC_BF16X3, PREC_BF16X1 = 0, 1, 2

STATUS = {
    0: "STENCIL_OK", 1: "STENCIL_ERR_INVALID_ARG", 2: "STENCIL_ERR_UNSUPPORTED",
    3: "STENCIL_ERR_OOM", 4: "STENCIL_ERR_CUDA", 5: "STENCIL_ERR_TIMEOUT",
    6: "STENCIL_ERR_DEVICE_CHECK",
}

# Every entry point include/stencil.h declares.
EXPORTS = [
    "stencil_plan", "stencil_plan_set_option", "stencil_plan_get", "stencil_run",
    "stencil_run_batched", "stencil_sync", "stencil_folded_coeffs", "stencil_rel_l2",
    "stencil_fold_cost", "stencil_plan_destroy", "stencil_status_string", "stencil_last_error",
    "stencil_run_1d_noalloc", "stencil_fold_counterparts", "stencil_plan_ex",
    "stencil_tessellation_counts",
]


class StencilError(RuntimeError):
    """A C-ABI call returned a status other than STENCIL_OK."""

    def __init__(self, status: int, call: str, detail: str):
        super().__init__("%s -> %s (%s)" % (call, STATUS.get(status, status), detail))
        self.status = status


_lib = None
_c = ctypes
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("CUDA library %s is missing: run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        L.stencil_plan.argtypes = [ctypes.POINTER(_vp), _c.c_int, ctypes.POINTER(_i64), _c.c_int,
                                   ctypes.POINTER(_c.c_double), _c.c_int]
        L.stencil_plan_ex.argtypes = [ctypes.POINTER(_vp), _c.c_int, ctypes.POINTER(_i64),
                                      _c.c_int, ctypes.POINTER(_c.c_double), _c.c_int,
                                      ctypes.POINTER(_i64), _c.c_uint]
        L.stencil_plan_set_option.argtypes = [_vp, _c.c_char_p, _i64]
        L.stencil_plan_get.argtypes = [_vp, _c.c_char_p, ctypes.POINTER(_i64)]
        L.stencil_run.argtypes = [_vp, _vp, _vp, _i64, _c.c_int, _vp]
        L.stencil_run_batched.argtypes = [_c.c_int, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                          ctypes.POINTER(_vp), ctypes.POINTER(_i64),
                                          ctypes.POINTER(_c.c_int), _vp]
        L.stencil_sync.argtypes = [_vp, _vp]
        L.stencil_folded_coeffs.argtypes = [_vp, _c.c_int, ctypes.POINTER(_c.c_double), _c.c_size_t]
        L.stencil_rel_l2.argtypes = [_vp, _c.c_int, _vp, _i64, ctypes.POINTER(_c.c_double), _vp]
        L.stencil_fold_cost.argtypes = [_c.c_int, _c.c_int, ctypes.POINTER(_c.c_double), _c.c_int,
                                        ctypes.POINTER(_i64)]
        L.stencil_run_1d_noalloc.argtypes = [_vp, _vp, _i64, _c.c_int, ctypes.POINTER(_c.c_double),
                                             _i64, _c.c_int, _vp]
        L.stencil_run_1d_noalloc.restype = _c.c_int
        L.stencil_fold_counterparts.argtypes = [_c.c_int, ctypes.POINTER(_c.c_double), _c.c_int,
                                                ctypes.POINTER(_c.c_int),
                                                ctypes.POINTER(_c.c_double),
                                                ctypes.POINTER(_c.c_double)]
        L.stencil_fold_counterparts.restype = _c.c_int
        L.stencil_tessellation_counts.argtypes = [_c.c_int, _c.c_int, _c.c_int,
                                                  ctypes.POINTER(_c.c_int), ctypes.POINTER(_c.c_int)]
        L.stencil_tessellation_counts.restype = _c.c_int
        L.stencil_plan_destroy.argtypes = [_vp]
        L.stencil_plan_destroy.restype = None
        L.stencil_status_string.argtypes = [_c.c_int]
        L.stencil_status_string.restype = _c.c_char_p
        L.stencil_last_error.argtypes = []
        L.stencil_last_error.restype = _c.c_char_p
        for name in ("stencil_plan", "stencil_plan_ex", "stencil_plan_set_option", "stencil_plan_get", "stencil_run",
                     "stencil_run_batched", "stencil_sync", "stencil_folded_coeffs",
                     "stencil_rel_l2", "stencil_fold_cost"):
            getattr(L, name).restype = _c.c_int
        _lib = L
    return _lib


def _check(status: int, call: str):
    if status != 0:
        raise StencilError(status, call, lib().stencil_last_error().decode())


def _ptr(a):
    """Data pointer of a torch tensor or a numpy array."""
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    raise TypeError("expected a torch tensor or a numpy array")


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    return getattr(stream, "cuda_stream", stream)


def _coeff_array(coeffs, ndim):
    c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64))
    if c.ndim != ndim or any(s != c.shape[0] for s in c.shape) or c.shape[0] % 2 != 1:
        raise ValueError("coefficients must be a (2r+1)^ndim array")
    return c, (c.shape[0] - 1) // 2


class Plan:
    """A stencil plan: one grid shape, one base stencil, one dtype."""

    def __init__(self, shape, coeffs, dtype: str = "f32", pitch=None, flags: int = 0):
        """pitch: None (dense) or the ndim-1 strides in elements, C order
        (stencil_plan_ex); flags: stencil_plan_ex flags."""
        shape = tuple(int(s) for s in shape)
        c, r = _coeff_array(coeffs, len(shape))
        self.shape, self.radius, self.coeffs = shape, r, c
        self.dtype = F64 if dtype in ("f64", "float64", F64) else F32
        h = _vp()
        arr = (_i64 * len(shape))(*shape)
        cptr = c.ctypes.data_as(ctypes.POINTER(_c.c_double))
        if pitch is None and not flags:
            _check(lib().stencil_plan(ctypes.byref(h), len(shape), arr, r, cptr, self.dtype),
                   "stencil_plan")
        else:
            parr = (_i64 * max(1, len(pitch)))(*pitch) if pitch is not None else None
            _check(lib().stencil_plan_ex(ctypes.byref(h), len(shape), arr, r, cptr, self.dtype,
                                         parr, int(flags)), "stencil_plan_ex")
        self.handle = h

    def set_option(self, key: str, value: int):
        _check(lib().stencil_plan_set_option(self.handle, key.encode(), int(value)),
               "stencil_plan_set_option(%s)" % key)
        return self

    def get(self, key: str) -> int:
        v = _i64()
        _check(lib().stencil_plan_get(self.handle, key.encode(), ctypes.byref(v)), "stencil_plan_get")
        return int(v.value)

    def run(self, x, y, T: int, fold_m: int = 1, stream=None):
        """y <- T steps applied to x (device tensors or host numpy arrays)."""
        _check(lib().stencil_run(self.handle, _ptr(x), _ptr(y), int(T), int(fold_m), _stream(stream)),
               "stencil_run")
        return y

    def run_status(self, x, y, T: int, fold_m: int = 1, stream=None) -> int:
        """stencil_run's raw status (0 = OK)."""
        return lib().stencil_run(self.handle, _ptr(x), _ptr(y), int(T), int(fold_m), _stream(stream))

    def sync(self, stream=None):
        _check(lib().stencil_sync(self.handle, _stream(stream)), "stencil_sync")

    def sync_status(self, stream=None) -> int:
        return lib().stencil_sync(self.handle, _stream(stream))

    def folded_coeffs(self, m: int) -> np.ndarray:
        w = 2 * m * self.radius + 1
        out = np.empty((w,) * len(self.shape), dtype=np.float64)
        _check(lib().stencil_folded_coeffs(self.handle, int(m),
                                           out.ctypes.data_as(ctypes.POINTER(_c.c_double)), out.size),
               "stencil_folded_coeffs")
        return out

    def close(self):
        if getattr(self, "handle", None):
            lib().stencil_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run_batched(plans, xs, ys, Ts, fold_ms=None, stream=None):
    n = len(plans)
    hp = (_vp * n)(*[p.handle for p in plans])
    hi = (_vp * n)(*[_ptr(x) for x in xs])
    ho = (_vp * n)(*[_ptr(y) for y in ys])
    ht = (_i64 * n)(*[int(t) for t in Ts])
    hm = (_c.c_int * n)(*[int(m) for m in fold_ms]) if fold_ms is not None else None
    _check(lib().stencil_run_batched(n, hp, hi, ho, ht, hm, _stream(stream)), "stencil_run_batched")


def rel_l2(y, ref, stream=None):
    """(||y-ref||/||ref||, same with means removed); y FP32/FP64, ref FP64, on the device."""
    import torch
    ydt = F64 if y.dtype == torch.float64 else F32
    if ref.dtype != torch.float64:
        raise ValueError("ref must be float64")
    out = (_c.c_double * 2)()
    _check(lib().stencil_rel_l2(_ptr(y), ydt, _ptr(ref), y.numel(), out, _stream(stream)),
           "stencil_rel_l2")
    return float(out[0]), float(out[1])


def fold_cost(coeffs, m: int):
    """(|C(E)|, |C(E_lambda)|) of the scalar profitability analysis; host only."""
    c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64))
    r = (c.shape[0] - 1) // 2
    out = (_i64 * 2)()
    _check(lib().stencil_fold_cost(c.ndim, r, c.ctypes.data_as(ctypes.POINTER(_c.c_double)), int(m), out),
           "stencil_fold_cost")
    return int(out[0]), int(out[1])


def fold_counterparts(folded, max_k: int = 2):
    """Counterpart factorisation of W x W folded weights; host only.

    Returns (K, u, v) with folded = sum_k outer(u[k], v[k]) for K <= max_k;
    K = max_k + 1 when the rank is higher (u, v then hold max_k terms).
    """
    c = np.ascontiguousarray(np.asarray(folded, dtype=np.float64))
    W = c.shape[0]
    k = _c.c_int(0)
    u = np.zeros((max_k, W))
    v = np.zeros((max_k, W))
    P = ctypes.POINTER(_c.c_double)
    _check(lib().stencil_fold_counterparts(W, c.ctypes.data_as(P), int(max_k), ctypes.byref(k),
                                           u.ctypes.data_as(P), v.ctypes.data_as(P)),
           "stencil_fold_counterparts")
    K = int(k.value)
    return K, u[:min(K, max_k)], v[:min(K, max_k)]


def run_1d_noalloc(x, y, coeffs, T: int, stream=None):
    """y <- T plain 1D steps of x without any allocation (device tensors)."""
    import torch
    c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64))
    dt = F64 if x.dtype == torch.float64 else F32
    _check(lib().stencil_run_1d_noalloc(_ptr(x), _ptr(y), x.numel(), (c.size - 1) // 2,
                                        c.ctypes.data_as(ctypes.POINTER(_c.c_double)), int(T), dt,
                                        _stream(stream)),
           "stencil_run_1d_noalloc")
    return y


def status_string(code: int) -> str:
    return lib().stencil_status_string(int(code)).decode()


def tessellation_counts(W: int, b: int, R: int):
    """(stage-1, stage-2) steps per point of one tile; host only."""
    s1 = (_c.c_int * W)()
    s2 = (_c.c_int * W)()
    _check(lib().stencil_tessellation_counts(int(W), int(b), int(R), s1, s2),
           "stencil_tessellation_counts")
    return list(s1), list(s2)
