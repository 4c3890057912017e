"""CPU oracle for the folded-stencil library: plain, slow, obviously correct.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA path and never imports the library package.

Everything here is FP64 and follows Li et al., "Reducing Redundancy in Data
Organization and Arithmetic Calculation for Stencil Computations":

- ``run``: the plain stencil time loop of Section 1 (each point at t+1 is the
  weighted sum of itself and its neighbours at t), two alternating arrays as in
  Section 3.3.  Written in C (``stencil_oracle.c``) with OpenMP over the outer
  spatial loops.
- ``fold_coeffs``: the reassigned weights of the folding matrix (Section 3.2,
  Section 3.3 Eq. vfold): the m-step expansion of a linear stencil is the
  m-fold convolution power of its coefficient array.
- ``folded_run``: floor(T/m) sweeps of the folded stencil then T mod m plain
  steps (Section 3.4: the odd steps are skipped when m = 2).
- ``spectral_run``: the per-Fourier-mode closed form of the plain loop, used to
  check full-size grids whose time loop would take too long on the host.
- ``rel_l2``: the relative L2 error used by every parity test.

Readings (the paper is silent on them): correlation orientation
out[x] = sum_o c[o] in[x+o]; periodic boundaries; dense (2r+1)^ndim
coefficient arrays with axis order (z, y, x).

Pins: ``tests/test_oracle_pins.py`` checks every function here against exact
rational brute force, closed forms, invariants and the values the paper prints.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stencil_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, -O3, OpenMP) into ``oracle/liboracle.so``."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O3", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.oracle_stencil_run.restype = ctypes.c_int
        lib.oracle_stencil_run.argtypes = [
            ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_int,
            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
            ctypes.POINTER(ctypes.c_double), ctypes.c_int64, ctypes.c_int]
        lib.oracle_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def max_threads() -> int:
    """Threads the C oracle uses by default (OpenMP's maximum)."""
    return int(_load().oracle_max_threads())


def _radius_of(coeffs: np.ndarray) -> int:
    w = coeffs.shape[0]
    if w % 2 != 1 or any(s != w for s in coeffs.shape):
        raise ValueError("coefficients must be a (2r+1)^ndim array")
    return (w - 1) // 2


def run(x: np.ndarray, coeffs: np.ndarray, T: int, nthreads: int = 0) -> np.ndarray:
    """T plain steps of out[p] = sum_o c[o] * in[(p + o) mod shape] in FP64."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    c = np.ascontiguousarray(coeffs, dtype=np.float64)
    if c.ndim != x.ndim:
        raise ValueError("coefficient rank must equal grid rank")
    r = _radius_of(c)
    out = np.empty_like(x)
    shape = (ctypes.c_int64 * x.ndim)(*x.shape)
    dp = ctypes.POINTER(ctypes.c_double)
    rc = _load().oracle_stencil_run(
        x.ndim, shape, r, c.ctypes.data_as(dp), x.ctypes.data_as(dp),
        out.ctypes.data_as(dp), int(T), int(nthreads))
    if rc != 0:
        raise RuntimeError("oracle_stencil_run failed")
    return out


def _convolve_full(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Full discrete convolution of two centred odd-sized arrays, by its sum.

    out[p + q] += a[p] * b[q] over every pair of taps, offsets measured from
    each array's centre; the result is centred too.
    """
    out = np.zeros(tuple(sa + sb - 1 for sa, sb in zip(a.shape, b.shape)))
    for q in np.ndindex(*b.shape):
        w = b[q]
        if w == 0.0:
            continue
        sl = tuple(slice(qi, qi + sa) for qi, sa in zip(q, a.shape))
        out[sl] += w * a
    return out


def fold_coeffs(coeffs: np.ndarray, m: int) -> np.ndarray:
    """Folded weights of m steps: the m-fold convolution power c * c * ... * c.

    For a radius-r stencil the result has radius m*r.  m = 0 gives the
    identity (a single unit tap).  Section 3.2 (folding matrix of reassigned
    weights), Section 3.3 Eq. vfold.
    """
    c = np.asarray(coeffs, dtype=np.float64)
    if m < 0:
        raise ValueError("m must be >= 0")
    out = np.ones((1,) * c.ndim)
    for _ in range(m):
        out = _convolve_full(out, c)
    return out


def folded_run(x: np.ndarray, coeffs: np.ndarray, T: int, m: int,
               nthreads: int = 0) -> np.ndarray:
    """floor(T/m) sweeps of the folded stencil, then T mod m plain steps."""
    q, rem = divmod(int(T), int(m))
    y = run(x, fold_coeffs(coeffs, m), q, nthreads) if q else np.asarray(x, np.float64)
    return run(y, coeffs, rem, nthreads) if rem else y


def eigenvalues(coeffs: np.ndarray, shape) -> np.ndarray:
    """lambda(k) = sum_o c[o] exp(+2 pi i k.o / N) on the rfftn frequency grid.

    A Fourier mode exp(2 pi i k.x / N) is scaled by lambda(k) in one step.
    Taps are placed at (o mod N), so a stencil wider than the grid aliases
    exactly as the periodic loop does.
    """
    c = np.asarray(coeffs, dtype=np.float64)
    r = _radius_of(c)
    kern = np.zeros(tuple(shape))
    for idx in np.ndindex(*c.shape):
        if c[idx] != 0.0:
            pos = tuple((i - r) % n for i, n in zip(idx, shape))
            kern[pos] += c[idx]
    return np.conj(np.fft.rfftn(kern))


def spectral_run(x: np.ndarray, coeffs: np.ndarray, T: int) -> np.ndarray:
    """Closed form of T plain steps: irfftn(rfftn(x) * lambda^T)."""
    x = np.asarray(x, dtype=np.float64)
    lam = eigenvalues(coeffs, x.shape)
    axes = tuple(range(x.ndim))
    return np.fft.irfftn(np.fft.rfftn(x, axes=axes) * lam ** int(T), s=x.shape, axes=axes)


def rel_l2(y: np.ndarray, ref: np.ndarray) -> float:
    """||y - ref||_2 / ||ref||_2, accumulated in FP64."""
    y = np.asarray(y, dtype=np.float64).ravel()
    r = np.asarray(ref, dtype=np.float64).ravel()
    return float(np.linalg.norm(y - r) / np.linalg.norm(r))


def rel_l2_zero_mean(y: np.ndarray, ref: np.ndarray) -> float:
    """rel_l2 after removing each array's own mean."""
    y = np.asarray(y, dtype=np.float64).ravel()
    r = np.asarray(ref, dtype=np.float64).ravel()
    return float(np.linalg.norm((y - y.mean()) - (r - r.mean())) /
                 np.linalg.norm(r - r.mean()))
