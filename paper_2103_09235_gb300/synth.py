"""Seeded synthetic inputs for the folded-stencil workloads.

This module only draws numbers: grid values, dyadic stencil coefficients and
the shapes of a batched workload.  It holds none of the stencil arithmetic, so
both the CPU oracle's tests and the GPU path's tests and bench can use it.

Generator: a counter-based SplitMix64.  Value ``idx`` of stream ``seed`` is
``splitmix64(seed XOR (idx * PHI))`` with ``PHI = 0x9E3779B97F4A7C15``; its top
53 bits scaled by 2**-53 give a double in [0, 1).  SplitMix64 is Steele, Lea
and Flood's finaliser ("Fast splittable pseudorandom number generators",
OOPSLA 2014): add PHI, then two xor-shift-multiply rounds and a final xor-shift.
"""

from __future__ import annotations

import numpy as np

PHI = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Seeds of the five standard workloads: workload i uses BASE_SEED + i.
BASE_SEED = 2103092350

# Dyadic coefficients are integers over 2**24: exact in FP32 and FP64.
COEF_DENOM_BITS = 24


def splitmix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied elementwise to uint64 states."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + PHI
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, start: int = 0, chunk: int = 1 << 24) -> np.ndarray:
    """Doubles in [0, 1): element i is draw number ``start + i`` of ``seed``."""
    out = np.empty(n, dtype=np.float64)
    s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    for lo in range(0, n, chunk):
        hi = min(n, lo + chunk)
        idx = np.arange(start + lo, start + hi, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = splitmix64(s ^ (idx * PHI))
        out[lo:hi] = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return out


def grid(seed: int, shape, dtype=np.float32) -> np.ndarray:
    """A C-order grid of values uniform in [0, 1), rounded to ``dtype``."""
    n = int(np.prod(shape))
    return uniform(seed, n).astype(dtype).reshape(tuple(shape))


def stencil_offsets(ndim: int, radius: int, kind: str):
    """Offsets of a star or box stencil, in the dense tap order.

    The dense coefficient array has shape (2r+1,)*ndim with axis order
    (z, y, x) and each axis indexed by offset + r.  A star keeps the centre and
    the taps on the axes; a box keeps all taps.
    """
    offs = []
    for o in np.ndindex(*((2 * radius + 1,) * ndim)):
        off = tuple(int(v) - radius for v in o)
        nonzero_axes = sum(1 for v in off if v != 0)
        if kind == "box" or nonzero_axes <= 1:
            offs.append(off)
    return offs


def dyadic_coeffs(seed: int, ndim: int, radius: int, kind: str) -> np.ndarray:
    """Random positive coefficients that sum to exactly 1.

    Every tap is an integer numerator k >= 1 over 2**24 and the numerators sum
    to 2**24, so the values are exact in FP32 and FP64 and the stencil
    conserves the grid sum exactly.  Raw weights are 1 + floor(u * 2**20); they
    are scaled to 2**24 with floor rounding and the leftover goes to the
    centre tap.
    """
    offs = stencil_offsets(ndim, radius, kind)
    u = uniform(seed, len(offs))
    raw = 1 + np.floor(u * (1 << 20)).astype(np.int64)
    total = int(raw.sum())
    denom = 1 << COEF_DENOM_BITS
    k = (raw * denom) // total
    centre = offs.index((0,) * ndim)
    k[centre] += denom - int(k.sum())
    assert int(k.sum()) == denom and int(k.min()) >= 1
    c = np.zeros((2 * radius + 1,) * ndim, dtype=np.float64)
    for off, kk in zip(offs, k):
        c[tuple(v + radius for v in off)] = float(kk) / denom
    return c


def _dyadic_1d(seed: int, radius: int, bits: int) -> np.ndarray:
    """Positive 1D weights k_i / 2**bits summing to exactly 1 (leftover to the centre)."""
    u = uniform(seed, 2 * radius + 1)
    raw = 1 + np.floor(u * (1 << 10)).astype(np.int64)
    denom = 1 << bits
    k = (raw * denom) // int(raw.sum())
    k[radius] += denom - int(k.sum())
    return k.astype(np.float64) / denom


def separable_coeffs(seed: int, radius: int, rank: int = 1) -> np.ndarray:
    """2D box weights that are a sum of `rank` (1 or 2) separable terms.

    Rank 1: outer(u, v) with u, v dyadic 1D weights over 2**12, so every tap is
    an integer over 2**24 and exact in FP32.  Rank 2: the mean of two such
    products with 1D weights over 2**11 (taps over 2**23).  Both sum to 1.
    """
    if rank == 1:
        return np.outer(_dyadic_1d(seed, radius, 12), _dyadic_1d(seed + 1, radius, 12))
    if rank == 2:
        a = np.outer(_dyadic_1d(seed, radius, 11), _dyadic_1d(seed + 1, radius, 11))
        b = np.outer(_dyadic_1d(seed + 2, radius, 11), _dyadic_1d(seed + 3, radius, 11))
        return (a + b) / 2
    raise ValueError("rank must be 1 or 2")


def heat2d_coeffs() -> np.ndarray:
    """The symmetric 2D 5-point heat stencil: 1/2 at the centre, 1/8 on each axis neighbour."""
    c = np.zeros((3, 3))
    c[1, 1] = 0.5
    c[0, 1] = c[2, 1] = c[1, 0] = c[1, 2] = 0.125
    return c


def heat1d_coeffs() -> np.ndarray:
    """The 1D 3-point heat stencil (0.25, 0.5, 0.25)."""
    return np.array([0.25, 0.5, 0.25], dtype=np.float64)


def batched_workload(seed: int, n_grids: int = 256, side_lo: int = 64,
                     side_hi: int = 1024, t_lo: int = 10, t_hi: int = 500):
    """Descriptions of a batch of independent 2D grids of uneven size.

    Grid j draws, from stream ``seed + 1`` and draw numbers 4j..4j+3: its
    height and width uniform in [side_lo, side_hi], a 50/50 choice between a
    5-point star and a 9-point box, and T uniform in [t_lo, t_hi].  Its
    coefficients come from stream ``seed + 1000 + j`` and its values from
    stream ``seed + 100000 + j``.
    """
    u = uniform(seed + 1, 4 * n_grids)
    grids = []
    for j in range(n_grids):
        ny = side_lo + int(u[4 * j] * (side_hi - side_lo + 1))
        nx = side_lo + int(u[4 * j + 1] * (side_hi - side_lo + 1))
        kind = "star" if u[4 * j + 2] < 0.5 else "box"
        T = t_lo + int(u[4 * j + 3] * (t_hi - t_lo + 1))
        grids.append({
            "shape": (ny, nx), "kind": kind, "T": T,
            "coeff_seed": seed + 1000 + j, "value_seed": seed + 100000 + j,
        })
    return grids
