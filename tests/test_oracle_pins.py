"""Pins of the CPU oracle to facts that do not come from the oracle itself.

Each test checks one oracle function against something the paper or the
mathematics fixes: cyclic shifts (numpy.roll), single Fourier modes, the
textbook heat-kernel eigenvalue cos^2(pi k / N), FFT convolution, exact sum
conservation, the binomial form of the folded 1D heat stencil, and the values
the paper prints for its 9-point box example (Section 3.3).  The mutation
tests at the end plant plausible mistakes in a copy of the oracle and show
that these pins catch them.
"""

import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_2103_09235_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_worked_examples.txt")


def golden():
    vals = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = (s.strip() for s in line.split("=", 1))
            vals[k] = [float(t) for t in v.split()]
    return vals


def roll_step(x, c):
    """One step as a sum of cyclic shifts: tap at offset o reads x[p + o]."""
    r = (c.shape[0] - 1) // 2
    out = np.zeros_like(x, dtype=np.float64)
    for idx in np.ndindex(*c.shape):
        if c[idx] == 0.0:
            continue
        off = tuple(i - r for i in idx)
        out += c[idx] * np.roll(x, shift=tuple(-o for o in off), axis=tuple(range(x.ndim)))
    return out


CASES = [
    ((13,), 1, "box"), ((11,), 2, "box"), ((6, 7), 1, "star"), ((6, 7), 1, "box"),
    ((5, 9), 2, "star"), ((4, 5, 6), 1, "star"), ((4, 5, 6), 1, "box"), ((5, 5, 7), 2, "star"),
]


@pytest.mark.parametrize("shape,r,kind", CASES)
def test_run_equals_cyclic_shift_sum(oracle_mod, shape, r, kind):
    """Small-integer inputs and dyadic weights: every FP64 operation is exact."""
    c = synth.dyadic_coeffs(7 + r, len(shape), r, kind)
    x = np.floor(synth.uniform(3, int(np.prod(shape))) * 16).reshape(shape)
    ref = x.astype(np.float64)
    for T in range(1, 4):
        ref = roll_step(ref, c)
        got = oracle_mod.run(x, c, T)
        assert np.array_equal(got, ref), (shape, r, kind, T)


def test_run_exact_rational_tiny_1d(oracle_mod):
    """Exact rational arithmetic on a 7-point ring with an asymmetric stencil."""
    c = np.array([0.125, 0.5, 0.375])
    x = [3, 1, 4, 1, 5, 9, 2]
    n = len(x)
    cur = [Fraction(v) for v in x]
    cf = [Fraction(v).limit_denominator() for v in c]
    for _ in range(5):
        cur = [sum(cf[k] * cur[(i + k - 1) % n] for k in range(3)) for i in range(n)]
    got = oracle_mod.run(np.array(x, float), c, 5)
    assert [Fraction(v) for v in got] == cur


@pytest.mark.parametrize("N,k,T", [(32, 1, 7), (32, 5, 20), (45, 11, 3), (64, 31, 50)])
def test_heat1d_fourier_mode(oracle_mod, N, k, T):
    """(0.25, 0.5, 0.25) scales cos(2 pi k x / N) by cos^2(pi k / N) per step."""
    xs = np.arange(N)
    x = np.cos(2 * np.pi * k * xs / N)
    got = oracle_mod.run(x, synth.heat1d_coeffs(), T)
    ref = math.cos(math.pi * k / N) ** (2 * T) * x
    assert np.max(np.abs(got - ref)) < 1e-13


@pytest.mark.parametrize("shape,r,kind,k", [((16, 20), 1, "box", (3, 5)),
                                           ((12, 10), 2, "star", (1, 4)),
                                           ((6, 8, 10), 1, "box", (1, 2, 3))])
def test_single_mode_closed_form(oracle_mod, shape, r, kind, k):
    """A complex mode e^{2 pi i k.p/N} becomes lambda(k)^T e^{2 pi i k.p/N}."""
    c = synth.dyadic_coeffs(11, len(shape), r, kind)
    grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    phase = sum(2 * np.pi * ki * g / n for ki, g, n in zip(k, grids, shape))
    lam = 0j
    for idx in np.ndindex(*c.shape):
        off = [i - r for i in idx]
        lam += c[idx] * np.exp(2j * np.pi * sum(ki * o / n for ki, o, n in zip(k, off, shape)))
    T = 9
    re = oracle_mod.run(np.cos(phase), c, T)
    im = oracle_mod.run(np.sin(phase), c, T)
    ref = lam ** T * np.exp(1j * phase)
    assert np.max(np.abs(re + 1j * im - ref)) < 1e-13


@pytest.mark.parametrize("shape,r,kind", [((64, 64), 1, "box"), ((48, 40), 2, "star"),
                                          ((16, 16, 16), 1, "box"), ((10, 12, 14), 1, "star")])
def test_run_matches_fft_convolution(oracle_mod, shape, r, kind):
    """One step is a circular correlation; numpy's FFT computes it independently."""
    c = synth.dyadic_coeffs(5, len(shape), r, kind)
    x = synth.grid(17, shape, np.float64)
    kern = np.zeros(shape)
    for idx in np.ndindex(*c.shape):
        kern[tuple((i - r) % n for i, n in zip(idx, shape))] += c[idx]
    # correlation: out[p] = sum_o c[o] x[p+o]  <=>  F(out) = conj(F(kern)) * F(x)
    ref = x
    for _ in range(4):
        ref = np.real(np.fft.ifftn(np.conj(np.fft.fftn(kern)) * np.fft.fftn(ref)))
    got = oracle_mod.run(x, c, 4)
    assert np.max(np.abs(got - ref)) < 1e-12


@pytest.mark.parametrize("shape,r,kind", [((64, 48), 1, "box"), ((8, 9, 10), 1, "star")])
def test_spectral_run_matches_time_loop(oracle_mod, shape, r, kind):
    c = synth.dyadic_coeffs(23, len(shape), r, kind)
    x = synth.grid(29, shape, np.float64)
    got = oracle_mod.spectral_run(x, c, 37)
    ref = oracle_mod.run(x, c, 37)
    assert np.max(np.abs(got - ref)) < 1e-12


@pytest.mark.parametrize("scale", [1.0, 0.875])
def test_sum_conservation(oracle_mod, scale):
    """sum(A_T) = sum(A_0) * (sum c)^T; with sum c = 1 the sum is conserved."""
    c = synth.dyadic_coeffs(31, 2, 1, "box") * scale
    x = synth.grid(37, (33, 29), np.float64)
    T = 25
    got = oracle_mod.run(x, c, T)
    assert abs(got.sum() - x.sum() * c.sum() ** T) < 1e-12 * abs(x.sum())


@pytest.mark.parametrize("m", [1, 2, 3, 4, 7])
def test_fold_heat1d_binomial(oracle_mod, m):
    """(1/4, 1/2, 1/4)^{*m}[j] = C(2m, m+j) / 4^m."""
    f = oracle_mod.fold_coeffs(synth.heat1d_coeffs(), m)
    ref = np.array([math.comb(2 * m, m + j) / 4.0 ** m for j in range(-m, m + 1)])
    assert f.shape == (2 * m + 1,)
    assert np.max(np.abs(f - ref)) < 1e-15


@pytest.mark.parametrize("ndim,r,kind,m", [(1, 1, "box", 3), (2, 1, "star", 2), (2, 1, "star", 4),
                                           (2, 1, "box", 4), (2, 2, "star", 2), (3, 1, "star", 2),
                                           (3, 1, "box", 2)])
def test_fold_is_reflected_delta_response(oracle_mod, ndim, r, kind, m):
    """m plain steps applied to a unit impulse at the origin give c^{(m)}[-p]."""
    c = synth.dyadic_coeffs(41 + m, ndim, r, kind)
    R = m * r
    n = 2 * R + 3
    x = np.zeros((n,) * ndim)
    x[(0,) * ndim] = 1.0
    resp = oracle_mod.run(x, c, m)
    f = oracle_mod.fold_coeffs(c, m)
    for idx in np.ndindex(*f.shape):
        off = tuple(i - R for i in idx)
        assert abs(resp[tuple((-o) % n for o in off)] - f[idx]) < 1e-15


@pytest.mark.parametrize("ndim,r,kind,m", [(2, 1, "box", 4), (2, 1, "star", 3), (3, 1, "box", 2)])
def test_fold_dft_is_power(oracle_mod, ndim, r, kind, m):
    """DFT(c^{(m)}) = DFT(c)^m on a grid wide enough not to alias."""
    c = synth.dyadic_coeffs(53, ndim, r, kind)
    f = oracle_mod.fold_coeffs(c, m)
    n = f.shape[0] + 2
    pad_c = np.zeros((n,) * ndim)
    pad_c[tuple(slice(0, s) for s in c.shape)] = c
    pad_f = np.zeros((n,) * ndim)
    pad_f[tuple(slice(0, s) for s in f.shape)] = f
    assert np.max(np.abs(np.fft.fftn(pad_c) ** m - np.fft.fftn(pad_f))) < 1e-14


def test_fold_paper_unit_box():
    """Unit 3x3 box, m = 2: the paper's lambda^(1) and counterpart multiples."""
    import oracle
    g = golden()
    f = oracle.fold_coeffs(np.ones((3, 3)), 2)
    lam1 = np.array(g["lambda1"])
    assert np.array_equal(f, np.outer(lam1, lam1))
    # column b of the folded matrix is lambda^(1) times the horizontal weight of b
    for b, w in enumerate(g["horizontal_weights"]):
        assert np.array_equal(f[:, b], w * lam1)
    mult = g["counterpart_multiples"]
    assert np.array_equal(f[:, 1], mult[1] * f[:, 0]) and np.array_equal(f[:, 2], mult[2] * f[:, 0])
    assert g["omega2"] == [2.0] and g["omega3"] == [0.0, 3.0]
    assert np.array_equal(f[:, 1], g["omega2"][0] * f[:, 0])
    assert np.array_equal(f[:, 2], g["omega3"][0] * f[:, 1] + g["omega3"][1] * f[:, 0])


@pytest.mark.parametrize("shape,r,kind,m,T", [((40, 36), 1, "star", 2, 9), ((40, 36), 1, "box", 4, 13),
                                              ((64,), 1, "box", 3, 20), ((9, 10, 11), 1, "star", 2, 7)])
def test_folded_run_equals_plain(oracle_mod, shape, r, kind, m, T):
    c = synth.dyadic_coeffs(61, len(shape), r, kind)
    x = synth.grid(67, shape, np.float64)
    ref = oracle_mod.run(x, c, T)
    got = oracle_mod.folded_run(x, c, T, m)
    assert np.max(np.abs(got - ref)) < 1e-13


def test_rel_l2(oracle_mod):
    r = np.array([3.0, 4.0])
    assert oracle_mod.rel_l2(r, r) == 0.0
    assert abs(oracle_mod.rel_l2(np.array([3.0, 5.0]), r) - 0.2) < 1e-15
    assert abs(oracle_mod.rel_l2_zero_mean(np.array([4.0, 6.0]), np.array([1.0, 2.0])) - 1.0) < 1e-15


def test_tessellation_profiles_sum():
    """Section 3.4: a triangle and an inverted triangle together advance 4 steps."""
    g = golden()
    tri, inv = np.array(g["tess_triangle"]), np.array(g["tess_inverted"])
    assert np.all(tri + inv == 4)


# ---- mutation tests: plausible mistakes planted in a copy of the oracle ----

def test_mutation_flipped_orientation_is_caught(oracle_mod):
    """Reading in[p - o] instead of in[p + o] fails the cyclic-shift pin."""
    c = synth.dyadic_coeffs(8, 2, 1, "box")
    x = np.floor(synth.uniform(3, 42) * 16).reshape(6, 7)
    wrong = oracle_mod.run(x, c[::-1, ::-1].copy(), 1)
    assert not np.array_equal(wrong, roll_step(x, c))


def test_mutation_dropped_fold_term_is_caught(oracle_mod):
    """A fold that applies one convolution too few fails the binomial pin."""
    f = oracle_mod.fold_coeffs(synth.heat1d_coeffs(), 2)
    bad = np.pad(oracle_mod.fold_coeffs(synth.heat1d_coeffs(), 1), 1)
    ref = np.array([math.comb(4, 2 + j) / 16 for j in range(-2, 3)])
    assert np.max(np.abs(f - ref)) < 1e-15 and np.max(np.abs(bad - ref)) > 1e-3


def test_mutation_transposed_coeffs_is_caught(oracle_mod):
    """Swapping the y and x axes of an asymmetric stencil fails the mode pin."""
    c = synth.dyadic_coeffs(11, 2, 1, "box")
    x = synth.grid(5, (12, 16), np.float64)
    assert np.max(np.abs(oracle_mod.run(x, c.T.copy(), 3) - oracle_mod.spectral_run(x, c, 3))) > 1e-3
