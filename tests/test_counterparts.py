"""Counterpart factorisation of folded 2D weights (Section 3.3, Eq. vfold and
Eq. horifold; Section 3.5), pinned on the CPU.

The library's factors must rebuild the oracle's c^(m) exactly (to FP64
rounding) with the smallest number of separable terms; the paper's worked
example fixes the counterpart weights of the unit 9-point box at m = 2.
"""

import os

import numpy as np
import pytest

from paper_2103_09235_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def blib():
    from paper_2103_09235_gb300 import build, binding
    build.build()
    return binding


def golden():
    vals = {}
    with open(os.path.join(ROOT, "tests", "golden", "paper_worked_examples.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = (s.strip() for s in line.split("=", 1))
                vals[k] = np.array([float(t) for t in v.split()])
    return vals


def rebuilt(u, v):
    return sum(np.outer(u[k], v[k]) for k in range(len(u)))


def test_paper_unit_box_counterparts(blib, oracle_mod):
    """Unit 9-point box, m = 2: one counterpart.  Its vertical weights are the
    paper's lambda^(1) = {1, 2, 3, 2, 1}; the horizontal weights {1, 2, 3, 2, 1}
    make the columns 1, 2, 3 times c_1 (lambda^(2) = 2 lambda^(1), lambda^(3) =
    3 lambda^(1); omega_2 = (2))."""
    g = golden()
    cm = oracle_mod.fold_coeffs(np.ones((3, 3)), 2)
    K, u, v = blib.fold_counterparts(cm, 2)
    assert K == 1
    assert np.allclose(u[0] / u[0][0], g["lambda1"] / g["lambda1"][0], rtol=0, atol=1e-14)
    assert np.allclose(v[0] / v[0][0], g["horizontal_weights"] / g["horizontal_weights"][0],
                       rtol=0, atol=1e-14)
    mult = v[0][:3] / v[0][0]
    assert np.allclose(mult, g["counterpart_multiples"], rtol=0, atol=1e-14)
    assert mult[1] == g["omega2"][0]
    assert np.array_equal(rebuilt(u, v), cm)


@pytest.mark.parametrize("m", [1, 2, 3, 4, 6, 8])
def test_separable_stays_rank_one(blib, oracle_mod, m):
    """A separable base stays separable under folding: c^(m) = u^(m) (x) v^(m)."""
    c = synth.separable_coeffs(900 + m, 1, 1)
    cm = oracle_mod.fold_coeffs(c, m)
    K, u, v = blib.fold_counterparts(cm, 2)
    assert K == 1
    err = np.max(np.abs(rebuilt(u, v) - cm)) / np.max(np.abs(cm))
    assert err < 1e-14, err


@pytest.mark.parametrize("m", [1, 2, 3, 4])
def test_two_term_base_has_m_plus_1_terms(blib, oracle_mod, m):
    """(A + B)^m = sum_j C(m, j) A^j B^(m-j) for separable A, B: c^(m) is a sum
    of m + 1 separable terms, and no fewer for generic weights."""
    c = synth.separable_coeffs(920 + m, 1, 2)
    cm = oracle_mod.fold_coeffs(c, m)
    W = cm.shape[0]
    K, u, v = blib.fold_counterparts(cm, W)
    assert K == m + 1
    err = np.max(np.abs(rebuilt(u, v) - cm)) / np.max(np.abs(cm))
    assert err < 1e-14, err
    K2, _, _ = blib.fold_counterparts(cm, 2)
    assert K2 == min(m + 1, 3)


@pytest.mark.parametrize("r", [1, 2, 4])
def test_two_term_base_radius(blib, r):
    """A base of two separable terms is rank 2 at any radius."""
    c = synth.separable_coeffs(930 + r, r, 2)
    K, u, v = blib.fold_counterparts(c, 2)
    assert K == 2
    assert np.max(np.abs(rebuilt(u, v) - c)) / np.max(np.abs(c)) < 1e-14


@pytest.mark.parametrize("m", [1, 2, 3, 4])
def test_symmetric_heat_star_has_m_plus_1_counterparts(blib, oracle_mod, m):
    """The paper's bound of m + 1 counterparts for a symmetric radius-1 stencil,
    reached by the 2D heat star (c^(m) is a sum of m + 1 separable terms)."""
    cm = oracle_mod.fold_coeffs(synth.heat2d_coeffs(), m)
    W = cm.shape[0]
    K, u, v = blib.fold_counterparts(cm, W)
    assert K == m + 1
    assert np.max(np.abs(rebuilt(u, v) - cm)) < 1e-14


@pytest.mark.parametrize("kind,m", [("box", 2), ("box", 3), ("star", 2), ("star", 4)])
def test_random_weights_are_full_rank(blib, oracle_mod, kind, m):
    """Random weights give no saving: c^(m) needs more than two terms, and the
    full factorisation still rebuilds it."""
    c = synth.dyadic_coeffs(910 + m, 2, 1, kind)
    cm = oracle_mod.fold_coeffs(c, m)
    W = cm.shape[0]
    K2, _, _ = blib.fold_counterparts(cm, 2)
    assert K2 == 3
    K, u, v = blib.fold_counterparts(cm, W)
    assert 3 <= K <= W
    assert np.max(np.abs(rebuilt(u, v) - cm)) / np.max(np.abs(cm)) < 1e-13


def test_bad_arguments(blib):
    with pytest.raises(blib.StencilError):
        blib.fold_counterparts(np.ones((19, 19)), 2)
    with pytest.raises(blib.StencilError):
        blib.fold_counterparts(np.ones((3, 3)), 4)


def test_zero_weights(blib):
    K, u, v = blib.fold_counterparts(np.zeros((5, 5)), 2)
    assert K == 0


@pytest.mark.parametrize("r", [1, 2, 4])
@pytest.mark.parametrize("rank", [1, 2])
def test_separable_generator(r, rank):
    """The separable test weights are exact in FP32, positive, sum to exactly 1
    and have the stated rank (numpy's SVD rank, independent of the library)."""
    c = synth.separable_coeffs(960 + r, r, rank)
    assert c.shape == (2 * r + 1, 2 * r + 1)
    assert np.all(c > 0)
    assert np.array_equal(c.astype(np.float32).astype(np.float64), c)
    assert c.sum() == 1.0
    assert np.linalg.matrix_rank(c) == rank


def test_heat2d_weights():
    c = synth.heat2d_coeffs()
    assert c.sum() == 1.0 and np.count_nonzero(c) == 5
    assert np.linalg.matrix_rank(c) == 2


def test_scalar_and_sparse_weights(blib, oracle_mod):
    """A single weight is one term; a folded star keeps its zero corners
    (the factors rebuild them exactly); asking for W terms of a full-rank
    matrix returns its rank."""
    K, u, v = blib.fold_counterparts(np.array([[0.75]]), 1)
    assert K == 1 and u[0][0] * v[0][0] == 0.75
    cm = oracle_mod.fold_coeffs(synth.dyadic_coeffs(971, 2, 1, "star"), 2)
    W = cm.shape[0]
    K, u, v = blib.fold_counterparts(cm, W)
    R = rebuilt(u, v)
    assert np.max(np.abs(R - cm)) < 1e-15
    assert np.all(np.abs(R[cm == 0]) < 1e-15)
    rng = np.random.default_rng(972)
    full = rng.random((9, 9))
    K, u, v = blib.fold_counterparts(full, 9)
    assert K == np.linalg.matrix_rank(full) == 9
    assert np.max(np.abs(rebuilt(u, v) - full)) < 1e-13

