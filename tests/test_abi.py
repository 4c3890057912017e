"""Host-side checks of the C-ABI library: it builds, loads, exports every
entry point the header declares, rejects bad arguments before touching a GPU,
and its planner counts match the values the paper prints (Section 3.2)."""

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def blib():
    from paper_2103_09235_gb300 import build, binding
    build.build()
    return binding


def header_symbols():
    with open(os.path.join(ROOT, "include", "stencil.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"\b(stencil_[a-z0-9_]+)\s*\(", text)))


def test_header_and_binding_agree(blib):
    assert header_symbols() == sorted(blib.EXPORTS)


def test_library_exports_every_declared_symbol(blib):
    L = blib.lib()
    for name in header_symbols():
        assert hasattr(L, name), name


def test_status_strings(blib):
    for code, name in blib.STATUS.items():
        assert blib.status_string(code) == name


def test_plan_rejects_bad_arguments_without_gpu(blib):
    import ctypes
    L = blib.lib()
    h = ctypes.c_void_p()
    shape = (ctypes.c_int64 * 2)(8, 8)
    c = np.ones((3, 3))
    cp = c.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert L.stencil_plan(ctypes.byref(h), 4, shape, 1, cp, 0) == 1        # ndim
    assert L.stencil_plan(ctypes.byref(h), 2, shape, 0, cp, 0) == 1        # radius
    small = (ctypes.c_int64 * 2)(2, 8)
    assert L.stencil_plan(ctypes.byref(h), 2, small, 1, cp, 0) == 1        # extent < 2r+1
    assert L.stencil_plan(ctypes.byref(h), 2, shape, 1, cp, 7) == 1        # unknown dtype
    assert L.stencil_plan(ctypes.byref(h), 2, shape, 1, None, 0) == 1
    assert "stencil_plan" in L.stencil_last_error().decode()


def golden():
    vals = {}
    with open(os.path.join(ROOT, "tests", "golden", "paper_worked_examples.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = (s.strip() for s in line.split("=", 1))
                vals[k] = [float(t) for t in v.split()]
    return vals


def test_fold_cost_paper_example(blib):
    """Unit 9-point box, m = 2: |C(E)| = 90, |C(E_lambda)| = 25, P = 3.6."""
    g = golden()
    naive, folded = blib.fold_cost(np.ones((3, 3)), 2)
    assert naive == g["collect_naive"][0] and folded == g["collect_folded"][0]
    assert abs(naive / folded - g["profitable_index"][0]) < 1e-12


@pytest.mark.parametrize("ndim,kind,m,folded", [(2, "star", 2, 13), (2, "star", 4, 41),
                                                (2, "box", 4, 81), (3, "star", 2, 25),
                                                (3, "box", 2, 125), (1, "box", 3, 7)])
def test_fold_cost_support_sizes(blib, ndim, kind, m, folded):
    from paper_2103_09235_gb300 import synth
    c = synth.dyadic_coeffs(1, ndim, 1, kind)
    naive, f = blib.fold_cost(c, m)
    assert f == folded
    base = int(np.count_nonzero(c))
    assert naive >= base * m


def test_plan_ex_rejects_flags_and_pitches_before_device_work(blib):
    """stencil_plan_ex: unknown flag bits are INVALID_ARG, a non-periodic
    boundary is UNSUPPORTED, pitches below the dense strides are INVALID_ARG;
    all of them are decided on the host, before any device call."""
    L = blib.lib()
    h = ctypes.c_void_p()
    c = np.zeros((3, 3)); c[1, 1] = 1.0
    cp = c.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    shape = (ctypes.c_int64 * 2)(64, 100)
    good = (ctypes.c_int64 * 1)(128)
    assert L.stencil_plan_ex(ctypes.byref(h), 2, shape, 1, cp, 0, good, 4) == 1      # unknown bit
    assert L.stencil_plan_ex(ctypes.byref(h), 2, shape, 1, cp, 0, good, 1) == 2      # non-periodic
    assert "periodic" in L.stencil_last_error().decode()
    short = (ctypes.c_int64 * 1)(99)
    assert L.stencil_plan_ex(ctypes.byref(h), 2, shape, 1, cp, 0, short, 0) == 1     # row < nx
    c3 = np.zeros((3, 3, 3)); c3[1, 1, 1] = 1.0
    cp3 = c3.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    shape3 = (ctypes.c_int64 * 3)(8, 10, 12)
    flat = (ctypes.c_int64 * 2)(16 * 9, 16)                                          # plane < row*ny
    assert L.stencil_plan_ex(ctypes.byref(h), 3, shape3, 1, cp3, 0, flat, 0) == 1
    assert not h.value
