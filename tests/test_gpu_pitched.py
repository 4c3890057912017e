"""Grids with row (and plane) strides larger than dense: stencil_plan_ex.

Each case embeds the grid in a larger buffer whose gaps hold a sentinel,
runs the library on the strided view, compares the points with the FP64
oracle (relative L2 <= 1e-5; the oracle runs on the dense copy of the same
points) and checks that no gap element of the output buffer was written.
"""

import numpy as np
import pytest

from paper_2103_09235_gb300 import synth

pytestmark = pytest.mark.gpu

SENTINEL = -7.25


@pytest.fixture(scope="module")
def env(oracle_mod):
    import torch
    from paper_2103_09235_gb300 import build, binding
    build.build()
    assert torch.cuda.is_available()
    torch.cuda.init()
    return torch, binding, oracle_mod


def strided(torch, dense, pad):
    """A buffer one pad wider per axis (all but the first) holding `dense`,
    sentinel in the gaps; returns the buffer and the view of the grid."""
    full = tuple(s + (p if i else 0) for i, (s, p) in enumerate(zip(dense.shape, pad)))
    buf = torch.full(full, SENTINEL, dtype=torch.float32, device="cuda")
    view = buf[tuple(slice(0, s) for s in dense.shape)]
    view.copy_(torch.from_numpy(dense).cuda())
    return buf, view


def pitches_of(view):
    return [int(s) for s in view.stride()[:-1]]


def gaps_untouched(buf, shape):
    mask = np.ones(buf.shape, bool)
    mask[tuple(slice(0, s) for s in shape)] = False
    b = buf.cpu().numpy()
    return bool(np.all(b[mask] == SENTINEL))


@pytest.mark.parametrize("shape,pad,kind,T,m,opts", [
    ((300, 520), (0, 37), "star", 37, 2, {}),
    ((300, 520), (0, 9), "box", 41, 4, {"precision": 1}),
    ((257, 300), (0, 12), "box", 29, 3, {"block_b": 3}),
    ((40, 50, 60), (0, 3, 4), "star", 23, 2, {}),
    ((36, 40, 44), (0, 0, 20), "box", 21, 1, {"block_b": 2}),
    # the persistent multi-pass launch writes its last pass into the strided grid
    ((40, 50, 60), (0, 3, 4), "box", 19, 1, {"block_b": 1, "persistent": 1}),
    ((36, 40, 44), (0, 5, 0), "star", 25, 2, {"block_b": 1, "persistent": 1, "z_chunk": 6}),
])
def test_pitched_device_grid_matches_oracle(env, shape, pad, kind, T, m, opts):
    torch, binding, oracle = env
    ndim = len(shape)
    c = synth.dyadic_coeffs(91 + ndim, ndim, 1, kind)
    x = synth.grid(300 + T, shape, np.float32)
    xbuf, xv = strided(torch, x, pad)
    ybuf, yv = strided(torch, np.zeros(shape, np.float32), pad)
    ybuf.fill_(SENTINEL)
    plan = binding.Plan(shape, c, pitch=pitches_of(xv))
    for k, v in opts.items():
        plan.set_option(k, v)
    plan.run(xv, yv, T, fold_m=m)
    plan.sync()
    ref = oracle.run(x.astype(np.float64), c, T)
    assert oracle.rel_l2(yv.cpu().numpy(), ref) <= 1e-5
    assert gaps_untouched(ybuf, shape)
    assert gaps_untouched(xbuf, shape)
    plan.close()


def test_pitched_autotuned_and_t0(env):
    """fold_m = 0 (the autotuner times candidates on scratch grids in the
    caller's strided layout) and T = 0 (a strided copy)."""
    torch, binding, oracle = env
    shape, pad = (200, 260), (0, 20)
    c = synth.dyadic_coeffs(93, 2, 1, "box")
    x = synth.grid(333, shape, np.float32)
    _, xv = strided(torch, x, pad)
    ybuf, yv = strided(torch, np.zeros(shape, np.float32), pad)
    ybuf.fill_(SENTINEL)
    plan = binding.Plan(shape, c, pitch=pitches_of(xv))
    plan.run(xv, yv, 0, fold_m=1)
    plan.sync()
    assert np.array_equal(yv.cpu().numpy(), x)
    assert gaps_untouched(ybuf, shape)
    plan.run(xv, yv, 30, fold_m=0)
    plan.sync()
    assert oracle.rel_l2(yv.cpu().numpy(), oracle.run(x.astype(np.float64), c, 30)) <= 1e-5
    assert gaps_untouched(ybuf, shape)
    plan.close()


def test_pitched_host_grid(env):
    """Host (numpy) grids with the same strides: the library copies the points
    in and out row by row and leaves the caller's gaps alone."""
    _, binding, oracle = env
    shape, pitch = (120, 130), 136
    c = synth.dyadic_coeffs(94, 2, 1, "star")
    x = synth.grid(334, shape, np.float32)
    xb = np.full((shape[0], pitch), SENTINEL, np.float32)
    xb[:, :shape[1]] = x
    yb = np.full_like(xb, SENTINEL)
    plan = binding.Plan(shape, c, pitch=[pitch])
    plan.run(xb, yb, 17, fold_m=2)  # host pointers: synchronous
    assert oracle.rel_l2(yb[:, :shape[1]], oracle.run(x.astype(np.float64), c, 17)) <= 1e-5
    assert np.all(yb[:, shape[1]:] == SENTINEL)
    plan.close()


def test_pitched_batched(env):
    """A batch mixing dense and strided plans in one persistent launch."""
    torch, binding, oracle = env
    plans, xs, ys, bufs, data = [], [], [], [], []
    for j, (shape, pad, kind, T) in enumerate([((150, 200), (0, 24), "star", 33),
                                               ((96, 128), (0, 0), "box", 20),
                                               ((210, 170), (0, 6), "box", 45)]):
        c = synth.dyadic_coeffs(95 + j, 2, 1, kind)
        x = synth.grid(400 + j, shape, np.float32)
        _, xv = strided(torch, x, pad)
        ybuf, yv = strided(torch, np.zeros(shape, np.float32), pad)
        ybuf.fill_(SENTINEL)
        plans.append(binding.Plan(shape, c, pitch=pitches_of(xv)))
        xs.append(xv)
        ys.append(yv)
        bufs.append(ybuf)
        data.append((x, c, T, shape))
    binding.run_batched(plans, xs, ys, [d[2] for d in data])
    plans[0].sync()
    for (x, c, T, shape), y, yb in zip(data, ys, bufs):
        assert oracle.rel_l2(y.cpu().numpy(), oracle.run(x.astype(np.float64), c, T)) <= 1e-5
        assert gaps_untouched(yb, shape)
    for p in plans:
        p.close()
