"""GPU parity of the batched persistent launch: every grid of a batch of
uneven shapes, stencils, step counts and fold depths must match the FP64
oracle run on that grid alone (relative L2 <= 1e-5 per grid)."""

import numpy as np
import pytest

from paper_2103_09235_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env(oracle_mod):
    import torch
    from paper_2103_09235_gb300 import build, binding
    build.build()
    assert torch.cuda.is_available()
    torch.cuda.init()
    return torch, binding, oracle_mod


def make_batch(n, seed, side_lo, side_hi, t_lo, t_hi):
    grids = synth.batched_workload(seed, n, side_lo, side_hi, t_lo, t_hi)
    out = []
    for g in grids:
        c = synth.dyadic_coeffs(g["coeff_seed"], 2, 1, g["kind"])
        x = synth.grid(g["value_seed"], g["shape"], np.float32)
        out.append((g, c, x))
    return out


@pytest.mark.parametrize("fold", [None, 1, 2, 4])
def test_batched_parity(env, fold):
    torch, binding, oracle = env
    batch = make_batch(14, 9000 + (fold or 0), 20, 300, 0, 45)
    plans, xs, ys, Ts = [], [], [], []
    for g, c, x in batch:
        plans.append(binding.Plan(g["shape"], c))
        xs.append(torch.from_numpy(x).cuda())
        ys.append(torch.full_like(xs[-1], float("nan")))
        Ts.append(g["T"])
    ms = None if fold is None else [fold] * len(plans)
    for _ in range(2):  # the second call replays the captured graph
        for y in ys:
            y.fill_(float("nan"))
        binding.run_batched(plans, xs, ys, Ts, ms)
        plans[0].sync()
        for (g, c, x), y in zip(batch, ys):
            ref = oracle.run(x.astype(np.float64), c, g["T"])
            err = oracle.rel_l2(y.cpu().numpy(), ref)
            assert err <= 1e-5, (g, err)
    for p in plans:
        p.close()


@pytest.mark.parametrize("shapes", [[(300, 260)], [(300, 260), (33, 40)], [(64, 128)] * 3])
def test_batched_dependency_chains(env, shapes):
    """Few grids and many passes: nearly every item waits for the previous
    pass of its own grid, often for the item its own CTA is finishing."""
    torch, binding, oracle = env
    plans, xs, ys, refs = [], [], [], []
    for j, shape in enumerate(shapes):
        c = synth.dyadic_coeffs(9100 + j, 2, 1, "star" if j % 2 == 0 else "box")
        x = synth.grid(9200 + j, shape, np.float32)
        plans.append(binding.Plan(shape, c))
        xs.append(torch.from_numpy(x).cuda())
        ys.append(torch.full_like(xs[-1], float("nan")))
        refs.append(oracle.run(x.astype(np.float64), c, 37 + 5 * j))
    Ts = [37 + 5 * j for j in range(len(shapes))]
    binding.run_batched(plans, xs, ys, Ts, [1] * len(shapes))
    plans[0].sync()
    for y, ref in zip(ys, refs):
        assert oracle.rel_l2(y.cpu().numpy(), ref) <= 1e-5
    binding.run_batched(plans, xs, ys, Ts)
    plans[0].sync()
    for y, ref in zip(ys, refs):
        assert oracle.rel_l2(y.cpu().numpy(), ref) <= 1e-5
    for p in plans:
        p.close()


def test_batched_rejects_non_2d(env):
    torch, binding, _ = env
    p1 = binding.Plan((100,), synth.heat1d_coeffs())
    x = torch.zeros(100, device="cuda")
    with pytest.raises(binding.StencilError) as ei:
        binding.run_batched([p1], [x], [x], [5])
    assert ei.value.status == 2
