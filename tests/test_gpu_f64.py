"""FP64 2D and 3D grids, plain and folded (the paper's own precision).

Each case runs through stencil_run on FP64 device grids and is compared with
the FP64 oracle's time loop, relative L2 <= 1e-12 and max-abs <= 1e-12; at
full size (4096^2, T = 1000) with the oracle's closed form.
"""

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


def run(env, shape, c, x, T, m, **opts):
    torch, binding, _ = env
    plan = binding.Plan(shape, c, "f64")
    for k, v in opts.items():
        plan.set_option(k, v)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    plan.run(xd, yd, T, fold_m=m)
    plan.sync()
    y = yd.cpu().numpy()
    last_m = plan.get("last_m")
    plan.close()
    return y, last_m


@pytest.mark.parametrize("shape,kind,r,T,m", [
    ((100, 130), "star", 1, 17, 1), ((100, 130), "star", 1, 17, 4), ((97, 45), "box", 1, 13, 3),
    ((80, 70), "box", 2, 9, 2), ((300, 520), "box", 1, 26, 8), ((64, 90), "star", 2, 11, 4),
    ((20, 24, 28), "star", 1, 9, 2), ((20, 24, 28), "box", 1, 7, 1), ((18, 21, 33), "box", 1, 8, 4),
    ((16, 20, 24), "box", 2, 5, 2),
])
def test_f64_sweeps_match_oracle(env, shape, kind, r, T, m):
    _, _, oracle = env
    c = synth.dyadic_coeffs(600 + T, len(shape), r, kind)
    x = synth.grid(700 + T, shape, np.float64)
    y, last_m = run(env, shape, c, x, T, m)
    assert last_m == m
    ref = oracle.run(x, c, T)
    assert oracle.rel_l2(y, ref) <= 1e-12
    assert np.max(np.abs(y - ref)) <= 1e-12


def test_f64_autotuned_in_place_and_pitched(env, tmp_path, monkeypatch):
    """fold_m = 0 (the autotuner times the FP64 folds), one sweep in place,
    and a grid whose rows are padded to a larger stride."""
    torch, binding, oracle = env
    monkeypatch.setenv("STENCIL_TUNE_CACHE", str(tmp_path / "tune.jsonl"))
    shape = (120, 150)
    c = synth.dyadic_coeffs(611, 2, 1, "box")
    x = synth.grid(612, shape, np.float64)
    y, _ = run(env, shape, c, x, 40, 0)
    assert oracle.rel_l2(y, oracle.run(x, c, 40)) <= 1e-12
    plan = binding.Plan(shape, c, "f64")
    xd = torch.from_numpy(x).cuda()
    plan.run(xd, xd, 3, fold_m=3)
    plan.sync()
    assert oracle.rel_l2(xd.cpu().numpy(), oracle.run(x, c, 3)) <= 1e-12
    plan.close()
    buf = torch.full((shape[0], 160), -3.0, dtype=torch.float64, device="cuda")
    view = buf[:, :shape[1]]
    view.copy_(torch.from_numpy(x).cuda())
    out = torch.full_like(buf, -3.0)
    plan = binding.Plan(shape, c, "f64", pitch=[160])
    plan.run(view, out[:, :shape[1]], 21, fold_m=2)
    plan.sync()
    assert oracle.rel_l2(out[:, :shape[1]].cpu().numpy(), oracle.run(x, c, 21)) <= 1e-12
    assert bool((out[:, shape[1]:] == -3.0).all())
    plan.close()


def test_f64_star4096_T1000(env):
    """The 2D star workload in FP64, folded m = 4, against the closed form."""
    _, _, oracle = env
    shape = (4096, 4096)
    c = synth.dyadic_coeffs(synth.BASE_SEED + 2, 2, 1, "star")
    x = synth.grid(synth.BASE_SEED + 2, shape, np.float32).astype(np.float64)
    y, _ = run(env, shape, c, x, 1000, 4)
    ref = oracle.spectral_run(x, c, 1000)
    err = oracle.rel_l2(y, ref)
    zm = oracle.rel_l2_zero_mean(y, ref)
    print("f64 star4096 m=4 rel-L2 %.3e zero-mean %.3e" % (err, zm))
    assert err <= 1e-12 and zm <= 1e-10
