"""GPU parity of the counterpart form of the 2D CUDA-core sweep (Section 3.3,
Eq. vfold and Eq. horifold; Section 3.5) against the FP64 oracle.

Separable bases stay separable under folding (one counterpart); a base of two
separable terms is rank 2 unfolded.  Shapes have ragged tiles in both
directions; T leaves a remainder after folding.
"""

import numpy as np
import pytest

from paper_2103_09235_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def env(oracle_mod):
    import torch
    from paper_2103_09235_gb300 import build, binding
    build.build()
    assert torch.cuda.is_available()
    torch.cuda.init()
    return torch, binding, oracle_mod


def coeffs(kind, r, seed):
    if kind == "sep":
        return synth.separable_coeffs(seed, r, 1)
    if kind == "two":
        return synth.separable_coeffs(seed, r, 2)
    if kind == "gb":  # the paper's Gaussian blur, [1 2 1] (x) [1 2 1] / 16
        w = np.array([1.0, 2.0, 1.0]) / 4
        return np.outer(w, w)
    return synth.dyadic_coeffs(seed, 2, r, kind)


def run(env, shape, c, x, T, m, b, mode, stages=0):
    torch, binding, _ = env
    plan = binding.Plan(shape, c).set_option("counterparts", mode).set_option("block_b", b)
    plan.set_option("stages", stages)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    plan.run(xd, yd, T, fold_m=m)
    plan.sync()
    k = plan.get("last_cp")
    plan.close()
    return yd.cpu().numpy(), k


CASES = [
    # shape, kind, r, T, m, b, mode (0 automatic, 1 forced), counterparts expected
    ((300, 520), "sep", 1, 13, 4, 1, 0, 1),
    ((300, 520), "sep", 1, 17, 8, 2, 0, 1),
    ((256, 384), "sep", 1, 12, 2, 2, 0, 1),
    ((130, 200), "sep", 1, 10, 3, 3, 1, 1),
    ((300, 520), "sep", 1, 25, 6, 2, 0, 1),
    ((200, 300), "gb", 1, 11, 2, 1, 0, 1),
    ((200, 300), "gb", 1, 9, 4, 2, 1, 1),
    ((260, 300), "sep", 2, 9, 2, 2, 0, 1),    # folded radius 4
    ((260, 300), "sep", 4, 5, 2, 1, 0, 1),    # folded radius 8
    ((300, 520), "two", 4, 5, 1, 1, 0, 2),    # wide two-term base, chosen unfolded
    ((300, 520), "two", 1, 7, 1, 2, 1, 2),    # forced, radius 1, two fused sweeps
    ((200, 300), "two", 2, 6, 1, 3, 1, 2),
    ((70, 90), "sep", 1, 8, 8, 1, 1, 1),      # a single small tile, 17 x 17 fold
]


@pytest.mark.parametrize("shape,kind,r,T,m,b,mode,k", CASES)
def test_counterpart_parity(env, shape, kind, r, T, m, b, mode, k):
    _, _, oracle = env
    c = coeffs(kind, r, 940 + T)
    x = synth.grid(950 + T, shape, np.float32)
    ref = oracle.run(x.astype(np.float64), c, T)
    y, got_k = run(env, shape, c, x, T, m, b, mode)
    err = oracle.rel_l2(y, ref)
    print("counterparts %s %s r=%d T=%d m=%d b=%d: K=%d rel-L2 %.3e"
          % (shape, kind, r, T, m, b, got_k, err))
    assert got_k == k
    assert err <= TOL
    assert np.max(np.abs(y.astype(np.float64) - ref)) <= 1e-5


@pytest.mark.parametrize("stages", [1, 2, 4])
def test_counterpart_stage_counts(env, stages):
    """Single sweeps with a ring of 1, 2 or 4 TMA stages (no early refill)."""
    _, _, oracle = env
    shape = (300, 520)
    c = coeffs("sep", 1, 960)
    x = synth.grid(961, shape, np.float32)
    T = 12
    ref = oracle.run(x.astype(np.float64), c, T)
    y, k = run(env, shape, c, x, T, 4, 1, 1, stages=stages)
    assert k == 1
    assert oracle.rel_l2(y, ref) <= TOL


def test_direct_form_for_random_weights(env):
    """Full-rank weights keep the direct form, and forcing the split is refused."""
    torch, binding, oracle = env
    shape = (200, 300)
    c = coeffs("box", 1, 970)
    x = synth.grid(971, shape, np.float32)
    ref = oracle.run(x.astype(np.float64), c, 8)
    y, k = run(env, shape, c, x, 8, 4, 1, 0)
    assert k == 0
    assert oracle.rel_l2(y, ref) <= TOL
    plan = binding.Plan(shape, c).set_option("counterparts", 1)
    xd = torch.from_numpy(x).cuda()
    assert plan.run_status(xd, torch.empty_like(xd), 8, 4) == 2  # UNSUPPORTED
    plan.close()


def test_never_option_matches(env):
    """counterparts = 2 runs the direct form on a separable base; both agree."""
    _, _, oracle = env
    shape = (256, 384)
    c = coeffs("sep", 1, 980)
    x = synth.grid(981, shape, np.float32)
    y_cp, k_cp = run(env, shape, c, x, 16, 4, 2, 0)
    y_d, k_d = run(env, shape, c, x, 16, 4, 2, 2)
    assert (k_cp, k_d) == (1, 0)
    ref = oracle.run(x.astype(np.float64), c, 16)
    assert oracle.rel_l2(y_cp, ref) <= TOL and oracle.rel_l2(y_d, ref) <= TOL


def test_autotune_respects_the_option(env, tmp_path, monkeypatch):
    """The tuning cache keys on the counterparts option: a choice tuned with the
    counterpart form (a fold with no direct kernel) is not replayed for a plan
    that forbids it."""
    torch, binding, oracle = env
    monkeypatch.setenv("STENCIL_TUNE_CACHE", str(tmp_path / "tune.jsonl"))
    shape = (256, 512)
    c = coeffs("sep", 1, 990)
    x = synth.grid(991, shape, np.float32)
    T = 24
    ref = oracle.run(x.astype(np.float64), c, T)
    for mode in (0, 2, 0, 2):
        y, k = run(env, shape, c, x, T, 0, 0, mode)
        assert oracle.rel_l2(y, ref) <= TOL
        if mode == 2:
            assert k == 0


def test_option_range(env):
    torch, binding, _ = env
    plan = binding.Plan((64, 64), coeffs("sep", 1, 995))
    for bad in (-1, 3):
        with pytest.raises(binding.StencilError):
            plan.set_option("counterparts", bad)
    for ok in (0, 1, 2):
        plan.set_option("counterparts", ok)
    plan.close()
