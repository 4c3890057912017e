"""GPU parity of the tcgen05 folded box sweep (BF16 hi/lo split) against the
FP64 oracle.

BF16X3 must reach relative L2 <= 1e-5 after T steps; the single-product
BF16X1 error is reported beside it and must be larger.  Shapes span several
128 x 32 tiles with ragged tails in both directions; T leaves a remainder
after folding so the CUDA-core plain sweep finishes the run.
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


def run_tc(env, shape, c, x, T, m, precision=1, center=1, form=0):
    torch, binding, _ = env
    plan = binding.Plan(shape, c)
    plan.set_option("precision", precision).set_option("tc_center", center)
    plan.set_option("tc_form", form)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    plan.run(xd, yd, T, fold_m=m)
    plan.sync()
    assert plan.get("last_engine") == 1
    R = m * (c.shape[0] // 2)
    want = form if form else (2 if R >= 6 else 1)
    assert plan.get("last_tc_form") == want
    y = yd.cpu().numpy()
    plan.close()
    return y


CASES = [
    # shape, r, T, m
    ((300, 520), 1, 13, 4),
    # ragged in x and y, two folded sweeps and no remainder: the first sweep's
    # ragged tiles must not leave by the clipped TMA store
    ((97, 203), 1, 8, 4),
    ((300, 520), 1, 16, 2),
    ((256, 256), 1, 12, 3),
    ((300, 520), 1, 27, 8),
    ((130, 70), 1, 9, 4),
    ((200, 300), 2, 10, 2),
    ((200, 300), 2, 9, 4),
]


@pytest.mark.parametrize("form", [1, 2])
@pytest.mark.parametrize("shape,r,T,m", CASES)
def test_tc_bf16x3_parity(env, shape, r, T, m, form):
    """Both tensor-core kernels: one MMA per row offset (1) and four offsets per MMA (2)."""
    _, _, oracle = env
    c = synth.dyadic_coeffs(500 + r, 2, r, "box")
    x = synth.grid(600 + T, shape, np.float32)
    ref = oracle.run(x.astype(np.float64), c, T)
    y3 = run_tc(env, shape, c, x, T, m, precision=1, form=form)
    err3 = oracle.rel_l2(y3, ref)
    y1 = run_tc(env, shape, c, x, T, m, precision=2, form=form)
    err1 = oracle.rel_l2(y1, ref)
    print("TC form %d %s r=%d T=%d m=%d: BF16x3 rel-L2 %.3e, BF16x1 rel-L2 %.3e"
          % (form, shape, r, T, m, err3, err1))
    assert err3 <= TOL
    assert err1 > err3


def test_tc_without_centering(env):
    """Without subtracting the grid mean the split is still accurate to 1e-5 here."""
    _, _, oracle = env
    shape = (300, 520)
    c = synth.dyadic_coeffs(501, 2, 1, "box")
    x = synth.grid(700, shape, np.float32)
    ref = oracle.run(x.astype(np.float64), c, 20)
    y = run_tc(env, shape, c, x, 20, 4, precision=1, center=0)
    err = oracle.rel_l2(y, ref)
    print("TC no centering rel-L2 %.3e" % err)
    assert err <= TOL


@pytest.mark.parametrize("shape,T,m", [((300, 520), 21, 4), ((256, 384), 14, 2)])
def test_tc_star_parity(env, shape, T, m):
    """A folded star is a diamond inside the (2R+1)^2 window: the panels carry its zeros."""
    _, _, oracle = env
    c = synth.dyadic_coeffs(800, 2, 1, "star")
    x = synth.grid(801, shape, np.float32)
    ref = oracle.run(x.astype(np.float64), c, T)
    y = run_tc(env, shape, c, x, T, m, precision=1)
    err = oracle.rel_l2(y, ref)
    print("TC star %s T=%d m=%d rel-L2 %.3e" % (shape, T, m, err))
    assert err <= TOL


@pytest.mark.parametrize("form", [1, 2])
def test_tc_bounded_waits_report_timeout(env, form):
    """Both tensor-core kernels: with the test hook that stops the MMA issuer
    before its first MMA, the producer's, converters' and epilogue's bounded
    waits run out (50 ms), the status reads TIMEOUT, tensor memory is freed,
    and the next run on the same plan matches the oracle."""
    torch, binding, oracle = env
    shape, T, m = (300, 520), 13, 4
    c = synth.dyadic_coeffs(31, 2, 1, "box")
    x = synth.grid(32, shape, np.float32)
    plan = binding.Plan(shape, c).set_option("precision", 1).set_option("tc_form", form)
    plan.set_option("wait_limit_ms", 50).set_option("fault_withhold_mma", 1)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    plan.run(xd, yd, T, fold_m=m)
    assert plan.sync_status() == 5
    assert plan.sync_status() == 0
    plan.set_option("fault_withhold_mma", 0)
    plan.run(xd, yd, T, fold_m=m)
    plan.sync()
    assert plan.get("last_engine") == 1 and plan.get("last_tc_form") == form
    assert oracle.rel_l2(yd.cpu().numpy(), oracle.run(x.astype(np.float64), c, T)) <= 1e-5
    plan.close()


TF32_CASES = [((300, 520), 1, 13, 4), ((256, 256), 1, 12, 3), ((300, 520), 1, 16, 2),
              ((130, 70), 1, 9, 4), ((200, 300), 2, 10, 2), ((97, 203), 1, 11, 4)]


@pytest.mark.parametrize("shape,r,T,m", TF32_CASES)
def test_tc_tf32x3_parity(env, shape, r, T, m):
    """TF32 hi/lo operands (kind::tf32, three products): about 22 significant
    bits per operand pair, so the error sits below the BF16x3 split's on the
    same case; both within the FP32 tolerance."""
    _, _, oracle = env
    c = synth.dyadic_coeffs(500 + r, 2, r, "box")
    x = synth.grid(600 + T, shape, np.float32)
    ref = oracle.run(x.astype(np.float64), c, T)
    yt = run_tc(env, shape, c, x, T, m, precision=3, form=1)
    yb = run_tc(env, shape, c, x, T, m, precision=1, form=1)
    et, eb = oracle.rel_l2(yt, ref), oracle.rel_l2(yb, ref)
    print("TC %s r=%d T=%d m=%d: TF32x3 rel-L2 %.3e, BF16x3 rel-L2 %.3e" % (shape, r, T, m, et, eb))
    assert et <= TOL
    # the TF32 split is exact to about 2^-22, below the FP32 rounding of the
    # accumulation and output: the error sits at the FP32 floor
    assert et <= 3e-7


def test_tc_tf32x3_rejects_wide_folds(env):
    torch, binding, _ = env
    c = synth.dyadic_coeffs(501, 2, 1, "box")
    plan = binding.Plan((200, 200), c).set_option("precision", 3)
    x = torch.zeros((200, 200), device="cuda")
    assert plan.run_status(x, x, 12, 6) == 2  # folded radius 6 > 4: UNSUPPORTED
    plan.close()



TC3D_CASES = [
    # shape (z, y, x), kind, r, T, m
    ((40, 36, 70), "box", 1, 7, 2),      # three folded sweeps and one plain step
    ((20, 30, 40), "box", 1, 4, 2),      # no remainder
    ((33, 140, 64), "star", 1, 9, 4),    # two ragged y tiles per plane
    ((24, 24, 24), "box", 2, 5, 2),      # folded radius 4
    ((12, 9, 70), "star", 1, 6, 2),      # ghost bands overlapping in z and y
]


@pytest.mark.parametrize("shape,kind,r,T,m", TC3D_CASES)
def test_tc3d_parity(env, shape, kind, r, T, m):
    """3D folded sweeps on the tensor cores: per sweep one per-offset launch per
    plane offset dz, over every plane, the terms added in the output grid."""
    torch, binding, oracle = env
    c = synth.dyadic_coeffs(3700 + r, 3, r, kind)
    x = synth.grid(3800 + T, shape, np.float32)
    ref = oracle.run(x.astype(np.float64), c, T)
    errs = {}
    for prec in (1, 2) + ((3,) if m * r <= 4 else ()):
        plan = binding.Plan(shape, c).set_option("precision", prec)
        xd = torch.from_numpy(x).cuda()
        yd = torch.empty_like(xd)
        plan.run(xd, yd, T, fold_m=m)
        plan.sync()
        assert plan.get("last_engine") == 1 and plan.get("last_m") == m
        errs[prec] = oracle.rel_l2(yd.cpu().numpy(), ref)
        plan.close()
    print("TC 3D %s %s r=%d T=%d m=%d: %s" % (shape, kind, r, T, m,
          ", ".join("prec %d rel-L2 %.3e" % kv for kv in sorted(errs.items()))))
    assert errs[1] <= TOL and errs[2] > errs[1]
    if 3 in errs:
        assert errs[3] <= TOL


def test_tc3d_in_place_and_uncentred(env):
    """in == out, and the split without subtracting the grid mean."""
    torch, binding, oracle = env
    shape = (30, 40, 50)
    c = synth.dyadic_coeffs(3900, 3, 1, "box")
    x = synth.grid(3901, shape, np.float32)
    ref = oracle.run(x.astype(np.float64), c, 9)
    plan = binding.Plan(shape, c).set_option("precision", 1).set_option("tc_center", 0)
    xd = torch.from_numpy(x).cuda()
    plan.run(xd, xd, 9, fold_m=2)
    plan.sync()
    assert oracle.rel_l2(xd.cpu().numpy(), ref) <= TOL
    plan.close()


def test_tc3d_bounded_waits_report_timeout(env):
    """With the hook that stops the MMA issuer, the 3D tensor-core terms' waits
    run out, the status reads TIMEOUT, and the next run matches the oracle."""
    torch, binding, oracle = env
    shape, T, m = (20, 30, 40), 5, 2
    c = synth.dyadic_coeffs(3902, 3, 1, "box")
    x = synth.grid(3903, shape, np.float32)
    plan = binding.Plan(shape, c).set_option("precision", 1)
    plan.set_option("wait_limit_ms", 50).set_option("fault_withhold_mma", 1)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    plan.run(xd, yd, T, fold_m=m)
    assert plan.sync_status() == 5
    assert plan.sync_status() == 0
    plan.set_option("fault_withhold_mma", 0)
    plan.run(xd, yd, T, fold_m=m)
    plan.sync()
    assert oracle.rel_l2(yd.cpu().numpy(), oracle.run(x.astype(np.float64), c, T)) <= TOL
    plan.close()

