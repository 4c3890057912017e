"""The allocation-free 1D entry point against the plan-based one and the oracle.

stencil_run_1d_noalloc serves callers that cannot call cudaMalloc: code inside
a framework whose own allocator owns all device memory, and deployments that
must not touch the allocator after start-up.  This file is collected last so
that a stop at the first failure has already run every other test.

Each case calls the new entry point twice in a row through the C ABI and
compares both results with stencil_run on a plan (the existing entry point)
and with the FP64 oracle's plain time loop, within the FP32 and FP64
tolerances the other parity tests use (relative L2 <= 1e-5 and <= 1e-12).
The cases reach every pass schedule of the entry point: out of place with an
even and an odd pass count, in place with a pass count raised by one (and
then shortened passes), and the one-step in-place path.
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


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# (n, T, dtype, in place): passes of up to 32 steps.
#   (1<<20, 100, f32, out)  4 passes, the first into the scratch array
#   (65539, 65, f32, out)   3 passes, the first straight into `out`
#   (4097, 64, f64, out)    2 passes
#   (65539, 37, f32, in)    2 passes, the first into the scratch array
#   (5000, 33, f64, in)     2 passes
#   (4097, 20, f64, in)     1 pass raised to 2 (19 + 1 steps)
#   (5000, 65, f64, in)     3 passes raised to 4 (32 + 31 + 1 + 1 steps)
#   (1000, 1, f32, in)      one step through the scratch array and a copy back
CASES = [(1 << 20, 100, "f32", False), (65539, 65, "f32", False), (4097, 64, "f64", False),
         (65539, 37, "f32", True), (5000, 33, "f64", True), (4097, 20, "f64", True),
         (5000, 65, "f64", True), (1000, 1, "f32", True)]


@pytest.mark.parametrize("n,T,dt,inplace", CASES)
def test_noalloc_matches_plan_run_and_oracle(env, n, T, dt, inplace):
    torch, binding, oracle = env
    c = synth.heat1d_coeffs() if n % 2 == 0 else synth.dyadic_coeffs(77, 1, 1, "box")
    npdt = np.float64 if dt == "f64" else np.float32
    tol = 1e-12 if dt == "f64" else 1e-5
    x = synth.grid(4000 + n, (n,), npdt)
    want = oracle.run(x.astype(np.float64), c, T)
    plan = binding.Plan((n,), c, dt)
    xd = torch.from_numpy(x).cuda()
    ref = torch.empty_like(xd)
    plan.run(xd, ref, T, fold_m=1)
    plan.sync()
    ref_h = ref.cpu().numpy()
    assert rel_l2(ref_h, want) <= tol
    for _ in range(2):
        if inplace:
            y = xd.clone()
            binding.run_1d_noalloc(y, y, c, T)
        else:
            y = torch.empty_like(xd)
            binding.run_1d_noalloc(xd, y, c, T)
        torch.cuda.synchronize()
        y_h = y.cpu().numpy()
        assert rel_l2(y_h, ref_h) <= tol
        assert rel_l2(y_h, want) <= tol
    plan.close()


def test_noalloc_rejects_oversize_grid(env):
    torch, binding, _ = env
    x = torch.zeros((1 << 21) + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.StencilError) as ei:
        binding.run_1d_noalloc(x, x, synth.heat1d_coeffs(), 3)
    assert ei.value.status == 1
    assert "16777216" in str(ei.value)
