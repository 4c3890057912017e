"""The allocation-free 1D entry point against the plan-based one.

stencil_run_1d_noalloc serves callers that cannot call cudaMalloc (a graph
capture that forbids allocation, a framework that owns all device memory, a
deployment that must not allocate after start-up).  This file is collected
last so that a stop at the first failure has already run every other test.
Each case calls the new entry point twice in a row through the C ABI and
compares both results with stencil_run on a plan, within the FP32 and FP64
tolerances the other parity tests use.
"""

import numpy as np
import pytest

from paper_2103_09235_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2103_09235_gb300 import build, binding
    build.build()
    assert torch.cuda.is_available()
    torch.cuda.init()
    return torch, binding


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("n,T,dt,inplace", [(1 << 20, 100, "f32", False), (65539, 37, "f32", True),
                                            (4097, 64, "f64", False), (5000, 33, "f64", True),
                                            (1000, 1, "f32", True)])
def test_noalloc_matches_plan_run(env, n, T, dt, inplace):
    torch, binding = env
    c = synth.heat1d_coeffs() if n % 2 == 0 else synth.dyadic_coeffs(77, 1, 1, "box")
    npdt = np.float64 if dt == "f64" else np.float32
    tol = 1e-12 if dt == "f64" else 1e-5
    x = synth.grid(4000 + n, (n,), npdt)
    plan = binding.Plan((n,), c, dt)
    xd = torch.from_numpy(x).cuda()
    ref = torch.empty_like(xd)
    plan.run(xd, ref, T, fold_m=1)
    plan.sync()
    ref_h = ref.cpu().numpy()
    for _ in range(2):
        if inplace:
            y = xd.clone()
            binding.run_1d_noalloc(y, y, c, T)
        else:
            y = torch.empty_like(xd)
            binding.run_1d_noalloc(xd, y, c, T)
        torch.cuda.synchronize()
        assert rel_l2(y.cpu().numpy(), ref_h) <= tol
    plan.close()


def test_noalloc_rejects_oversize_grid(env):
    torch, binding = env
    x = torch.zeros((1 << 21) + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.StencilError) as ei:
        binding.run_1d_noalloc(x, x, synth.heat1d_coeffs(), 3)
    assert ei.value.status == 1
    assert "16777216" in str(ei.value)
