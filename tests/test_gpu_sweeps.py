"""GPU parity of the CUDA-core sweeps against the FP64 oracle.

Every case draws seeded inputs, runs the library through the C ABI and
compares element by element with the oracle's plain time loop.  Tolerance:
relative L2 <= 1e-5 (FP32), <= 1e-12 (FP64), and max abs error <= 1e-5 (FP32,
values in [0, 1)).  Shapes cover several 128 x 64 tiles with ragged tails,
grids narrower than one tile, and T values that leave a remainder after
folding.
"""

import numpy as np
import pytest

from paper_2103_09235_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5


@pytest.fixture(scope="module")
def env(oracle_mod):
    import torch
    from paper_2103_09235_gb300 import build, binding
    build.build()
    assert torch.cuda.is_available()
    torch.cuda.init()
    return torch, binding, oracle_mod


def gpu_run(env, shape, c, x, T, m, dtype="f32", **opts):
    torch, binding, _ = env
    plan = binding.Plan(shape, c, dtype)
    for k, v in opts.items():
        plan.set_option(k, v)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    plan.run(xd, yd, T, fold_m=m)
    plan.sync()
    y = yd.cpu().numpy()
    info = {"m": plan.get("last_m"), "b": plan.get("last_b"), "launches": plan.get("launches")}
    plan.close()
    return y, info


def check(y, ref, tol=TOL_F32, abs_tol=1e-5):
    import oracle
    err = oracle.rel_l2(y, ref)
    assert err <= tol, err
    if abs_tol is not None:
        assert np.max(np.abs(y.astype(np.float64) - ref)) <= abs_tol
    return err


CASES_2D = [
    # shape, kind, r, T, m, b
    ((64, 128), "star", 1, 5, 1, 1),
    ((300, 520), "star", 1, 17, 1, 1),
    ((300, 520), "star", 1, 17, 1, 4),
    ((37, 45), "star", 1, 9, 1, 2),
    ((300, 520), "star", 1, 21, 2, 1),
    ((300, 520), "star", 1, 21, 2, 4),
    ((129, 257), "star", 1, 30, 3, 2),
    ((300, 520), "star", 1, 41, 4, 2),
    ((300, 520), "star", 1, 41, 4, 0),
    ((300, 520), "box", 1, 13, 1, 1),
    ((300, 520), "box", 1, 13, 1, 3),
    ((129, 257), "box", 1, 22, 2, 2),
    ((300, 520), "box", 1, 25, 4, 1),
    ((300, 520), "box", 1, 25, 4, 2),
    ((41, 77), "box", 1, 11, 3, 1),
    ((200, 300), "star", 2, 9, 1, 1),
    ((200, 300), "star", 2, 9, 2, 2),
    ((200, 300), "box", 2, 7, 1, 2),
    ((200, 300), "box", 2, 7, 2, 1),
    ((90, 140), "box", 3, 5, 1, 1),
    ((90, 140), "box", 4, 5, 1, 2),
    ((130, 17), "star", 1, 12, 2, 1),
]


@pytest.mark.parametrize("shape,kind,r,T,m,b", CASES_2D)
def test_sweep2d_parity(env, shape, kind, r, T, m, b):
    _, _, oracle = env
    c = synth.dyadic_coeffs(1000 + r, 2, r, kind)
    x = synth.grid(2000 + T, shape, np.float32)
    opts = {"block_b": b} if b else {}
    y, info = gpu_run(env, shape, c, x, T, m, **opts)
    ref = oracle.run(x.astype(np.float64), c, T)
    check(y, ref)
    assert info["m"] == m


@pytest.mark.parametrize("tile_y,stages,threads", [(16, 0, 0), (32, 0, 0), (48, 0, 0), (96, 0, 0),
                                                   (128, 0, 0), (160, 1, 0), (64, 1, 0),
                                                   (64, 2, 256), (96, 1, 256), (32, 3, 0)])
def test_sweep2d_tile_shapes(env, tile_y, stages, threads):
    """Tile heights, TMA stage counts (one stage: refilled after a tile's first
    sweep) and half-size CTAs all give the oracle's result; the plan reports
    the CTA size and stage count its first pass ran with."""
    torch, binding, oracle = env
    shape = (250, 300)
    c = synth.dyadic_coeffs(7, 2, 1, "star")
    x = synth.grid(8, shape, np.float32)
    plan = binding.Plan(shape, c)
    for k, v in dict(block_b=3, tile_y=tile_y, stages=stages, cta_threads=threads).items():
        plan.set_option(k, v)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    plan.run(xd, yd, 18, fold_m=2)
    plan.sync()
    check(yd.cpu().numpy(), oracle.run(x.astype(np.float64), c, 18))
    assert plan.get("last_threads") == (256 if threads == 256 else 512)
    if stages:
        assert plan.get("last_stages") == stages
    plan.close()


CASES_1D = [
    (1000, 1, 1, "f32"), (4097, 37, 1, "f32"), (65539, 100, 1, "f32"), (65539, 100, 2, "f32"),
    (65539, 99, 3, "f32"), (4097, 37, 1, "f64"), (65539, 100, 1, "f64"), (65539, 101, 4, "f64"),
    (9, 50, 1, "f64"), (300, 64, 1, "f32"),
    # deep 1D folds (radius 8 and 16) with a plain remainder
    (65539, 101, 8, "f32"), (65539, 100, 16, "f32"), (65539, 83, 8, "f64"),
    (65539, 100, 16, "f64"), (1000, 37, 16, "f32"),
]


@pytest.mark.parametrize("n,T,m,dt", CASES_1D)
def test_sweep1d_parity(env, n, T, m, dt):
    _, _, oracle = env
    c = synth.heat1d_coeffs() if n % 2 else synth.dyadic_coeffs(5, 1, 1, "box")
    npdt = np.float64 if dt == "f64" else np.float32
    x = synth.grid(3000 + n, (n,), npdt)
    y, _ = gpu_run(env, (n,), c, x, T, m, dt)
    ref = oracle.run(x.astype(np.float64), c, T)
    if dt == "f64":
        check(y, ref, tol=1e-12, abs_tol=1e-12)
    else:
        check(y, ref)


# (n, T, m, b, dtype): exact tessellate tiling of the 1D passes (Section 3.4)
CASES_TESS = [
    (1 << 20, 100, 16, 32, "f64"), (1 << 20, 100, 6, 64, "f32"), (1 << 20, 100, 1, 32, "f32"),
    (65539, 200, 4, 16, "f32"),   # ragged: the last tile takes n mod 4096 more points
    (5000, 77, 2, 8, "f64"),      # two tiles, the second 2952 points wide
    (3000, 40, 3, 10, "f64"),     # one tile: its boundary wraps around the line
    (9000, 61, 16, 7, "f32"), (4100, 33, 12, 5, "f64"),
    (3000, 40, 4, 8, "f32"),      # one FP32 tile of strips, its boundary wrapping around
]


@pytest.mark.parametrize("tile", [256, 512, 1024, 2048, 4096])
@pytest.mark.parametrize("n,T,m,b,dt,tess", [
    (65539, 100, 4, 32, "f32", 0), (65539, 100, 6, 16, "f32", 1), (1000, 37, 2, 16, "f32", 0),
    (65539, 100, 16, 32, "f64", 1), (65539, 83, 8, 16, "f64", 0), (4097, 50, 3, 64, "f64", 1)])
def test_sweep1d_tile_sizes(env, n, T, m, b, dt, tess, tile):
    """The tile_1d option: every tile size, overlapped or tessellated (passes
    that do not fit a short tile fall back to overlapped tiles), on ragged
    lengths, matches the oracle (FP64 to 1e-12); the plan reports the size."""
    torch, binding, oracle = env
    c = synth.heat1d_coeffs() if n % 2 == 0 else synth.dyadic_coeffs(6, 1, 1, "box")
    npdt = np.float64 if dt == "f64" else np.float32
    x = synth.grid(3900 + n, (n,), npdt)
    plan = binding.Plan((n,), c, dt)
    plan.set_option("tessellate", tess).set_option("block_b", b).set_option("tile_1d", tile)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    plan.run(xd, yd, T, fold_m=m)
    plan.sync()
    assert plan.get("last_tile_y") == tile
    ref = oracle.run(x.astype(np.float64), c, T)
    if dt == "f64":
        check(yd.cpu().numpy(), ref, tol=1e-12, abs_tol=1e-12)
    else:
        check(yd.cpu().numpy(), ref)
    plan.close()


@pytest.mark.parametrize("n,T,m,b,dt", CASES_TESS)
def test_sweep1d_tessellated(env, n, T, m, b, dt):
    """Triangles then inverted triangles: every pass that fits the tile runs
    in the two-stage exact tessellation and the result matches the oracle
    (FP64 to 1e-12); the first pass reports that it was tessellated."""
    torch, binding, oracle = env
    c = synth.heat1d_coeffs() if n % 2 == 0 else synth.dyadic_coeffs(5, 1, 1, "box")
    npdt = np.float64 if dt == "f64" else np.float32
    x = synth.grid(3100 + n, (n,), npdt)
    plan = binding.Plan((n,), c, dt).set_option("tessellate", 1).set_option("block_b", b)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    plan.run(xd, yd, T, fold_m=m)
    plan.sync()
    assert plan.get("last_tess") == 1
    ref = oracle.run(x.astype(np.float64), c, T)
    y = yd.cpu().numpy()
    if dt == "f64":
        check(y, ref, tol=1e-12, abs_tol=1e-12)
    else:
        check(y, ref)
    plan.run(xd, xd, T, fold_m=m)  # in place
    plan.sync()
    if dt == "f64":
        check(xd.cpu().numpy(), ref, tol=1e-12, abs_tol=1e-12)
    else:
        check(xd.cpu().numpy(), ref)
    plan.close()


def test_sweep1d_radius2(env):
    _, _, oracle = env
    c = synth.dyadic_coeffs(9, 1, 2, "box")
    x = synth.grid(10, (5003,), np.float32)
    y, _ = gpu_run(env, (5003,), c, x, 40, 2)
    check(y, oracle.run(x.astype(np.float64), c, 40))


def test_host_pointers(env):
    """Host numpy arrays in and out: the call copies through plan-owned buffers."""
    torch, binding, oracle = env
    shape = (100, 140)
    c = synth.dyadic_coeffs(11, 2, 1, "box")
    x = synth.grid(12, shape, np.float32)
    y = np.empty_like(x)
    plan = binding.Plan(shape, c)
    plan.run(x, y, 10, fold_m=2)
    check(y, oracle.run(x.astype(np.float64), c, 10))
    x1 = synth.grid(13, (777,), np.float64)
    y1 = np.empty_like(x1)
    p1 = binding.Plan((777,), synth.heat1d_coeffs(), "f64")
    p1.run(x1, y1, 20)
    check(y1, oracle.run(x1, synth.heat1d_coeffs(), 20), tol=1e-12, abs_tol=1e-12)


@pytest.mark.parametrize("ndim", [1, 2])
def test_in_place_and_zero_steps(env, ndim):
    torch, binding, oracle = env
    shape = (5000,) if ndim == 1 else (96, 160)
    kind = "box"
    c = synth.dyadic_coeffs(14, ndim, 1, kind)
    x = synth.grid(15, shape, np.float32)
    plan = binding.Plan(shape, c)
    xd = torch.from_numpy(x).cuda()
    plan.run(xd, xd, 7, fold_m=1)
    plan.sync()
    check(xd.cpu().numpy(), oracle.run(x.astype(np.float64), c, 7))
    yd = torch.empty_like(xd)
    plan.run(xd, yd, 0)
    plan.sync()
    assert torch.equal(xd, yd)


def test_split_run_equals_whole(env):
    """run(T1) then run(T2) matches run(T1 + T2): resuming is calling again."""
    torch, binding, oracle = env
    shape = (140, 200)
    c = synth.dyadic_coeffs(16, 2, 1, "star")
    x = synth.grid(17, shape, np.float32)
    plan = binding.Plan(shape, c)
    xd = torch.from_numpy(x).cuda()
    y1, y2 = torch.empty_like(xd), torch.empty_like(xd)
    plan.run(xd, y1, 12, fold_m=4)
    plan.run(y1, y2, 9, fold_m=2)
    plan.sync()
    check(y2.cpu().numpy(), oracle.run(x.astype(np.float64), c, 21))


@pytest.mark.parametrize("ndim,r,kind,m", [(1, 1, "box", 5), (2, 1, "star", 4), (2, 1, "box", 4),
                                           (2, 1, "box", 8), (2, 2, "star", 3), (3, 1, "star", 2),
                                           (3, 1, "box", 2)])
def test_folded_coeffs_fp64_on_gpu(env, ndim, r, kind, m):
    """The plan's FP64 folded weights (computed by a GPU kernel) equal the oracle's."""
    torch, binding, oracle = env
    c = synth.dyadic_coeffs(18 + m, ndim, r, kind)
    shape = (64,) * ndim
    plan = binding.Plan(shape, c)
    got = plan.folded_coeffs(m)
    ref = oracle.fold_coeffs(c, m)
    assert got.shape == ref.shape
    assert np.max(np.abs(got - ref)) < 1e-15


def test_rel_l2_on_gpu(env):
    torch, binding, oracle = env
    ref = synth.grid(19, (1000, 37), np.float64)
    y = (ref + 1e-3 * synth.grid(20, (1000, 37), np.float64)).astype(np.float32)
    got = binding.rel_l2(torch.from_numpy(y).cuda(), torch.from_numpy(ref).cuda())
    assert abs(got[0] - oracle.rel_l2(y, ref)) < 1e-12
    assert abs(got[1] - oracle.rel_l2_zero_mean(y, ref)) < 1e-9


def test_bad_fold_rejected(env):
    torch, binding, _ = env
    plan = binding.Plan((20, 20), synth.dyadic_coeffs(1, 2, 1, "star"))
    x = torch.zeros((20, 20), device="cuda")
    assert plan.run_status(x, x, 10, 10) == 1   # folded width 21 > 20
    assert plan.run_status(x, x, -1, 1) == 1


@pytest.mark.parametrize("m,b,stages", [(1, 1, 0), (2, 2, 0), (2, 2, 1)])
def test_bounded_wait_reports_timeout(env, m, b, stages):
    """A copy that never arrives ends the kernel's wait with a status, not a hang
    (single sweeps, and blocked sweeps whose stage is refilled early)."""
    torch, binding, oracle = env
    shape = (200, 260)
    c = synth.dyadic_coeffs(21, 2, 1, "star")
    x = synth.grid(22, shape, np.float32)
    plan = binding.Plan(shape, c).set_option("block_b", b).set_option("stages", stages)
    plan.set_option("wait_limit_ms", 50).set_option("fault_withhold_copy", 1)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    T = 2 * m * b
    plan.run(xd, yd, T, fold_m=m)
    assert plan.sync_status() == 5
    assert plan.sync_status() == 0          # cleared
    plan.set_option("fault_withhold_copy", 0)
    plan.run(xd, yd, T, fold_m=m)            # the context is still usable
    plan.sync()
    check(yd.cpu().numpy(), oracle.run(x.astype(np.float64), c, T))


@pytest.mark.parametrize("kind,m,b", [("star", 1, 1), ("box", 2, 1), ("star", 1, 2), ("star", 2, 2)])
def test_bounded_wait_reports_timeout_3d(env, kind, m, b):
    """Both 3D kernels (single sweeps, b = 1, and two fused sweeps, b = 2): a
    withheld chunk ends the consumer warps' waits and the producer's with a
    status, for a padded destination (ghost refresh) and the dense last pass
    alike; the next run is correct."""
    torch, binding, oracle = env
    shape = (40, 48, 64)
    c = synth.dyadic_coeffs(23, 3, 1, kind)
    x = synth.grid(24, shape, np.float32)
    plan = binding.Plan(shape, c).set_option("block_b", b)
    plan.set_option("wait_limit_ms", 50).set_option("fault_withhold_copy", 1)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    T = 2 * m * b
    plan.run(xd, yd, T, fold_m=m)
    assert plan.get("last_b") == b
    assert plan.sync_status() == 5
    assert plan.sync_status() == 0
    plan.set_option("fault_withhold_copy", 0)
    plan.run(xd, yd, T, fold_m=m)
    plan.sync()
    check(yd.cpu().numpy(), oracle.run(x.astype(np.float64), c, T))


def test_graph_replay_matches_direct_launches(env):
    """A run replayed from its captured graph equals the same run launched kernel by kernel."""
    torch, binding, oracle = env
    shape = (300, 520)
    c = synth.dyadic_coeffs(23, 2, 1, "box")
    x = synth.grid(24, shape, np.float32)
    xd = torch.from_numpy(x).cuda()
    outs = []
    for graph in (1, 1, 0):
        plan = binding.Plan(shape, c).set_option("graph", graph).set_option("block_b", 2)
        y = torch.empty_like(xd)
        plan.run(xd, y, 37, fold_m=3)
        plan.run(xd, y, 37, fold_m=3)     # second call replays the captured graph
        plan.sync()
        outs.append(y.cpu().numpy())
        plan.close()
    assert np.array_equal(outs[0], outs[2]) and np.array_equal(outs[1], outs[2])
    check(outs[0], oracle.run(x.astype(np.float64), c, 37))


def test_run_inside_user_stream_capture(env):
    """stencil_run enqueued while the caller captures a CUDA graph (after a warm-up run)."""
    torch, binding, oracle = env
    shape = (200, 256)
    c = synth.dyadic_coeffs(25, 2, 1, "star")
    x = synth.grid(26, shape, np.float32)
    plan = binding.Plan(shape, c)
    xd = torch.from_numpy(x).cuda()
    y = torch.empty_like(xd)
    plan.run(xd, y, 20, fold_m=2)
    torch.cuda.synchronize()
    y.zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.run(xd, y, 20, fold_m=2, stream=s)
    g.replay()
    torch.cuda.synchronize()
    check(y.cpu().numpy(), oracle.run(x.astype(np.float64), c, 20))


CASES_3D = [
    # shape (z, y, x), kind, r, T, m
    ((100, 40, 70), "star", 1, 6, 1),
    ((100, 40, 70), "box", 1, 5, 1),
    ((100, 40, 70), "star", 1, 9, 2),
    ((66, 33, 130), "box", 1, 7, 2),
    ((40, 36, 64), "star", 2, 4, 1),
    ((40, 36, 64), "box", 2, 3, 1),
    ((12, 9, 11), "star", 1, 5, 2),
    # ghost bands overlapping in every axis; many z chunks per tile column
    ((7, 6, 9), "box", 1, 4, 2),
    ((150, 20, 24), "star", 1, 5, 2),
    ((150, 20, 24), "box", 1, 4, 1),
]


@pytest.mark.parametrize("stages", [0, 2, 3])
@pytest.mark.parametrize("shape,kind,r,T,m", CASES_3D)
def test_sweep3d_parity(env, shape, kind, r, T, m, stages):
    """Single 3D sweeps with the automatic ring and with 2 and 3 stages."""
    _, _, oracle = env
    c = synth.dyadic_coeffs(3100 + r, 3, r, kind)
    x = synth.grid(3200 + T, shape, np.float32)
    y, info = gpu_run(env, shape, c, x, T, m, block_b=1, stages=stages)
    ref = oracle.run(x.astype(np.float64), c, T)
    check(y, ref)
    assert info["m"] == m


@pytest.mark.parametrize("zc", [2, 4, 6, 8, 14, 32, 1024])
@pytest.mark.parametrize("shape,kind,m", [((150, 20, 24), "box", 1), ((100, 40, 70), "star", 2)])
def test_sweep3d_z_chunk(env, shape, kind, m, zc):
    """The z_chunk option (output planes per CTA): chunks shorter than the halo,
    longer than the grid, and between all give the oracle's result."""
    _, _, oracle = env
    c = synth.dyadic_coeffs(3150, 3, 1, kind)
    x = synth.grid(3151, shape, np.float32)
    y, info = gpu_run(env, shape, c, x, 7, m, block_b=1, z_chunk=zc)
    check(y, oracle.run(x.astype(np.float64), c, 7))
    assert info["m"] == m


CASES_3D_PERSISTENT = [
    # shape (z, y, x), kind, r, T, m, z_chunk: many passes in one persistent
    # launch; ragged tiles, tiny grids (one or two tiles per axis, so a piece
    # is its own periodic neighbour), many z chunks, folded runs with a plain
    # remainder, and fewer items per pass than resident CTAs
    ((100, 40, 70), "star", 1, 23, 1, 0),
    ((100, 40, 70), "box", 1, 21, 1, 0),
    ((66, 33, 130), "box", 1, 17, 2, 0),
    ((100, 40, 70), "star", 1, 19, 2, 8),
    ((40, 36, 64), "star", 2, 12, 1, 0),
    ((40, 36, 64), "box", 2, 9, 1, 4),
    ((12, 9, 11), "star", 1, 15, 2, 0),
    ((7, 6, 9), "box", 1, 14, 1, 4),
    ((150, 20, 24), "box", 1, 25, 1, 8),
    ((150, 20, 24), "box", 1, 19, 1, 6),
    ((100, 40, 70), "star", 1, 17, 1, 14),
    ((150, 20, 24), "star", 1, 31, 3, 0),
    ((96, 80, 200), "box", 1, 12, 1, 0),
]


@pytest.mark.parametrize("shape,kind,r,T,m,zc", CASES_3D_PERSISTENT)
def test_sweep3d_persistent(env, shape, kind, r, T, m, zc):
    """The persistent multi-pass launch: bit-identical to one launch per pass
    (the same arithmetic in the same order) and within the oracle's bounds;
    the passes of one stencil take one launch."""
    _, _, oracle = env
    c = synth.dyadic_coeffs(3300 + r, 3, r, kind)
    x = synth.grid(3400 + T, shape, np.float32)
    y0, i0 = gpu_run(env, shape, c, x, T, m, block_b=1, z_chunk=zc, persistent=0)
    y1, i1 = gpu_run(env, shape, c, x, T, m, block_b=1, z_chunk=zc, persistent=1)
    assert np.array_equal(y0, y1)
    check(y1, oracle.run(x.astype(np.float64), c, T))
    assert i1["m"] == m
    nfold, rem = divmod(T, m)
    per_pass = nfold + rem
    groups = (nfold >= 2) + (rem >= 2) + (nfold == 1) + (rem == 1)
    assert i0["launches"] - i1["launches"] == per_pass - groups


@pytest.mark.parametrize("shape,expect", [((256, 256, 256), 1), ((64, 64, 64), 0)])
def test_sweep3d_persistent_automatic(env, shape, expect):
    """The automatic choice (persistent option -1): one persistent launch when
    a pass has between one and 3.5 waves of pieces (the 256^3 grid: 1024
    pieces on 608 resident CTAs), one launch per pass for a grid with fewer
    pieces than CTAs; the result is the oracle's either way (checked at 64^3)."""
    torch, binding, oracle = env
    c = synth.dyadic_coeffs(3500, 3, 1, "box")
    x = synth.grid(3501, shape, np.float32)
    plan = binding.Plan(shape, c).set_option("block_b", 1).set_option("autotune", 0)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    plan.run(xd, yd, 4, fold_m=1)
    plan.sync()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    if shape[0] == 256 and sms == 152:
        assert plan.get("last_persistent") == expect
    if shape[0] == 64:
        assert plan.get("last_persistent") == expect
        check(yd.cpu().numpy(), oracle.run(x.astype(np.float64), c, 4))
    plan.close()


@pytest.mark.parametrize("in_place", [False, True])
def test_sweep3d_persistent_replay_and_in_place(env, in_place):
    """A second run of the same persistent 3D launch replays its captured graph
    (the pass counters are zeroed inside it) and gives the same result; in
    place (in == out) the input is imported before the first pass."""
    torch, binding, oracle = env
    shape = (70, 48, 100)
    c = synth.dyadic_coeffs(3800, 3, 1, "box")
    x = synth.grid(3801, shape, np.float32)
    ref = oracle.run(x.astype(np.float64), c, 13)
    plan = binding.Plan(shape, c).set_option("block_b", 1).set_option("persistent", 1)
    outs = []
    for _ in range(2):
        xd = torch.from_numpy(x).cuda()
        yd = xd if in_place else torch.empty_like(xd)
        plan.run(xd, yd, 13, fold_m=1)
        plan.sync()
        assert plan.get("last_persistent") == 1
        outs.append(yd.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    check(outs[1], ref)
    plan.close()


@pytest.mark.parametrize("hook", ["fault_withhold_dep", "fault_withhold_copy"])
def test_bounded_wait_reports_timeout_3d_persistent(env, hook):
    """The persistent 3D launch: dependencies that never count as met, or a
    withheld chunk, end the producer's and the consumers' bounded waits with
    a status; the next run is correct."""
    torch, binding, oracle = env
    shape = (40, 48, 64)
    c = synth.dyadic_coeffs(25, 3, 1, "box")
    x = synth.grid(26, shape, np.float32)
    plan = binding.Plan(shape, c).set_option("block_b", 1).set_option("persistent", 1)
    plan.set_option("wait_limit_ms", 50).set_option(hook, 1)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    plan.run(xd, yd, 6, fold_m=1)
    assert plan.sync_status() == 5
    assert plan.sync_status() == 0
    plan.set_option(hook, 0)
    plan.run(xd, yd, 6, fold_m=1)
    plan.sync()
    check(yd.cpu().numpy(), oracle.run(x.astype(np.float64), c, 6))
    plan.close()


CASES_3D_FUSED = [
    # shape (z, y, x), kind, r, T, m: two fused sweeps per pass (block_b = 2)
    ((100, 40, 70), "star", 1, 7, 1),    # three pairs and one single sweep
    ((100, 40, 70), "box", 1, 6, 1),
    ((100, 40, 70), "star", 1, 9, 2),    # two folded pairs, then the plain step
    ((66, 33, 130), "box", 1, 10, 2),    # two pairs and one single folded sweep
    ((40, 36, 64), "star", 2, 5, 1),
    ((12, 9, 11), "star", 1, 6, 1),      # ghost bands overlapping in every axis
    ((7, 6, 9), "box", 1, 5, 1),
    ((150, 20, 24), "star", 1, 11, 2),   # many z chunks per tile column
]


@pytest.mark.parametrize("shape,kind,r,T,m", CASES_3D_FUSED)
def test_sweep3d_fused_pairs(env, shape, kind, r, T, m):
    """3D temporal blocking: two sweeps per HBM round trip match the oracle."""
    _, _, oracle = env
    c = synth.dyadic_coeffs(3400 + r, 3, r, kind)
    x = synth.grid(3500 + T, shape, np.float32)
    y, info = gpu_run(env, shape, c, x, T, m, block_b=2)
    check(y, oracle.run(x.astype(np.float64), c, T))
    assert info["m"] == m and info["b"] == 2


def test_sweep3d_fused_pairs_rejects_wide(env):
    """A fused pair needs folded radius <= 2 and a ghost band of 2R."""
    torch, binding, _ = env
    c = synth.dyadic_coeffs(3600, 3, 1, "star")
    plan = binding.Plan((40, 40, 40), c).set_option("block_b", 2)
    x = torch.zeros((40, 40, 40), device="cuda")
    with pytest.raises(binding.StencilError) as ei:
        plan.run(x, x, 12, fold_m=3)
    assert ei.value.status == 2
    with pytest.raises(binding.StencilError):
        binding.Plan((40, 40, 40), c).set_option("block_b", 3).run(x, x, 12, fold_m=1)
    plan.close()


@pytest.mark.parametrize("shape,kind", [((300, 520), "star"), ((260, 300), "box"), ((6000,), "box"),
                                        ((40, 36, 70), "star")])
def test_autotune_choice_is_correct_and_cached(env, shape, kind, tmp_path, monkeypatch):
    """fold_m = 0 times candidates, runs the fastest and caches the choice on disk."""
    torch, binding, oracle = env
    monkeypatch.setenv("STENCIL_TUNE_CACHE", str(tmp_path / "tune.jsonl"))
    c = synth.dyadic_coeffs(27, len(shape), 1, kind)
    x = synth.grid(28, shape, np.float32)
    y, info = gpu_run(env, shape, c, x, 37, 0)
    check(y, oracle.run(x.astype(np.float64), c, 37))
    assert info["m"] >= 1
    lines = (tmp_path / "tune.jsonl").read_text().strip().splitlines()
    assert len(lines) == 1 and '"m": %d' % info["m"] in lines[0]
    y2, info2 = gpu_run(env, shape, c, x, 37, 0)      # a new plan hits the file cache
    assert info2["m"] == info["m"]
    assert len((tmp_path / "tune.jsonl").read_text().strip().splitlines()) == 1
    assert np.array_equal(y, y2)


@pytest.mark.parametrize("shape,T,m", [((70, 40, 66), 10, 3), ((40, 36, 70), 9, 4)])
def test_sweep3d_deeper_folds(env, shape, T, m):
    _, _, oracle = env
    c = synth.dyadic_coeffs(3300, 3, 1, "star")
    x = synth.grid(3301, shape, np.float32)
    y, info = gpu_run(env, shape, c, x, T, m)
    check(y, oracle.run(x.astype(np.float64), c, T))
