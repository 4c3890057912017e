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


def _batch_plans(binding, torch, specs):
    plans, xs, ys, refs_in = [], [], [], []
    for j, (shape, kind, r, T, seed) in enumerate(specs):
        c = synth.dyadic_coeffs(seed, 2, r, kind)
        x = synth.grid(seed + 7, shape, np.float32)
        plans.append(binding.Plan(shape, c))
        xs.append(torch.from_numpy(x).cuda())
        ys.append(torch.full_like(xs[-1], float("nan")))
        refs_in.append((x, c, T))
    return plans, xs, ys, refs_in


SPECS = [((200, 300), "star", 1, 40, 9300), ((150, 140), "box", 1, 33, 9301),
         ((256, 200), "star", 1, 57, 9302), ((180, 230), "box", 1, 21, 9303)]


def test_batched_autotuner_tunes_and_caches(env, tmp_path, monkeypatch):
    """fold_m = 0 for every grid: the batch autotuner times (m, b) per class of
    grids and the tile height, writes its choices to the cache file, and the
    run matches the oracle."""
    torch, binding, oracle = env
    cache = tmp_path / "tune.jsonl"
    monkeypatch.setenv("STENCIL_TUNE_CACHE", str(cache))
    plans, xs, ys, refs_in = _batch_plans(binding, torch, SPECS)
    binding.run_batched(plans, xs, ys, [t for _, _, t in refs_in])
    plans[0].sync()
    for y, (x, c, T) in zip(ys, refs_in):
        assert oracle.rel_l2(y.cpu().numpy(), oracle.run(x.astype(np.float64), c, T)) <= 1e-5
    text = cache.read_text()
    assert text.count('"key": "batched|2d|') >= 2 and '"key": "batched-tile|' in text
    for p in plans:
        p.close()


@pytest.mark.parametrize("threads", [512, 256])
def test_batched_uses_cached_choice(env, tmp_path, monkeypatch, threads):
    """A cache entry decides the fold and blocking depth the batched launch
    picks for its class of grids (here: stars m = 1, b = 3; boxes m = 2, b = 1),
    and the batch's tile height and CTA shape."""
    import math
    torch, binding, oracle = env
    gpu = torch.cuda.get_device_name()
    cache = tmp_path / "tune.jsonl"
    lines, classes = [], []
    for shape, kind, r, T, seed in SPECS:
        pat = 0 if kind == "star" else 1
        cls = (r, pat, int(math.floor(math.log2(shape[0] * shape[1]))))
        if cls not in classes:
            classes.append(cls)
        val = "1 3" if kind == "star" else "2 1"
        lines.append('{"key": "batched|2d|r%d|pat%d|area2^%d|f32|%s", "value": "%s"}'
                     % (cls + (gpu, val)))
    tile = "batched-tile|" + "".join("r%d.p%d.a%d;" % c for c in sorted(classes)) + "|" + gpu
    lines.append('{"key": "%s", "value": "48 %d"}' % (tile, threads))
    cache.write_text("\n".join(lines) + "\n")
    monkeypatch.setenv("STENCIL_TUNE_CACHE", str(cache))
    plans, xs, ys, refs_in = _batch_plans(binding, torch, SPECS)
    binding.run_batched(plans, xs, ys, [t for _, _, t in refs_in])
    plans[0].sync()
    for p, (shape, kind, r, T, seed) in zip(plans, SPECS):
        assert (p.get("last_m"), p.get("last_b")) == ((1, 3) if kind == "star" else (2, 1))
        assert p.get("last_tile_y") == 48 and p.get("last_threads") == threads
    for y, (x, c, T) in zip(ys, refs_in):
        assert oracle.rel_l2(y.cpu().numpy(), oracle.run(x.astype(np.float64), c, T)) <= 1e-5
    for p in plans:
        p.close()


def _class_keys(specs):
    import math
    classes = []
    for shape, kind, r, T, seed in specs:
        cls = (r, 0 if kind == "star" else 1, int(math.floor(math.log2(shape[0] * shape[1]))))
        if cls not in classes:
            classes.append(cls)
    return sorted(classes)


def test_batched_composition_entry_wins(env, tmp_path, monkeypatch):
    """A batch composition's cache entry carries its own per-class choices
    ("tile_y threads" then "m b" per class in class order) and they take
    precedence over the per-class entries another batch may have written."""
    torch, binding, oracle = env
    gpu = torch.cuda.get_device_name()
    classes = _class_keys(SPECS)
    lines = ['{"key": "batched|2d|r%d|pat%d|area2^%d|f32|%s", "value": "1 3"}' % (c + (gpu,))
             for c in classes]
    own = " ".join("3 2" if c[1] == 0 else "2 2" for c in classes)
    tile = "batched-tile|" + "".join("r%d.p%d.a%d;" % c for c in classes) + "|" + gpu
    lines.append('{"key": "%s", "value": "64 512 %s"}' % (tile, own))
    cache = tmp_path / "tune.jsonl"
    cache.write_text("\n".join(lines) + "\n")
    monkeypatch.setenv("STENCIL_TUNE_CACHE", str(cache))
    plans, xs, ys, refs_in = _batch_plans(binding, torch, SPECS)
    binding.run_batched(plans, xs, ys, [t for _, _, t in refs_in])
    plans[0].sync()
    for p, (shape, kind, r, T, seed) in zip(plans, SPECS):
        assert (p.get("last_m"), p.get("last_b")) == ((3, 2) if kind == "star" else (2, 2))
        assert p.get("last_tile_y") == 64 and p.get("last_threads") == 512
    for y, (x, c, T) in zip(ys, refs_in):
        assert oracle.rel_l2(y.cpu().numpy(), oracle.run(x.astype(np.float64), c, T)) <= 1e-5
    for p in plans:
        p.close()


def test_batched_new_composition_ignores_other_class_entries(env, tmp_path, monkeypatch):
    """Class entries alone (written by other batches) do not seed a batch
    whose composition has no entry: with autotuning off it runs the default
    choices (stars m = 3, boxes m = 2, b = 2), not the cached b = 3."""
    torch, binding, oracle = env
    gpu = torch.cuda.get_device_name()
    lines = ['{"key": "batched|2d|r%d|pat%d|area2^%d|f32|%s", "value": "1 3"}' % (c + (gpu,))
             for c in _class_keys(SPECS)]
    cache = tmp_path / "tune.jsonl"
    cache.write_text("\n".join(lines) + "\n")
    monkeypatch.setenv("STENCIL_TUNE_CACHE", str(cache))
    plans, xs, ys, refs_in = _batch_plans(binding, torch, SPECS)
    for p in plans:
        p.set_option("autotune", 0)
    binding.run_batched(plans, xs, ys, [t for _, _, t in refs_in])
    plans[0].sync()
    for p, (shape, kind, r, T, seed) in zip(plans, SPECS):
        assert (p.get("last_m"), p.get("last_b")) == ((3, 2) if kind == "star" else (2, 2))
    for y, (x, c, T) in zip(ys, refs_in):
        assert oracle.rel_l2(y.cpu().numpy(), oracle.run(x.astype(np.float64), c, T)) <= 1e-5
    for p in plans:
        p.close()


@pytest.mark.parametrize("tile", [64, 96])
def test_batched_tile_pinned_by_first_plan(env, tile):
    """The first plan's tile_y option pins the batch's tile height."""
    torch, binding, oracle = env
    plans, xs, ys, refs_in = _batch_plans(binding, torch, SPECS)
    plans[0].set_option("tile_y", tile)
    binding.run_batched(plans, xs, ys, [t for _, _, t in refs_in], [3, 2, 3, 2])
    plans[0].sync()
    assert all(p.get("last_tile_y") == tile for p in plans)
    for y, (x, c, T) in zip(ys, refs_in):
        assert oracle.rel_l2(y.cpu().numpy(), oracle.run(x.astype(np.float64), c, T)) <= 1e-5
    for p in plans:
        p.close()


@pytest.mark.parametrize("fold", [None, [1, 1, 1, 1], [3, 2, 3, 2]])
def test_batched_half_size_ctas(env, fold):
    """cta_threads 256 on the first plan runs the batch as two 256-thread
    CTAs per SM (7 consumer warps each) with tiles that fit half an SM's
    shared memory; the results match the oracle as with the wide CTA."""
    torch, binding, oracle = env
    plans, xs, ys, refs_in = _batch_plans(binding, torch, SPECS)
    plans[0].set_option("cta_threads", 256)
    binding.run_batched(plans, xs, ys, [t for _, _, t in refs_in], fold)
    plans[0].sync()
    assert all(p.get("last_tile_y") <= 96 and p.get("last_threads") == 256 for p in plans)
    for y, (x, c, T) in zip(ys, refs_in):
        assert oracle.rel_l2(y.cpu().numpy(), oracle.run(x.astype(np.float64), c, T)) <= 1e-5
    for p in plans:
        p.close()


@pytest.mark.parametrize("threads", [0, 256])
@pytest.mark.parametrize("fold", [None, 1, 2, 8])
def test_batched_radius2_and_fold_clamp(env, fold, threads):
    """Radius-2 bases (stars folded up to m = 2, boxes plain) beside radius-1
    ones, with either CTA shape; a fold request above the kernel's (8) is
    lowered to the largest it has, which gives the same T steps."""
    torch, binding, oracle = env
    specs = [((220, 260), "star", 2, 31, 9400), ((130, 170), "box", 2, 17, 9401),
             ((160, 150), "star", 1, 29, 9402), ((200, 120), "box", 1, 23, 9403)]
    plans, xs, ys, refs_in = _batch_plans(binding, torch, specs)
    plans[0].set_option("cta_threads", threads)
    folds = None if fold is None else [fold] * len(specs)
    binding.run_batched(plans, xs, ys, [t for _, _, t in refs_in], folds)
    plans[0].sync()
    for y, (x, c, T) in zip(ys, refs_in):
        assert oracle.rel_l2(y.cpu().numpy(), oracle.run(x.astype(np.float64), c, T)) <= 1e-5
    if fold == 8:
        assert [p.get("last_m") for p in plans] == [2, 1, 4, 2]
    for p in plans:
        p.close()


def test_batched_dependency_wait_times_out(env):
    """The producer's wait for a previous pass's tiles is bounded: with the
    test hook that keeps every dependency unmet, it runs out (50 ms), the
    status reads TIMEOUT, the context stays usable, and the next run matches
    the oracle."""
    torch, binding, oracle = env
    plans, xs, ys, refs_in = _batch_plans(binding, torch, SPECS[:2])
    Ts = [t for _, _, t in refs_in]
    plans[0].set_option("wait_limit_ms", 50).set_option("fault_withhold_dep", 1)
    binding.run_batched(plans, xs, ys, Ts, [1, 1])
    assert plans[0].sync_status() == 5
    assert plans[0].sync_status() == 0  # the status clears once read
    plans[0].set_option("fault_withhold_dep", 0)
    binding.run_batched(plans, xs, ys, Ts, [1, 1])
    plans[0].sync()
    for y, (x, c, T) in zip(ys, refs_in):
        assert oracle.rel_l2(y.cpu().numpy(), oracle.run(x.astype(np.float64), c, T)) <= 1e-5
    for p in plans:
        p.close()
