"""Benchmark of the folded-stencil hot path on one GB300 (or N replicas).

Workload: 2D 5-point star, 4096 x 4096 FP32 grid, seeded dyadic coefficients
summing to 1, values uniform in [0, 1), periodic, T = 1000 steps, advanced by
temporal computation folding with temporal blocking.  One "step" of this
bench is one full stencil_run of T = 1000 time steps on that grid.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on a bounded sample of the same workload instead.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2103_09235_gb300 import synth  # noqa: E402

METRIC = "GStencil/s and % HBM roofline, folded TC vs plain FP32 at rel-L2 <= 1e-5"
UNIT = "GStencil/s"
# Workloads: the default is the 2D 5-point star; "box8192" is the 2D 9-point
# box the tensor-core contraction targets.
CONFIGS = {
    "star4096": dict(shape=(4096, 4096), T=1000, kind="star", seed=synth.BASE_SEED + 2,
                     workload="2D 5-point star 4096x4096 FP32, periodic, T=1000, "
                              "dyadic coefficients (seeded)"),
    "box8192": dict(shape=(8192, 8192), T=512, kind="box", seed=synth.BASE_SEED + 3,
                    workload="2D 9-point box 8192x8192 FP32, periodic, T=512, "
                             "dyadic coefficients (seeded)"),
    "star512cube": dict(shape=(512, 512, 512), T=200, kind="star", seed=synth.BASE_SEED + 4,
                        workload="3D 7-point star 512^3 FP32, periodic, T=200, "
                                 "dyadic coefficients (seeded)"),
    "box256cube": dict(shape=(256, 256, 256), T=200, kind="box", seed=synth.BASE_SEED + 5,
                       workload="3D 27-point box 256^3 FP32, periodic, T=200, "
                                "dyadic coefficients (seeded)"),
    "sepbox8192": dict(shape=(8192, 8192), T=512, kind="sep", seed=synth.BASE_SEED + 7,
                       workload="2D 9-point separable box 8192x8192 FP32, periodic, T=512, "
                                "outer product of seeded dyadic 1D weights"),
}


def config_coeffs(seed: int, ndim: int, kind: str) -> np.ndarray:
    """The weights of a configuration: seeded dyadic star/box, or a separable box."""
    if kind == "sep":
        return synth.separable_coeffs(seed, 1, 1)
    return synth.dyadic_coeffs(seed, ndim, 1, kind)
SHAPE = CONFIGS["star4096"]["shape"]
T_STEPS = CONFIGS["star4096"]["T"]
KIND = CONFIGS["star4096"]["kind"]
SEED = CONFIGS["star4096"]["seed"]
WORKLOAD = CONFIGS["star4096"]["workload"]


def select_config(name: str):
    global SHAPE, T_STEPS, KIND, SEED, WORKLOAD
    c = CONFIGS[name]
    SHAPE, T_STEPS, KIND, SEED, WORKLOAD = c["shape"], c["T"], c["kind"], c["seed"], c["workload"]
L2_FLUSH_BYTES = 512 << 20


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def load_tensor_peak():
    """Dense BF16 TFLOP/s measured with cuBLAS over seconds (MEASURED_PEAKS.json)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops_sustained"])
    except Exception:
        return 1700.0


def fp32_peak_tflops():
    """CUDA-core FP32 peak: 152 SMs x 128 FMA/clk x 2 flop x the measured max SM clock."""
    mhz = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    except Exception:
        pass
    return 152 * 128 * 2 * mhz * 1e6 / 1e12


class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def oracle_sample(T_sample: int, shape=None):
    """Times the FP64 oracle on a bounded sample: the full grid, T_sample steps."""
    import oracle
    shape = SHAPE if shape is None else shape
    c = config_coeffs(SEED, len(shape), KIND)
    x = synth.grid(SEED, shape, np.float32).astype(np.float64)
    t0 = time.perf_counter()
    oracle.run(x, c, T_sample)
    dt = time.perf_counter() - t0
    return float(np.prod(shape)) * T_sample / dt / 1e9, dt, oracle.max_threads()


def calibrate_oracle_steps(target_s: float) -> int:
    _, dt, _ = oracle_sample(2)
    return int(max(2, min(2000, round(target_s / max(dt / 2, 1e-6)))))


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    T_sample = calibrate_oracle_steps(max(1.0, 60.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample(T_sample)
    vals, secs = [], []
    cores = 1
    for _ in range(args.steps):
        v, dt, cores = oracle_sample(T_sample)
        vals.append(v)
        secs.append(dt)
    value = statistics.median(vals)
    ms = 1e3 * float(np.prod(SHAPE)) * T_STEPS / (value * 1e9)
    sample = "full %s grid, %d of the %d steps per timed step (FP64 C oracle, OpenMP)" % (
        "x".join(map(str, SHAPE)), T_sample, T_STEPS)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": list(SHAPE), "T": T_STEPS},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _time_runs(torch, stream, flush, fn, reps=3, warm=1):
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def measure_variants(torch, binding, dev, stream, flush, args):
    """GStencil/s of the plain baseline and the other configurations."""
    out = {}

    def single(name, shape, kind, seed, T, m, ndim=2, dtype="f32", **opts):
        if kind == "heat":
            c = synth.heat1d_coeffs()
        elif kind == "sep":  # a separable 9-point box (one counterpart at every m)
            c = synth.separable_coeffs(seed, 1, 1)
        else:
            c = synth.dyadic_coeffs(seed, ndim, 1, kind)
        npdt = np.float64 if dtype == "f64" else np.float32
        x = torch.from_numpy(synth.grid(seed, shape, npdt)).to(dev)
        y = torch.empty_like(x)
        plan = binding.Plan(shape, c, dtype=dtype)
        for k, v in opts.items():
            plan.set_option(k, v)
        ms = _time_runs(torch, stream, flush, lambda: plan.run(x, y, T, fold_m=m, stream=stream))
        plan.sync(stream)
        out[name] = {"gstencil_s": float(np.prod(shape)) * T / (ms * 1e-3) / 1e9, "ms": ms,
                     "m": plan.get("last_m"), "b": plan.get("last_b"),
                     "tile_y": plan.get("last_tile_y") if ndim == 2 else None,
                     "engine": "tensor-core" if plan.get("last_engine") else "cuda-core"}
        if plan.get("last_engine"):
            out[name]["tc_kernel"] = "grouped" if plan.get("last_tc_form") == 2 else "per-offset"
        elif ndim == 2:
            out[name]["counterparts"] = plan.get("last_cp")
        plan.close()
        del x, y
        torch.cuda.empty_cache()

    s1 = synth.BASE_SEED + 1
    single("heat1d_2pow20_T100_fp32", (1 << 20,), "heat", s1, 100, 1, ndim=1)
    single("heat1d_2pow20_T100_fp64", (1 << 20,), "heat", s1, 100, 1, ndim=1, dtype="f64")
    single("heat1d_2pow20_T100_fp32_autotuned", (1 << 20,), "heat", s1, 100, 0, ndim=1)
    single("heat1d_2pow20_T100_fp64_autotuned", (1 << 20,), "heat", s1, 100, 0, ndim=1,
           dtype="f64")
    s2 = synth.BASE_SEED + 2
    single("star4096_T1000_plain_fp32", (4096, 4096), "star", s2, 1000, 1, block_b=1)
    single("star4096_T1000_tc_bf16x3_m4", (4096, 4096), "star", s2, 1000, 4, precision=1)
    s3 = synth.BASE_SEED + 3
    single("box8192_T512_plain_fp32", (8192, 8192), "box", s3, 512, 1, block_b=1)
    single("box8192_T512_cuda_core_m2b2", (8192, 8192), "box", s3, 512, 2, block_b=2)
    single("box8192_T512_cuda_core_autotuned", (8192, 8192), "box", s3, 512, 0)
    single("box8192_T512_tc_bf16x3_m4", (8192, 8192), "box", s3, 512, 4, precision=1)
    single("box8192_T512_tc_bf16x3_m6", (8192, 8192), "box", s3, 512, 6, precision=1)
    single("box8192_T512_tc_bf16x3_m8", (8192, 8192), "box", s3, 512, 8, precision=1)
    single("box8192_T512_tc_bf16x3_m8_per_offset", (8192, 8192), "box", s3, 512, 8, precision=1,
           tc_form=1)
    # a separable box (the paper's Gaussian-blur family): counterpart form
    # (Section 3.3) against the direct form, same grid and steps
    s7 = synth.BASE_SEED + 7
    single("sepbox8192_T512_autotuned", (8192, 8192), "sep", s7, 512, 0)
    single("sepbox8192_T512_counterparts_m8b1", (8192, 8192), "sep", s7, 512, 8, block_b=1)
    single("sepbox8192_T512_direct_autotuned", (8192, 8192), "sep", s7, 512, 0, counterparts=2)
    single("star512cube_T200_plain", (512, 512, 512), "star", synth.BASE_SEED + 4, 200, 1, ndim=3)
    single("star512cube_T200_plain_fused2", (512, 512, 512), "star", synth.BASE_SEED + 4, 200, 1,
           ndim=3, block_b=2)
    single("star512cube_T200_m2", (512, 512, 512), "star", synth.BASE_SEED + 4, 200, 2, ndim=3)
    single("box256cube_T200_plain", (256, 256, 256), "box", synth.BASE_SEED + 5, 200, 1, ndim=3)
    single("box256cube_T200_m2", (256, 256, 256), "box", synth.BASE_SEED + 5, 200, 2, ndim=3)
    # 256 independent grids in one persistent launch
    grids = synth.batched_workload(synth.BASE_SEED + 6)
    plans, xs, ys, Ts = [], [], [], []
    for g in grids:
        c = synth.dyadic_coeffs(g["coeff_seed"], 2, 1, g["kind"])
        plans.append(binding.Plan(g["shape"], c))
        xs.append(torch.from_numpy(synth.grid(g["value_seed"], g["shape"], np.float32)).to(dev))
        ys.append(torch.empty_like(xs[-1]))
        Ts.append(g["T"])
    ms = _time_runs(torch, stream, flush,
                    lambda: binding.run_batched(plans, xs, ys, Ts, stream=stream))
    plans[0].sync(stream)
    upd = sum(float(np.prod(g["shape"])) * g["T"] for g in grids)
    out["batched256_T10to500"] = {"gstencil_s": upd / (ms * 1e-3) / 1e9, "ms": ms,
                                  "grids": len(grids), "updates": upd}
    for p in plans:
        p.close()
    del xs, ys
    torch.cuda.empty_cache()
    return out


def max_over_ranks(torch, value: float, pg, device) -> float:
    """The largest of every rank's value (the whole job ends with its slowest
    rank); the value itself on one rank."""
    if pg is None:
        return value
    t = torch.tensor([value], device=device, dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(ws: int, npts: float, T: int, steps: int, ms_total: float) -> float:
    """GStencil/s of the whole job: every rank advances its own copy of the
    workload (replicas), so the job updates ws * npts * T points per step."""
    return ws * npts * T * steps / (ms_total * 1e-3) / 1e9


def run_gpu(args):
    import torch
    from paper_2103_09235_gb300 import build, binding

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    build.build()

    c = config_coeffs(SEED, len(SHAPE), KIND)
    x_host = synth.grid(SEED, SHAPE, np.float32)
    npts = float(np.prod(SHAPE))
    stream = torch.cuda.current_stream(dev)

    def make_plan(m, b, precision=0):
        plan = binding.Plan(SHAPE, c)
        plan.set_option("block_b", b).set_option("precision", precision)
        plan.set_option("tc_form", args.tc_form)
        if args.tile_y:
            plan.set_option("tile_y", args.tile_y)
        return plan

    xd = torch.from_numpy(x_host).to(dev)
    yd = torch.empty_like(xd)
    flush = torch.empty((64 if args.ncu else L2_FLUSH_BYTES) // 4, dtype=torch.float32, device=dev)

    def timed_steps(plan, m, T, k, w):
        for _ in range(w):
            plan.run(xd, yd, T, fold_m=m, stream=stream)
        plan.sync(stream)
        times = []
        launches0 = plan.get("launches")
        for _ in range(k):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.run(xd, yd, T, fold_m=m, stream=stream)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        plan.sync(stream)
        return times, plan.get("launches") - launches0

    m_best, b_best = args.fold_m, args.block_b
    plan = make_plan(m_best, b_best, args.precision)

    # --- main timed region: whole job, inputs resident on the device
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    times, launches = timed_steps(plan, m_best, T_STEPS, args.steps, args.warmup)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if pg:
        pg.barrier()
    ms_step = statistics.mean(times)
    ms_total = max_over_ranks(torch, sum(times), pg, dev)
    value = whole_job_rate(ws, npts, T_STEPS, args.steps, ms_total)
    used_m, used_b = plan.get("last_m"), plan.get("last_b")
    engine = "tensor-core" if plan.get("last_engine") == 1 else "cuda-core"
    grouped = engine == "tensor-core" and plan.get("last_tc_form") == 2
    if args.ncu:
        # profiling run: only the timed loop above, nothing else
        if rank == 0:
            print(json.dumps({"ncu_run": True, "value": value, "fold_m": used_m, "block_b": used_b}))
        plan.close()
        return

    # --- dominant kernel: average duration of one folded pass, by difference of
    # two CUDA-event-timed runs (T = one pass vs the full T) on the same stream
    T_one = used_m * used_b
    t_one, _ = timed_steps(plan, m_best, T_one, 5, 2)
    n_pass = T_STEPS // (used_m * used_b)
    rem_steps = T_STEPS - n_pass * used_m * used_b
    pass_ms = (statistics.median(times) - statistics.median(t_one)) / max(1, n_pass - 1)
    if rem_steps:
        pass_ms = statistics.median(times) / max(1, n_pass)
    peak, peak_kind = load_peaks()
    alg_bytes = 2 * 4 * npts  # one read and one write of the grid per pass
    achieved = alg_bytes / (pass_ms * 1e-3) / 1e9
    # algorithmic flops of one pass: b sweeps of the folded stencil, each
    # 2*nnz(c^(m)) - 1 flops per point (its own multiply-adds, not the
    # redundant rim, the Toeplitz zeros or the BF16 split)
    nnz = int(np.count_nonzero(plan.folded_coeffs(used_m)))
    alg_flops = npts * used_b * (2 * nnz - 1)
    used_cp = plan.get("last_cp") if (engine == "cuda-core" and len(SHAPE) == 2) else 0
    if used_cp:
        # counterpart form: K vertical and K horizontal folds of 2mr+1 taps,
        # the algorithm's own multiply-adds in that form
        alg_flops = npts * used_b * 2 * (2 * used_cp * (2 * used_m + 1))
    tflops = alg_flops / (pass_ms * 1e-3) / 1e12
    if engine == "tensor-core":
        bound, r_ach, r_peak, r_unit = "tensor", tflops, load_tensor_peak(), "TFLOP/s"
    elif used_m == 1 and used_b == 1:
        bound, r_ach, r_peak, r_unit = "hbm", achieved, peak, "GB/s"
    else:
        bound, r_ach, r_peak, r_unit = "alu", tflops, fp32_peak_tflops(), "TFLOP/s"
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tfile):
        try:
            with open(tfile) as f:
                tr = json.load(f)
            key = "%s_%s_m%d_b%d" % (args.config, engine + ("-grouped" if grouped else ""),
                                     used_m, used_b)
            traffic = tr.get(key)
        except Exception:
            traffic = None

    # --- end to end through the C ABI with host buffers (copies inside the timed region)
    xh = torch.from_numpy(x_host).pin_memory().numpy()
    yh = torch.empty(SHAPE, dtype=torch.float32).pin_memory().numpy()
    for _ in range(max(1, args.warmup)):
        plan.run(xh, yh, T_STEPS, fold_m=m_best, stream=stream)
    e_times = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.run(xh, yh, T_STEPS, fold_m=m_best, stream=stream)  # returns after the D2H copy
        e1.record(stream)
        e1.synchronize()
        e_times.append(e0.elapsed_time(e1))
    e2e_total = max_over_ranks(torch, sum(e_times), pg, dev)
    e2e = whole_job_rate(ws, npts, T_STEPS, args.steps, e2e_total)

    # --- the other configurations of the workload family, each timed the same
    # way (events around whole runs, L2 flushed between runs); reported beside
    # the headline, not folded into it
    variants = {}
    if not args.no_variants:
        variants = measure_variants(torch, binding, dev, stream, flush, args)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        Ts = calibrate_oracle_steps(args.cpu_seconds)
        v, dt, cores = oracle_sample(Ts)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "full %s grid, %d steps (%.1f s), FP64 C oracle" % (
                   "x".join(map(str, SHAPE)), Ts, dt)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": list(SHAPE), "T": T_STEPS,
                       "fold_m": used_m, "block_b": used_b, "tile_y": plan.get("last_tile_y"),
                       "engine": engine, "counterparts": used_cp,
                       "precision": ["fp32", "bf16x3", "bf16x1"][args.precision],
                       "l2": "flushed between timed steps (512 MB write)",
                       "parallelism": "replicas" if ws > 1 else "single"},
            "roofline": {"bound": bound, "achieved": r_ach, "peak": r_peak, "unit": r_unit,
                         "frac": r_ach / r_peak, "traffic": traffic,
                         "peak_source": peak_kind if bound == "hbm" else
                         ("MEASURED_PEAKS.json bf16_tflops_sustained" if bound == "tensor" else
                          "152 SMs x 128 FP32 FMA/clk x 2 flop x measured max SM clock"),
                         "kernel": ("k_tc2d_grouped" if grouped else "k_tc2d")
                                   if engine == "tensor-core" else
                                   ("k_sweep3d" if len(SHAPE) == 3 else "k_sweep2d"),
                         "pass_ms": pass_ms, "alg_bytes_per_launch": alg_bytes,
                         "alg_flops_per_launch": alg_flops,
                         "hbm_view": {"achieved_gbs": achieved, "peak_gbs": peak,
                                      "frac": achieved / peak}},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": int(npts * 4),
                    "d2h_bytes_per_step": int(npts * 4)},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "variants": variants,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if pg:
        pg.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", default="star4096", choices=sorted(CONFIGS))
    ap.add_argument("--fold-m", type=int, default=0,
                    help="fold depth; 0 = the library's autotuner chooses m, b and the tile")
    ap.add_argument("--block-b", type=int, default=0)
    ap.add_argument("--tile-y", type=int, default=0,
                    help="rows per 2D tile (0 = the autotuner's or the library's choice)")
    ap.add_argument("--tc-form", type=int, default=0, choices=[0, 1, 2],
                    help="tensor-core kernel: 0 by folded radius, 1 per row offset, 2 grouped")
    ap.add_argument("--precision", type=int, default=0, choices=[0, 1, 2],
                    help="0 = FP32 CUDA cores, 1 = BF16x3 tensor cores, 2 = BF16x1")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--ncu", action="store_true",
                    help="profiling run: timed loop only, no L2 flush buffer, no extra legs")
    args = ap.parse_args()
    select_config(args.config)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
