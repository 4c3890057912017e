"""Benchmark of the folded-stencil hot path on one GB300 (or N replicas).

Headline workload: 2D 5-point star, 4096 x 4096 FP32 grid, seeded dyadic
coefficients summing to 1, values uniform in [0, 1), periodic, T = 1000
steps, advanced by temporal computation folding with temporal blocking.  One
"step" of this bench is one full stencil_run of T = 1000 time steps on that
grid.  The other workloads (1D heat, the 8192^2 box on CUDA and tensor cores,
a separable box in counterpart form, the 3D star and box, the 256-grid batch)
are reported in ``variants`` with the same fields as the headline: GStencil/s,
the roofline of their dominant kernel, the SM clocks seen while they ran, and
the relative L2 error of the timed output against the FP64 oracle.

Roofline of a pass (one kernel launch): t_roof = max(bytes / HBM bandwidth,
algorithmic flops / pipe peak), where bytes = one read and one write of the
grid, and flops = the folded stencil's own multiply-adds (2 nnz(c^(m)) - 1 per
point and sweep; in counterpart form the two folds' 2K(2R+1) multiply-adds).
``bound`` names the larger term, ``achieved`` is that term's quantity over the
measured pass time, ``frac`` = t_roof / pass time.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on a bounded sample of the same workload instead.
"""

from __future__ import annotations

import argparse
import bisect
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
    "heat1d": dict(shape=(1 << 20,), T=100, kind="heat", seed=synth.BASE_SEED + 1,
                   workload="1D 3-point heat stencil (1/4, 1/2, 1/4), 2^20 points FP32, "
                            "periodic, T=100"),
}
L2_FLUSH_BYTES = 512 << 20


def config_coeffs(seed: int, ndim: int, kind: str) -> np.ndarray:
    """The weights of a workload: 1D heat, seeded dyadic star/box, or a separable box."""
    if kind == "heat":
        return synth.heat1d_coeffs()
    if kind == "sep":
        return synth.separable_coeffs(seed, 1, 1)
    return synth.dyadic_coeffs(seed, ndim, 1, kind)


def workload_config(name: str) -> dict:
    """The `config` object of a workload: what it is, not how it was run."""
    c = CONFIGS[name]
    return {"workload": c["workload"], "grid": list(c["shape"]), "T": c["T"]}


# ---- peaks --------------------------------------------------------------------

def _peaks_file():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return None


def hbm_peak():
    d = _peaks_file()
    if d and "hbm_gbs" in d:
        return float(d["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (measured copy)"
    return 6800.0, "fallback 6.8 TB/s"


def tensor_peak():
    """Dense BF16 TFLOP/s, sustained (the kernels run inside long steps)."""
    d = _peaks_file()
    if d and "bf16_tflops_sustained" in d:
        return float(d["bf16_tflops_sustained"]), "MEASURED_PEAKS.json bf16_tflops_sustained"
    return 1700.0, "fallback 1.7 PFLOP/s sustained"


def sm_max_mhz():
    d = _peaks_file()
    try:
        return float(d.get("sm_max_mhz", 2070.0))
    except Exception:
        return 2070.0


def fp32_peak(sms: int):
    """CUDA-core FP32: SMs x 128 FMA/clk x 2 flop x the maximum SM clock."""
    return sms * 128 * 2 * sm_max_mhz() * 1e6 / 1e12, \
        "%d SMs x 128 FP32 FMA/clk x 2 flop x %.0f MHz" % (sms, sm_max_mhz())


def fp64_peak():
    """GB300's nominal dense FP64 rate (no measured figure exists on this machine)."""
    return 1.25, "nominal GB300 FP64 1.25 TFLOP/s"


# ---- clocks -----------------------------------------------------------------------

class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons while running; each
    sample is stamped with the host time it was read, so that the samples of
    any time window can be summarised."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.samples = []  # (host time, sm MHz, max MHz, reasons)
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
            parts = [p.strip() for p in line.strip().split(",")]
            if len(parts) < 9:
                continue
            try:
                sm, smax = float(parts[1]), float(parts[2])
            except ValueError:
                continue
            reasons = {nm for nm, v in zip(self.NAMES, parts[5:9]) if v.lower() == "active"}
            self.samples.append((time.time(), sm, smax, reasons))

    def stop(self):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)

    def summary(self, t0=None, t1=None):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        s = self.samples
        if t0 is not None:
            sel = [x for x in s if t0 <= x[0] <= t1]
            if not sel and s:  # a window shorter than the sampling period: nearest sample
                times = [x[0] for x in s]
                i = min(bisect.bisect_left(times, 0.5 * (t0 + t1)), len(s) - 1)
                sel = [s[i]]
            s = sel
        return {"sm_mhz": statistics.median([x[1] for x in s]) if s else None,
                "sm_max_mhz": max(x[2] for x in s) if s else None,
                "reasons": sorted(set().union(*[x[3] for x in s])) if s else [],
                "samples": len(s)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---- the CPU-baseline leg: the only part of this file that runs the oracle ----

class OracleLeg:
    """The CPU-baseline leg.

    It times the FP64 C oracle on the host cores (the ``cpu_baseline`` field
    and the reference arm), and it provides the oracle's results against which
    the accuracy of every timed GPU output is reported: the plain time loop
    for the 1D workloads, the per-Fourier-mode closed form (spectral_run)
    elsewhere.  Nothing else in this file imports the oracle.
    """

    def __init__(self):
        import oracle
        self.oracle = oracle
        self.cache = {}

    def sample(self, name: str, T_sample: int):
        """Times the oracle on the full grid of a workload for T_sample steps."""
        w = CONFIGS[name]
        c = config_coeffs(w["seed"], len(w["shape"]), w["kind"])
        x = synth.grid(w["seed"], w["shape"], np.float32).astype(np.float64)
        t0 = time.perf_counter()
        self.oracle.run(x, c, T_sample)
        dt = time.perf_counter() - t0
        return float(np.prod(w["shape"])) * T_sample / dt / 1e9, dt, self.oracle.max_threads()

    def calibrate(self, name: str, target_s: float) -> int:
        _, dt, _ = self.sample(name, 2)
        return int(max(2, min(2000, round(target_s / max(dt / 2, 1e-6)))))

    def expected(self, x: np.ndarray, c: np.ndarray, T: int) -> np.ndarray:
        """The FP64 result of T plain steps of c applied to x."""
        x64 = np.asarray(x, np.float64)
        if x.ndim == 1:
            return self.oracle.run(x64, c, T)
        return self.oracle.spectral_run(x64, c, T)

    def reference(self, key, x, c, T):
        if key not in self.cache:
            self.cache = {key: self.expected(x, c, T)}  # one workload held at a time
        return self.cache[key]


def run_reference(args):
    """The reference arm: the oracle as it stands, timed on the host cores."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    leg = OracleLeg()
    w = CONFIGS[args.config]
    # each timed step is a bounded sample of the workload: the whole grid for
    # T_sample of its T steps, sized so that warm-up and timed steps take
    # about a minute together
    T_sample = leg.calibrate(args.config, max(1.0, 60.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        leg.sample(args.config, T_sample)
    vals, secs = [], []
    cores = 1
    for _ in range(args.steps):
        v, dt, cores = leg.sample(args.config, T_sample)
        vals.append(v)
        secs.append(dt)
    npts = float(np.prod(w["shape"]))
    value = npts * T_sample * args.steps / sum(secs) / 1e9
    sample = ("full %s grid, %d of the workload's %d steps per timed step "
              "(FP64 C oracle, OpenMP)" % ("x".join(map(str, w["shape"])), T_sample, w["T"]))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(args.config),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---- timing and rooflines -------------------------------------------------------

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


def full_passes(T: int, m: int, b: int) -> int:
    """Passes of b folded sweeps that a run of T steps makes in full."""
    return (T // m) // b


def sweep_flops(npts, R, nnz, cp_k):
    """Algorithmic flops of one sweep: the folded stencil's multiply-adds, or
    in counterpart form K vertical and K horizontal folds of 2R+1 taps."""
    if cp_k:
        return npts * 2.0 * (2 * cp_k * (2 * R + 1))
    return npts * (2.0 * nnz - 1)


def pass_roofline(npts, m, b, R, nnz, cp_k, esz, pass_ms, engine, sms):
    """Roofline of one pass of b fused sweeps of the m-folded stencil."""
    return roofline_of(2.0 * esz * npts, b * sweep_flops(npts, R, nnz, cp_k), pass_ms, esz,
                       engine, sms)


def roofline_of(alg_bytes, alg_flops, pass_ms, esz, engine, sms):
    """t_roof = max(bytes / HBM, flops / pipe peak) against a measured time."""
    hbm, hbm_src = hbm_peak()
    if engine == "tensor-core":
        pk, pk_src, pipe = (*tensor_peak(), "tensor")
    elif esz == 8:
        pk, pk_src, pipe = (*fp64_peak(), "alu")
    else:
        pk, pk_src, pipe = (*fp32_peak(sms), "alu")
    t_bytes = alg_bytes / (hbm * 1e9)
    t_flops = alg_flops / (pk * 1e12)
    s = pass_ms * 1e-3
    if t_bytes >= t_flops:
        out = {"bound": "hbm", "achieved": alg_bytes / s / 1e9, "peak": hbm, "unit": "GB/s",
               "peak_source": hbm_src}
    else:
        out = {"bound": pipe, "achieved": alg_flops / s / 1e12, "peak": pk, "unit": "TFLOP/s",
               "peak_source": pk_src}
    out["frac"] = max(t_bytes, t_flops) / s
    out.update({"pass_ms": pass_ms, "alg_bytes_per_launch": alg_bytes,
                "alg_flops_per_launch": alg_flops,
                "hbm_view": {"achieved_gbs": alg_bytes / s / 1e9, "peak_gbs": hbm,
                             "frac": t_bytes / s},
                "flops_view": {"achieved_tflops": alg_flops / s / 1e12, "peak_tflops": pk,
                               "frac": t_flops / s}})
    return out


def kernel_name(engine, grouped, ndim, b, cp_k, esz=4, persistent=0, tessellated=0):
    if engine == "tensor-core":
        if ndim == 3:  # one launch per plane offset, then the re-import of the result
            return "k_tc2d per plane offset + k_import"
        return "k_tc2d_grouped" if grouped else "k_tc2d"
    if esz == 8 and ndim >= 2:
        return "k_sweep_f64"
    if ndim == 1:
        return "k_tess_tri + k_tess_inv" if tessellated else "k_sweep1d"
    if ndim == 3:
        return "k_sweep3d_tb" if b == 2 else ("k_sweep3d_q" if persistent else "k_sweep3d")
    return "k_sweep2d"


def plan_facts(plan, ndim):
    engine = "tensor-core" if plan.get("last_engine") == 1 else "cuda-core"
    f = {"m": plan.get("last_m"), "b": plan.get("last_b"), "engine": engine}
    if ndim == 2 and engine == "cuda-core":
        f["tile_y"] = plan.get("last_tile_y")
        f["counterparts"] = plan.get("last_cp")
        f["cta_threads"] = plan.get("last_threads")
        f["stages"] = plan.get("last_stages")
    if engine == "tensor-core":
        f["tc_kernel"] = "grouped" if plan.get("last_tc_form") == 2 else "per-offset"
    if ndim == 3 and engine == "cuda-core":
        f["persistent"] = plan.get("last_persistent")
    if ndim == 1:
        f["tile_1d"] = plan.get("last_tile_y")
        f["tessellated"] = plan.get("last_tess")
    return f


def measure_run(torch, binding, stream, flush, plan, x, y, T, m, npts, esz, sms, reps=3):
    """Times whole runs of T steps and derives the duration of one pass.

    The pass time is the difference of two event-timed runs on the same
    stream: the full T, which makes n full passes, and T' with one full pass
    and the same partial pass and plain remainder, so that
    t(T) - t(T') = (n - 1) passes.  Both runs use the same fold request, so
    an autotuned run keeps its tuned configuration.
    """
    ms_full = _time_runs(torch, stream, flush, lambda: plan.run(x, y, T, fold_m=m, stream=stream),
                         reps=reps)
    plan.sync(stream)
    f = plan_facts(plan, x.dim())
    mu, bu = max(1, f["m"]), max(1, f["b"])
    n = full_passes(T, mu, bu)
    R = mu * plan.radius
    nnz = int(np.count_nonzero(plan.folded_coeffs(mu)))
    cp_k = f.get("counterparts", 0)
    if n >= 2:
        T2 = T - (n - 1) * mu * bu
        ms2 = _time_runs(torch, stream, flush,
                         lambda: plan.run(x, y, T2, fold_m=m, stream=stream), reps=reps)
        pass_ms = max(1e-6, (ms_full - ms2) / (n - 1))
        roof = pass_roofline(npts, mu, bu, R, nnz, cp_k, esz, pass_ms, f["engine"], sms)
    else:
        # fewer than two full passes: the whole run is the unit (its partial
        # folded pass and plain remainder pass, import and export included)
        q, rem = divmod(T, mu)
        npass = -(-q // bu) + (1 if rem else 0)
        nnz1 = int(np.count_nonzero(plan.folded_coeffs(1)))
        flops = q * sweep_flops(npts, R, nnz, cp_k) + rem * (2.0 * nnz1 - 1) * npts
        roof = roofline_of(npass * 2.0 * esz * npts, flops, ms_full, esz, f["engine"], sms)
        roof["unit_of_work"] = "whole run (%d passes)" % npass
    # leave y holding the full run's output for the accuracy check
    plan.run(x, y, T, fold_m=m, stream=stream)
    plan.sync(stream)
    roof["kernel"] = kernel_name(f["engine"], f.get("tc_kernel") == "grouped", x.dim(), bu, cp_k,
                                 esz, f.get("persistent", 0), f.get("tessellated", 0))
    return ms_full, f, roof


def accuracy(torch, binding, stream, y, ref_host, dev):
    ref_d = torch.from_numpy(np.ascontiguousarray(ref_host)).to(dev)
    e, ez = binding.rel_l2(y, ref_d, stream=stream)
    del ref_d
    return {"rel_l2": e, "rel_l2_zero_mean": ez}


# Variants: (name, workload, fold_m, options).  fold_m = 0 lets the library's
# autotuner choose; the options pin what the name says.
VARIANTS = [
    ("star4096_T1000_plain_fp32", "star4096", 1, {"block_b": 1}, "f32"),
    ("star4096_T1000_tc_bf16x3_m4", "star4096", 4, {"precision": 1}, "f32"),
    ("heat1d_2pow20_T100_fp32", "heat1d", 1, {}, "f32"),
    ("heat1d_2pow20_T100_fp64", "heat1d", 1, {}, "f64"),
    ("heat1d_2pow20_T100_fp32_autotuned", "heat1d", 0, {}, "f32"),
    ("heat1d_2pow20_T100_fp64_autotuned", "heat1d", 0, {}, "f64"),
    ("heat1d_2pow20_T100_fp64_m16_overlapped", "heat1d", 16, {"block_b": 32, "tessellate": 0},
     "f64"),
    ("heat1d_2pow20_T100_fp64_m16_tessellated", "heat1d", 16, {"block_b": 32, "tessellate": 1},
     "f64"),
    ("heat1d_2pow20_T100_fp32_m6_tessellated", "heat1d", 6, {"block_b": 64, "tessellate": 1},
     "f32"),
    ("box8192_T512_plain_fp32", "box8192", 1, {"block_b": 1}, "f32"),
    ("box8192_T512_cuda_core_m2b2", "box8192", 2, {"block_b": 2}, "f32"),
    ("box8192_T512_cuda_core_autotuned", "box8192", 0, {}, "f32"),
    ("box8192_T512_tc_bf16x3_m4", "box8192", 4, {"precision": 1}, "f32"),
    ("box8192_T512_tc_bf16x1_m4", "box8192", 4, {"precision": 2}, "f32"),
    ("box8192_T512_tc_tf32x3_m4", "box8192", 4, {"precision": 3}, "f32"),
    ("box8192_T512_tc_bf16x3_m6", "box8192", 6, {"precision": 1}, "f32"),
    ("box8192_T512_tc_bf16x3_m8", "box8192", 8, {"precision": 1}, "f32"),
    ("box8192_T512_tc_bf16x1_m8", "box8192", 8, {"precision": 2}, "f32"),
    ("box8192_T512_tc_bf16x3_m8_per_offset", "box8192", 8, {"precision": 1, "tc_form": 1}, "f32"),
    ("sepbox8192_T512_autotuned", "sepbox8192", 0, {}, "f32"),
    ("sepbox8192_T512_counterparts_m8b1", "sepbox8192", 8, {"block_b": 1}, "f32"),
    ("sepbox8192_T512_direct_autotuned", "sepbox8192", 0, {"counterparts": 2}, "f32"),
    ("star512cube_T200_plain", "star512cube", 1, {"block_b": 1}, "f32"),
    ("star512cube_T200_plain_fused2", "star512cube", 1, {"block_b": 2}, "f32"),
    ("star512cube_T200_m2", "star512cube", 2, {"block_b": 1}, "f32"),
    ("box256cube_T200_plain", "box256cube", 1, {"block_b": 1}, "f32"),
    ("box256cube_T200_m2", "box256cube", 2, {"block_b": 1}, "f32"),
    ("box256cube_T200_tc_bf16x3_m2", "box256cube", 2, {"precision": 1}, "f32"),
    ("box256cube_T200_tc_bf16x1_m2", "box256cube", 2, {"precision": 2}, "f32"),
    ("star4096_T1000_fp64_m4", "star4096", 4, {}, "f64"),
]


def measure_variants(torch, binding, dev, stream, flush, sampler, leg, sms, only=None):
    """Every other configuration, each timed, rooflined, clocked and checked."""
    out = {}
    for name, wname, m, opts, dtype in VARIANTS:
        if only and name not in only:
            continue
        w = CONFIGS[wname]
        shape, T = w["shape"], w["T"]
        c = config_coeffs(w["seed"], len(shape), w["kind"])
        npdt = np.float64 if dtype == "f64" else np.float32
        x_host = synth.grid(w["seed"], shape, npdt)
        x = torch.from_numpy(x_host).to(dev)
        y = torch.empty_like(x)
        plan = binding.Plan(shape, c, dtype=dtype)
        for k, v in opts.items():
            plan.set_option(k, v)
        t0 = time.time()
        ms, facts, roof = measure_run(torch, binding, stream, flush, plan, x, y, T, m,
                                      float(np.prod(shape)), 8 if dtype == "f64" else 4, sms)
        t1 = time.time()
        rec = {"gstencil_s": float(np.prod(shape)) * T / (ms * 1e-3) / 1e9, "ms": ms}
        rec.update(facts)
        rec["roofline"] = roof
        rec["clocks"] = sampler.summary(t0, t1)
        if leg is not None:
            ref = leg.reference((wname, dtype), x_host, c, T)
            rec.update(accuracy(torch, binding, stream, y, ref, dev))
        out[name] = rec
        plan.close()
        del x, y
        torch.cuda.empty_cache()
    if not only or "batched256_T10to500" in only:
        out["batched256_T10to500"] = measure_batched(torch, binding, dev, stream, flush, sampler,
                                                     leg, sms)
    return out


def measure_batched(torch, binding, dev, stream, flush, sampler, leg, sms):
    """256 independent grids in one persistent launch."""
    grids = synth.batched_workload(synth.BASE_SEED + 6)
    plans, xs, ys, Ts, host = [], [], [], [], []
    for g in grids:
        c = synth.dyadic_coeffs(g["coeff_seed"], 2, 1, g["kind"])
        plans.append(binding.Plan(g["shape"], c))
        xh = synth.grid(g["value_seed"], g["shape"], np.float32)
        host.append((xh, c))
        xs.append(torch.from_numpy(xh).to(dev))
        ys.append(torch.empty_like(xs[-1]))
        Ts.append(g["T"])
    t0 = time.time()
    ms = _time_runs(torch, stream, flush,
                    lambda: binding.run_batched(plans, xs, ys, Ts, stream=stream))
    t1 = time.time()
    plans[0].sync(stream)
    upd = sum(float(np.prod(g["shape"])) * g["T"] for g in grids)
    # roofline of the one launch: the algorithmic bytes and flops of every
    # grid's passes, summed; the launch is bound by the larger total
    hbm, hbm_src = hbm_peak()
    pk, pk_src = fp32_peak(sms)
    tot_bytes = tot_flops = 0.0
    ms_used = {}
    for p, g, T in zip(plans, grids, Ts):
        m, b = max(1, p.get("last_m")), max(1, p.get("last_b"))
        ms_used[(m, b)] = ms_used.get((m, b), 0) + 1
        npts = float(np.prod(g["shape"]))
        q, rem = divmod(T, m)
        nnz_m = int(np.count_nonzero(p.folded_coeffs(m)))
        nnz_1 = int(np.count_nonzero(p.folded_coeffs(1)))
        npass = -(-q // b) + (1 if rem else 0)
        tot_bytes += npass * 8.0 * npts
        tot_flops += npts * (q * (2.0 * nnz_m - 1) + rem * (2.0 * nnz_1 - 1))
    s = ms * 1e-3
    tb, tf = tot_bytes / (hbm * 1e9), tot_flops / (pk * 1e12)
    roof = ({"bound": "hbm", "achieved": tot_bytes / s / 1e9, "peak": hbm, "unit": "GB/s",
             "peak_source": hbm_src} if tb >= tf else
            {"bound": "alu", "achieved": tot_flops / s / 1e12, "peak": pk, "unit": "TFLOP/s",
             "peak_source": pk_src})
    roof.update({"frac": max(tb, tf) / s, "kernel": "k_batched", "launch_ms": ms,
                 "alg_bytes_per_launch": tot_bytes, "alg_flops_per_launch": tot_flops})
    rec = {"gstencil_s": upd / s / 1e9, "ms": ms, "grids": len(grids), "updates": upd,
           "m_b_counts": {"m%d_b%d" % k: v for k, v in sorted(ms_used.items())},
           "roofline": roof, "clocks": sampler.summary(t0, t1)}
    if leg is not None:
        worst = worst_zm = 0.0
        for (xh, c), y, T in zip(host, ys, Ts):
            acc = accuracy(torch, binding, stream, y, leg.expected(xh, c, T), dev)
            worst = max(worst, acc["rel_l2"])
            worst_zm = max(worst_zm, acc["rel_l2_zero_mean"])
        rec["rel_l2_max_over_grids"] = worst
        rec["rel_l2_zero_mean_max_over_grids"] = worst_zm
    for p in plans:
        p.close()
    del xs, ys
    torch.cuda.empty_cache()
    return rec


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
    sms = torch.cuda.get_device_properties(dev).multi_processor_count

    w = CONFIGS[args.config]
    SHAPE, T_STEPS = w["shape"], w["T"]
    dtype = "f32"
    c = config_coeffs(w["seed"], len(SHAPE), w["kind"])
    x_host = synth.grid(w["seed"], SHAPE, np.float32)
    npts = float(np.prod(SHAPE))
    stream = torch.cuda.current_stream(dev)

    plan = binding.Plan(SHAPE, c, dtype)
    plan.set_option("block_b", args.block_b).set_option("precision", args.precision)
    if len(SHAPE) == 2:
        plan.set_option("tc_form", args.tc_form)
    if args.tile_y:
        plan.set_option("tile_y", args.tile_y)
    if args.cta_threads:
        plan.set_option("cta_threads", args.cta_threads)
    if args.stages:
        plan.set_option("stages", args.stages)
    m_req = args.fold_m

    xd = torch.from_numpy(x_host).to(dev)
    yd = torch.empty_like(xd)
    flush = torch.empty((64 if args.ncu else L2_FLUSH_BYTES) // 4, dtype=torch.float32, device=dev)

    def timed_steps(T, k, wu):
        for _ in range(wu):
            plan.run(xd, yd, T, fold_m=m_req, stream=stream)
        plan.sync(stream)
        times = []
        launches0 = plan.get("launches")
        for _ in range(k):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.run(xd, yd, T, fold_m=m_req, stream=stream)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        plan.sync(stream)
        return times, plan.get("launches") - launches0

    sampler = ClockSampler(local)
    sampler.start()

    # --- main timed region: whole job, inputs resident on the device
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    t_a = time.time()
    times, launches = timed_steps(T_STEPS, args.steps, args.warmup)
    torch.cuda.synchronize()
    t_b = time.time()
    if pg:
        pg.barrier()
    ms_step = statistics.mean(times)
    ms_total = max_over_ranks(torch, sum(times), pg, dev)
    value = whole_job_rate(ws, npts, T_STEPS, args.steps, ms_total)
    facts = plan_facts(plan, len(SHAPE))
    if args.ncu:
        # profiling run: only the timed loop above, nothing else
        sampler.stop()
        if rank == 0:
            print(json.dumps({"ncu_run": True, "value": value, "fold_m": facts["m"],
                              "block_b": facts["b"]}))
        plan.close()
        return
    clocks = sampler.summary(t_a, t_b)
    y_timed = yd.clone()  # the output of the timed runs, checked below

    # --- dominant kernel: one pass, by difference of two event-timed runs
    mu, bu = max(1, facts["m"]), max(1, facts["b"])
    n = full_passes(T_STEPS, mu, bu)
    pass_ms = statistics.median(times) / max(1, n)
    if n >= 2:
        T2 = T_STEPS - (n - 1) * mu * bu
        t_two, _ = timed_steps(T2, 5, 2)
        pass_ms = max(1e-6, (statistics.median(times) - statistics.median(t_two)) / (n - 1))
    cp_k = facts.get("counterparts", 0)
    nnz = int(np.count_nonzero(plan.folded_coeffs(mu)))
    roof = pass_roofline(npts, mu, bu, mu * plan.radius, nnz, cp_k, 4, pass_ms,
                         facts["engine"], sms)
    roof["kernel"] = kernel_name(facts["engine"], facts.get("tc_kernel") == "grouped",
                                 len(SHAPE), bu, cp_k, 4, facts.get("persistent", 0))
    roof["traffic"] = None
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tfile):
        try:
            with open(tfile) as f:
                tr = json.load(f)
            key = "%s_%s_m%d_b%d" % (args.config, facts["engine"] +
                                     ("-grouped" if facts.get("tc_kernel") == "grouped" else "") +
                                     ("-persistent" if facts.get("persistent") else ""),
                                     mu, bu)
            roof["traffic"] = tr.get(key)
        except Exception:
            pass

    # --- end to end through the C ABI with host buffers (copies inside the timed region)
    xh = torch.from_numpy(x_host).pin_memory().numpy()
    yh = torch.empty(SHAPE, dtype=torch.float32).pin_memory().numpy()
    for _ in range(max(1, args.warmup)):
        plan.run(xh, yh, T_STEPS, fold_m=m_req, stream=stream)
    e_times = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.run(xh, yh, T_STEPS, fold_m=m_req, stream=stream)  # returns after the D2H copy
        e1.record(stream)
        e1.synchronize()
        e_times.append(e0.elapsed_time(e1))
    e2e_total = max_over_ranks(torch, sum(e_times), pg, dev)
    e2e = whole_job_rate(ws, npts, T_STEPS, args.steps, e2e_total)

    # --- the CPU-baseline leg (rank 0): the oracle timed on the host cores,
    # and the oracle's results the timed outputs are checked against
    leg = None
    cpu = None
    acc = None
    if rank == 0 and not args.no_cpu_baseline:
        leg = OracleLeg()
        Ts = leg.calibrate(args.config, args.cpu_seconds)
        v, dt, cores = leg.sample(args.config, Ts)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "full %s grid, %d steps (%.1f s), FP64 C oracle" % (
                   "x".join(map(str, SHAPE)), Ts, dt)}
        acc = accuracy(torch, binding, stream, y_timed,
                       leg.reference((args.config, dtype), x_host, c, T_STEPS), dev)

    # --- the other configurations of the workload family, each timed the same
    # way; reported beside the headline, not folded into it
    variants = {}
    if not args.no_variants:
        only = [v for v in args.variants.split(",") if v] or None
        variants = measure_variants(torch, binding, dev, stream, flush, sampler, leg, sms, only)
    sampler.stop()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(args.config),
            "run": {"fold_m": facts["m"], "block_b": facts["b"],
                    "tile_y": facts.get("tile_y"), "cta_threads": facts.get("cta_threads"),
                    "stages": facts.get("stages"), "engine": facts["engine"],
                    "counterparts": facts.get("counterparts", 0),
                    "tc_kernel": facts.get("tc_kernel"),
                    "precision": ["fp32", "bf16x3", "bf16x1", "tf32x3"][args.precision],
                    "chosen_by": "autotuner" if args.fold_m == 0 else "command line",
                    "parallelism": "replicas" if ws > 1 else "single"},
            "l2": "flushed between timed steps (512 MB write)",
            "accuracy": acc,
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": int(npts * 4),
                    "d2h_bytes_per_step": int(npts * 4)},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "sm_count": sms,
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
    ap.add_argument("--cta-threads", type=int, default=0, choices=[0, 256],
                    help="2D CUDA-core sweeps: 256 = two half-size CTAs per SM (0 = automatic)")
    ap.add_argument("--stages", type=int, default=0,
                    help="2D CUDA-core sweeps: TMA stages per CTA (0 = automatic)")
    ap.add_argument("--tc-form", type=int, default=0, choices=[0, 1, 2],
                    help="tensor-core kernel: 0 by folded radius, 1 per row offset, 2 grouped")
    ap.add_argument("--precision", type=int, default=0, choices=[0, 1, 2, 3],
                    help="0 = FP32 CUDA cores, 1 = BF16x3 tensor cores, 2 = BF16x1, 3 = TF32x3")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the CPU-baseline leg (and with it the accuracy checks)")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--variants", default="",
                    help="comma-separated variant names to time (default: all)")
    ap.add_argument("--ncu", action="store_true",
                    help="profiling run: timed loop only, no L2 flush buffer, no extra legs")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
