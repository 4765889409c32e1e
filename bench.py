"""Benchmark of the batched unbinned-likelihood hot path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload prod3_1e8_f32|decay_1e7|decay_generic_1e7|decay_toys_4096|...]
                    [--no-extras] [--no-cpu-baseline] [--blocks-per-sm B]

Default workload (the headline: NLL + gradient over 1e8 events): events/s
of one NLL + gradient pass over the 3-observable product model
[mass: Gauss + Chebychev1] x [decay time: exp(-t/tau) (x) Gauss + Chebychev2]
x [cos theta: Poly2], 12 free parameters, 1e8 events in three FP32 columns.
One step = one pass of the whole path over the dataset: the parameter-point
kernel and the fused event/adjoint/reduction kernel.  The device-resident
value times K steps with CUDA events (inputs already in HBM, 1.2 GB of
columns, L2 flushed between steps).  The end-to-end number runs the same
step through the C ABI with host buffers: host->device copy of the event
columns from pinned memory, rf_nll_grad with host parameters,
device->host read of the NLL and gradient.  Beside it the same line
reports the FP64 interpreter on the same events (`fp64_interpreter`) and,
under `extras`, the rest of the metric measured in the same run: the decay
model at 1e7 FP64 events (events/s and its 6-parameter fit), 4096 ragged
toys fitted together (toy fits/s), and learned-start against plain-start
fits of 1e4 fresh toys after training on 1e6 (toy fits/s, evaluations,
identical minima).

Other workloads, one line each: decay_1e7; decay_generic_1e7 (the FP64
interpreter); decay_toys_4096; learned_start; gauss_poly1_1e4 (1e4 events,
latency-bound); binned_4096.

Multi-GPU (torchrun): every rank evaluates its own dataset (weak scaling, no
collective on the data path); rank 0 prints one JSON line (no extras).
--shard: strong scaling instead, one 1e8-event dataset split over the ranks
(rf_shard), each step = every rank's partial pass + one all_gather of the
(1 + 12) x 2 compensated sums + the rank-ordered exact merge.
--impl reference times the CPU oracle (single thread, the machine's host cores)
on a bounded sample of the same workload, with the same metric.
--blocks-per-sm pins the event kernel's launch shape instead of the
autotuner's winner (for profiling runs, whose timings the profiler distorts).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2003_12861_gb300 import workloads as W  # noqa: E402

METRIC = "events/s of NLL+grad eval; toy fits/s learned-start vs plain at |ΔNLL|<1e-6"

WORKLOADS = {
    # name: model constructor, generating theta, events per dataset, FP32 columns, bytes/event
    "decay_1e7": ("decay_model", W.DECAY_TRUE, 10_000_000, False, 8),
    "decay_generic_1e7": ("decay_generic_model", W.DECAY_GENERIC_TRUE, 10_000_000, False, 8),
    "prod3_1e8_f32": ("prod3_model", W.PROD3_TRUE, 100_000_000, True, 12),
    "gauss_poly1_1e4": ("gauss_poly1_model", W.GAUSS_POLY1_TRUE, 10_000, False, 8),
    "decay_toys_4096": ("decay_model", W.DECAY_TRUE, 0, False, 8),
    "learned_start": ("decay_model", W.DECAY_TRUE, 0, False, 8),
    "binned_4096": ("binned_model", None, 0, False, 8),
}
DEFAULT_STEPS = {"decay_1e7": 400, "decay_generic_1e7": 40, "prod3_1e8_f32": 20, "gauss_poly1_1e4": 2000, "decay_toys_4096": 3,
                 "learned_start": 1, "binned_4096": 100}


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu, self.proc, self.out = gpu_index, None, None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is None:
            return
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            self.out, _ = self.proc.communicate()

    def summary(self):
        if not self.out:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = [r.split(", ") for r in self.out.strip().splitlines() if r.count(",") >= 8]
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for i, n in enumerate(names):
                if r[5 + i].strip() == "Active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ------------------------------------------------------------- CPU oracle

def oracle_events_per_s(wl: str, seconds: float, n_sample: int):
    """The oracle as it stands, single-threaded, on a bounded sample of the
    workload's model (oracle-generated events, fewer of them)."""
    import oracle

    ctor, theta, _, f32, _ = WORKLOADS[wl]
    spec = W.model_for(ctor)
    om = oracle.Model(spec.nodes, spec.root)
    cols = om.generate(theta, W.SEED_BASE + 1, 0, 0, n_sample)
    if f32:
        cols = [c.astype(np.float32).astype(np.float64) for c in cols]
    reps, t0 = 0, time.perf_counter()
    while True:
        om.nll(theta, cols)
        reps += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return reps * n_sample / dt, f"{reps} oracle NLL+gradient passes over {n_sample} events of the {ctor}, {dt:.1f} s"


def oracle_events_all_cores(wl: str, seconds: float, n_per_thread: int):
    """The same oracle pass split over every host core: contiguous event
    slices, one thread each (the oracle's C entry point runs without the
    interpreter lock), per-slice NLL and gradient summed in slice order."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor

    ctor, theta, _, f32, _ = WORKLOADS[wl]
    spec = W.model_for(ctor)
    om = oracle.Model(spec.nodes, spec.root)
    T = os.cpu_count() or 1
    cols = om.generate(theta, W.SEED_BASE + 1, 0, 0, n_per_thread * T)
    if f32:
        cols = [c.astype(np.float32).astype(np.float64) for c in cols]
    slices = [[c[t * n_per_thread:(t + 1) * n_per_thread] for c in cols] for t in range(T)]
    with ThreadPoolExecutor(T) as pool:
        reps, t0 = 0, time.perf_counter()
        while True:
            parts = list(pool.map(lambda sl: om.nll(theta, sl), slices))
            nll = sum(p[0] for p in parts)
            grad = np.sum([p[1] for p in parts], axis=0)
            reps += 1
            if time.perf_counter() - t0 >= seconds:
                break
        dt = time.perf_counter() - t0
    assert np.isfinite(nll) and np.all(np.isfinite(grad))
    return (reps * n_per_thread * T / dt, T,
            f"{reps} oracle passes over {T} threads x {n_per_thread} events of the {ctor}, {dt:.1f} s")


def oracle_toy_fits_per_s(seconds: float):
    """The oracle's own fitter on the toy workload's first toys (same seeds,
    sizes and generating parameters), one at a time, single-threaded."""
    import oracle

    spec = W.decay_model()
    om = oracle.Model(spec.nodes, spec.root)
    seed = W.SEED_BASE + 2
    mean = W.toy_mean_sizes(4096, seed)
    fits, dt = 0, 0.0
    while dt < seconds and fits < 4096:
        n = oracle.poisson(seed, fits, mean[fits])
        cols = om.generate(W.DECAY_TRUE, seed, fits, 0, n)
        t1 = time.perf_counter()
        om.fit(cols, tol_edm=1e-7, cov=False)
        dt += time.perf_counter() - t1
        fits += 1
    return fits / dt, f"oracle BFGS fits (plain start) of the first {fits} toys of the 4096-toy batch, {dt:.1f} s"


def oracle_toy_fits_all_cores(seconds: float):
    """The oracle's fitter on the toy workload's toys over every host core:
    each thread takes the next toy as it finishes one (the oracle's C entry
    points run without the interpreter lock); toys started after the time
    budget are skipped."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor

    spec = W.decay_model()
    om = oracle.Model(spec.nodes, spec.root)
    seed = W.SEED_BASE + 2
    mean = W.toy_mean_sizes(4096, seed)
    T = os.cpu_count() or 1
    n_toys = min(4096, 32 * T)
    with ThreadPoolExecutor(T) as pool:
        cols = list(pool.map(lambda s: om.generate(W.DECAY_TRUE, seed, s, 0, oracle.poisson(seed, s, mean[s])),
                             range(n_toys)))
        t0 = time.perf_counter()

        def fit(s):
            if time.perf_counter() - t0 > seconds:
                return None
            return om.fit(cols[s], tol_edm=1e-7, cov=False)["status"]

        done = [r for r in pool.map(fit, range(n_toys)) if r is not None]
        dt = time.perf_counter() - t0
    return len(done) / dt, T, f"oracle BFGS fits (plain start) of {len(done)} of the first {n_toys} toys, {T} threads, {dt:.1f} s"


def oracle_binned_per_s(seconds: float):
    """The binned oracle as it stands, single-threaded, on datasets of the
    binned workload's model (same parameter points, counts drawn at them)."""
    from oracle import binned as OB

    spec = W.binned_model()
    om = OB.from_spec(spec)
    th = W.binned_toy_thetas(64, W.SEED_BASE + 5, spec["n_params"])
    rng = np.random.Generator(np.random.PCG64(W.SEED_BASE + 6))
    counts = [rng.poisson(om.expected(t)[0]).astype(float) for t in th[:4]]
    n, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        om.nll(th[n % 4], counts[n % 4])
        n += 1
    dt = time.perf_counter() - t0
    return n / dt, f"{n} oracle NLL+gradient evaluations of datasets of the binned model, {dt:.1f} s"


def cpu_baseline(wl: str):
    if wl == "binned_4096":
        v, s = oracle_binned_per_s(10.0)
        return {"value": v, "unit": "datasets/s", "cores": 1, "kind": "oracle", "sample": s}
    if wl in ("decay_toys_4096", "learned_start"):
        v, s = oracle_toy_fits_per_s(15.0)
        out = {"value": v, "unit": "toy fits/s", "cores": 1, "kind": "oracle", "sample": s}
        va, cores, sa = oracle_toy_fits_all_cores(6.0)
        out["all_cores"] = {"value": va, "unit": "toy fits/s", "cores": cores, "sample": sa}
        return out
    v, s = oracle_events_per_s(wl, 12.0, 400_000 if wl != "gauss_poly1_1e4" else 10_000)
    out = {"value": v, "unit": "events/s", "cores": 1, "kind": "oracle", "sample": s}
    if wl != "gauss_poly1_1e4":
        va, cores, sa = oracle_events_all_cores(wl, 6.0, 100_000)
        out["all_cores"] = {"value": va, "unit": "events/s", "cores": cores, "sample": sa}
    return out


def run_reference(args):
    rank, _, _ = dist_env()
    if rank != 0:
        return 0
    wl = args.workload
    t0 = time.perf_counter()
    if wl == "binned_4096":
        v, s = oracle_binned_per_s(max(3.0, 0.5 * args.steps))
        unit = "datasets/s"
    elif wl in ("decay_toys_4096", "learned_start"):
        # each step: the oracle fits one toy of the batch
        v, s = oracle_toy_fits_per_s(max(3.0, 1.5 * args.steps))
        unit = "toy fits/s"
    else:
        import oracle

        ctor, theta, _, f32, _ = WORKLOADS[wl]
        spec = W.model_for(ctor)
        om = oracle.Model(spec.nodes, spec.root)
        n_sample = 200_000 if wl != "gauss_poly1_1e4" else 10_000
        cols = om.generate(theta, W.SEED_BASE + 1, 0, 0, n_sample)
        for _ in range(args.warmup):
            om.nll(theta, cols)
        t1 = time.perf_counter()
        for _ in range(args.steps):
            om.nll(theta, cols)
        dt = time.perf_counter() - t1
        v = args.steps * n_sample / dt
        s = f"each step: one oracle NLL+gradient pass over {n_sample} events of the {ctor}"
        unit = "events/s"
    dt_all = time.perf_counter() - t0
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": unit, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dt_all / max(1, args.steps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl},
        "cpu_baseline": {"value": v, "unit": unit, "cores": 1, "kind": "oracle", "sample": s},
        "e2e": {"value": v, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------- ours

def transcendental_ceiling(api, model_spec, slow_fraction, n_events, bytes_per_event, peaks, peak_kind, ff=True,
                           n_log=1):
    """ALU ceiling: per event the method's fast set {exp per Gauss/exp/decay
    leaf, log, reciprocal}; events in the decay resolution region add {exp,
    erfc} per decay leaf; rates measured in-run by the library's probe with
    the implementations the kernel uses (float-float, or CUDA's FP64
    functions for the generic FP64 interpreter).  The log stays in the count
    although the kernels take sum log p from a running product (one log per
    lane and part): the ceiling is set by the method's work, not moved by
    the implementation measured against it.  n_log=0 gives the ceiling
    without it, reported beside."""
    kinds = [n.kind for n in model_spec.nodes]
    n_exp = sum(k in ("gauss", "exp", "gaussexp") for k in kinds)
    n_ge = sum(k == "gaussexp" for k in kinds)
    kind = 4 if ff else 2
    fast = api.probe(kind, n_exp=n_exp, n_log=n_log, n_rcp=1)
    full = api.probe(kind, n_exp=n_exp + n_ge, n_erfc=n_ge, n_log=n_log, n_rcp=1) if n_ge else fast
    t_event = 1.0 / fast + slow_fraction * (1.0 / full - 1.0 / fast)
    alu = 1.0 / t_event
    hbm = peaks["hbm_gbs"] * 1e9 / bytes_per_event
    lg = "log, " if n_log else ""
    basis = (f"transcendental set per event measured in-run ({'float-float' if ff else 'CUDA FP64'} "
             f"implementations): fast {{{n_exp} exp, {lg}rcp}} {fast/1e9:.2f} "
             f"Gevent/s, slow {{{n_exp + n_ge} exp, {n_ge} erfc, {lg}rcp}} {full/1e9:.2f} Gevent/s, slow "
             f"fraction {slow_fraction:.4f}; HBM ceiling {hbm/1e9:.0f} Gevent/s at {peaks['hbm_gbs']} GB/s "
             f"({peak_kind}) x {bytes_per_event} B/event")
    return alu, hbm, basis


KERNEL_SOURCES = ["nll.cu", "nll_ff.cuh", "k1_ff.cuh", "ff.cuh", "ff_tables.h", "nll_kernels.cuh", "rf_internal.h", "expr.cuh"]


def kernel_digest():
    """First 16 hex digits of SHA-256 over the event kernel's sources."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2003_12861_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload):
    """DRAM bytes per launch of the fused kernel from the committed ncu
    summary of this workload, or None when there is none or the kernel
    sources changed since it was taken."""
    path = os.path.join(ROOT, "profiles", f"{workload}_events_ff.md")
    if not os.path.exists(path):
        return None
    fields = {}
    with open(path) as fh:
        for line in fh:
            if ":" in line and line.split(":")[0] in ("kernel_source_digest", "dram_bytes_per_launch"):
                k, v = line.split(":", 1)
                fields[k] = v.strip()
    if fields.get("kernel_source_digest") != kernel_digest() or "dram_bytes_per_launch" not in fields:
        return None
    return int(fields["dram_bytes_per_launch"])


def roofline(api, model, spec, data, kern_ms, kern_n, n_events, bpe, peaks, peak_kind, slow_frac=None,
             workload=None):
    if slow_frac is None:
        slow_frac = api.slow_events(data) / max(1, n_events)
    ff = "kernel=ff_" in model.describe()
    alu, hbm, basis = transcendental_ceiling(api, spec, slow_frac, n_events, bpe, peaks, peak_kind, ff)
    alu0, _, _ = transcendental_ceiling(api, spec, slow_frac, n_events, bpe, peaks, peak_kind, ff, n_log=0)
    # the fixed per-event count (every event charged the resolution region's
    # full set, whether or not its region needs it)
    alu_fixed, _, _ = transcendental_ceiling(api, spec, 1.0, n_events, bpe, peaks, peak_kind, ff)
    ceiling = min(alu, hbm)
    avg = kern_ms / max(1, kern_n)
    achieved = n_events / (avg * 1e-3)
    return {
        "bound": "alu" if alu < hbm else "hbm", "achieved": achieved / 1e9, "peak": ceiling / 1e9,
        "unit": "Gevent/s", "frac": achieved / ceiling,
        "traffic": profiled_traffic(workload) if workload else None,
        "kernel": model.describe(), "kernel_avg_ms": avg, "kernel_launches": kern_n, "peak_basis": basis,
        "fp64_fma_tflops_measured": api.probe(0) / 1e12,
        "hbm_frac": achieved * bpe / (peaks["hbm_gbs"] * 1e9),
        "peak_without_log": min(alu0, hbm) / 1e9, "frac_without_log": achieved / min(alu0, hbm),
        "peak_fixed_count": min(alu_fixed, hbm) / 1e9, "frac_fixed_count": achieved / min(alu_fixed, hbm),
    }


def path_dtype(model, f32: bool) -> str:
    """What the pass computes in: the float-float event programs keep every
    per-event quantity as a pair of floats (~48 significant bits) on the FP32
    pipe and merge chunks in an FP64 two-sum tree; the generic interpreter is
    FP64 throughout."""
    cols = "f32 columns" if f32 else "f64 columns"
    if "kernel=ff_" in model.describe():
        return f"float-float (~48-bit) per event on the FP32 pipe, f64 reduction tree; {cols}"
    return f"f64 per event (FP64 interpreter), f64 reduction tree; {cols}"


def fp64_interpreter_figure(api, torch, model, spec, data, theta, out, flags, stream, flush, n, bpe, peaks,
                            peak_kind, steps=10):
    """The same model and events through the FP64 graph interpreter (every
    node in double precision, CUDA's FP64 exp/erfc/log): events/s of a
    device-resident pass and its kernel's fraction of the FP64 ceiling."""
    model.set_fp64(True)
    try:
        def step():
            api.nll_grad_async(model, data, theta, out, flags, stream=stream)

        with torch.cuda.stream(stream):
            for _ in range(3):
                step()
        stream.synchronize()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        with torch.cuda.stream(stream):
            for i in range(steps):
                flush.zero_()
                starts[i].record(stream)
                step()
                ends[i].record(stream)
        torch.cuda.synchronize()
        total_ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends))
        api.kernel_time(reset=True)
        api.kernel_timing(True)
        with torch.cuda.stream(stream):
            for _ in range(steps):
                flush.zero_()
                step()
        torch.cuda.synchronize()
        api.kernel_timing(False)
        kern_ms, kern_n = api.kernel_time(reset=True)
        rl = roofline(api, model, spec, data, kern_ms, kern_n, n, bpe, peaks, peak_kind)
        return {"value": n * steps / (total_ms * 1e-3), "unit": "events/s", "ms_per_step": total_ms / steps,
                "dtype": "f64 (every node, CUDA FP64 functions)", "nll_check": float(out[0].item()),
                "roofline": {k: rl[k] for k in ("bound", "achieved", "peak", "unit", "frac", "kernel",
                                                 "kernel_avg_ms", "peak_basis", "frac_fixed_count")}}
    finally:
        model.set_fp64(False)


def pinned_launch(model, grid, args):
    """--blocks-per-sm: that grid entry, set on the model; None otherwise."""
    if not getattr(args, "blocks_per_sm", 0):
        return None
    for g in grid:
        if g[0] == args.blocks_per_sm:
            model.set_launch(128, g[0])
            return g
    raise SystemExit(f"--blocks-per-sm {args.blocks_per_sm}: not in the scanned grid {[g[0] for g in grid]}")


def run_events(args, api, torch, dist, rank, world, local, wl=None, steps=None, fp64_figure=False, fit_figure=False):
    wl = wl or args.workload
    steps = steps or args.steps
    ctor, theta_true, n, f32, bpe = WORKLOADS[wl]
    spec = W.model_for(ctor)
    model = api.Model.from_spec(spec)
    data = api.generate_toys(model, theta_true, W.SEED_BASE + 1 + 1000 * rank, [float(n)], poisson=False,
                             f32=[f32] * spec.n_obs)
    assert data.n_events == n
    grid = api.autotune_scan(model, data, passes=3)
    best = pinned_launch(model, grid, args) or min(grid, key=lambda g: g[1])
    tune = (128, best[0], best[1])
    P = model.n_free
    stream = torch.cuda.Stream()
    theta = torch.tensor(theta_true * (1 + 0.02 * np.cos(np.arange(P))), dtype=torch.float64, device="cuda")
    out = torch.zeros(1 + P, dtype=torch.float64, device="cuda")
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > L2 (129 MB)

    def step():
        api.nll_grad_async(model, data, theta, out, flags, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    stream.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    n_launch0 = api.launch_count()
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            for i in range(steps):
                flush.zero_()
                starts[i].record(stream)
                step()
                ends[i].record(stream)
        torch.cuda.synchronize()
    n_launches = api.launch_count() - n_launch0
    if dist:
        dist.barrier()
    total_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    # The fused kernel's own duration (for the roofline), in separate steps:
    # the timing events between K1 and K2 would break their overlap above.
    api.kernel_time(reset=True)
    api.kernel_timing(True)
    with torch.cuda.stream(stream):
        for i in range(min(steps, 50)):
            flush.zero_()
            step()
    torch.cuda.synchronize()
    api.kernel_timing(False)
    kern_ms, kern_n = api.kernel_time(reset=True)
    if dist:
        t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * n * steps / (total_ms * 1e-3)

    # End to end through the C ABI with host buffers (pinned columns).
    host_cols = []
    for c in range(spec.n_obs):
        hc = torch.empty(n, dtype=torch.float32 if f32 else torch.float64, pin_memory=True)
        hc.copy_(torch.from_numpy(data.read(c).astype(np.float32 if f32 else np.float64)))
        host_cols.append(hc)
    e2e_data = api.Data.upload(model, [h.numpy() for h in host_cols], f32=[f32] * spec.n_obs)
    th_host = theta.cpu().numpy()
    for _ in range(2):
        api.nll_grad_stream(model, e2e_data, host_cols, th_host)
    k_e2e = max(3, steps // 4)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        api.nll_grad_stream(model, e2e_data, host_cols, th_host)
    e2e_s = time.perf_counter() - t0
    if dist:
        t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = {"value": world * n * k_e2e / e2e_s, "unit": "events/s", "h2d_bytes_per_step": n * bpe + P * 8,
           "d2h_bytes_per_step": (1 + P) * 8 + 4, "steps": k_e2e}
    if rank != 0:
        return None
    peaks, peak_kind = measured_peaks()
    line = {
        "value": value, "unit": "events/s", "ms_per_step": total_ms / steps,
        "dtype": path_dtype(model, f32), "config": {"workload": wl, "n_events_per_gpu": n,
                                   "columns": f"{spec.n_obs} x {'f32' if f32 else 'f64'}",
                                   "free_parameters": P, "l2": "flushed between steps (256 MiB write)",
                                   "tile": {"threads_per_block": tune[0], "blocks_per_sm": tune[1],
                                            "grid_ms_per_pass": {str(b): round(t, 4) for b, t in grid}}},
        "roofline": roofline(api, model, spec, data, kern_ms, kern_n, n, bpe, peaks, peak_kind, workload=wl),
        "e2e": e2e, "gpu_launches": int(n_launches), "clocks": clk.summary(),
        "nll_check": float(out[0].item()),
    }
    if fp64_figure:
        line["fp64_interpreter"] = fp64_interpreter_figure(api, torch, model, spec, data, theta, out, flags, stream,
                                                           flush, n, bpe, peaks, peak_kind)
    if fit_figure:
        # the configuration's 6-parameter quasi-Newton fit from the default
        # start over the resident dataset: every evaluation is one pass
        api.fit(model, data, want_cov=False, max_evals=3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = api.fit(model, data, want_cov=True)
        wall = time.perf_counter() - t0
        ne = int(r["n_evals"][0])
        line["fit"] = {"wall_ms": 1e3 * wall, "n_evals": ne, "status": int(r["status"][0]),
                       "events_per_s_in_fit": ne * n / wall, "start": "plain default start", "tol_edm": 1e-7,
                       "theta": r["theta"][0].tolist(), "nll": float(r["nll"][0]),
                       "note": "wall time of rf_fit: host BFGS + one device pass per evaluation + covariance"}
    if wl == "gauss_poly1_1e4":
        # the configuration's full fit from its stated start, end to end
        host = api.Data.upload(model, [data.read(0)])
        t0 = time.perf_counter()
        r = api.fit(model, host, want_cov=True)
        line["fit"] = {"wall_ms": 1e3 * (time.perf_counter() - t0), "n_evals": int(r["n_evals"][0]),
                       "status": int(r["status"][0]), "theta": r["theta"][0].tolist()}
        line["us_per_eval"] = 1e3 * total_ms / steps
    return line


def run_toys(args, api, torch, dist, rank, world, local, steps=None, warmup=None):
    """4096 ragged toys of the decay model, every toy drawn at its generating
    values (the configuration of the batched fit), fitted together."""
    steps = steps or args.steps
    warmup = args.warmup if warmup is None else warmup
    spec = W.decay_model()
    model = api.Model.from_spec(spec)
    S = 4096
    seed = W.SEED_BASE + 2
    mean = W.toy_mean_sizes(S, seed)
    data = api.generate_toys(model, W.DECAY_TRUE, seed + 1000 * rank, mean, poisson=True)
    n_events = data.n_events
    grid = api.autotune_scan(model, data, passes=2)
    best = pinned_launch(model, grid, args) or min(grid, key=lambda g: g[1])
    tune = (128, best[0], best[1])
    P = model.n_free
    # roofline pass: one ragged persistent launch over all toys
    stream = torch.cuda.Stream()
    theta = torch.tensor(np.tile(W.DECAY_START, S), dtype=torch.float64, device="cuda")
    out = torch.zeros(S * (1 + P), dtype=torch.float64, device="cuda")
    flags = torch.zeros(S, dtype=torch.int32, device="cuda")
    with torch.cuda.stream(stream):
        for _ in range(3):
            api.nll_grad_async(model, data, theta, out, flags, stream=stream)
        stream.synchronize()
        api.kernel_time(reset=True)
        api.kernel_timing(True)
        for _ in range(5):
            api.nll_grad_async(model, data, theta, out, flags, stream=stream)
        stream.synchronize()
        api.kernel_timing(False)
    kern_ms, kern_n = api.kernel_time(reset=True)
    slow_frac = api.slow_events(data) / n_events

    for _ in range(warmup):
        api.fit(model, data, want_cov=False)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    evals, conv = [], []
    with ClockSampler(local) as clk:
        n_launch0 = api.launch_count()
        t0 = time.perf_counter()
        for _ in range(steps):
            r = api.fit(model, data, want_cov=False)
            evals.append(r["n_evals"])
            conv.append(r["status"] == 0)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        n_launches = api.launch_count() - n_launch0
    if dist:
        t = torch.tensor([dt], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dt = float(t.item())
    value = world * S * steps / dt
    ev = np.concatenate(evals)
    # end to end: host columns uploaded, fitted, results read back
    cols = [data.read(0)]
    off = data.offsets()
    t0 = time.perf_counter()
    hd = api.Data.upload(model, cols, offsets=off)
    api.fit(model, hd, want_cov=False)
    e2e_s = time.perf_counter() - t0
    if rank != 0:
        return None
    peaks, peak_kind = measured_peaks()
    rl = roofline(api, model, spec, data, kern_ms, kern_n, n_events, 8, peaks, peak_kind, slow_frac)
    rounds = int(ev.max())
    rl["toy_fits_per_s_ceiling"] = rl["peak"] * 1e9 / (n_events * float(ev.mean())) * S
    return {
        "value": value, "unit": "toy fits/s", "ms_per_step": 1e3 * dt / steps, "dtype": "f64",
        "config": {"workload": "decay_toys_4096", "toys": S, "events": int(n_events),
                   "sizes": "Poisson(N), N log-uniform in [1e3, 1e5]", "theta": "the decay model's values for every toy",
                   "start": "plain default start",
                   "tol_edm": 1e-7, "tile": {"threads_per_block": tune[0], "blocks_per_sm": tune[1],
                                             "grid_ms_per_pass": {str(b): round(t, 4) for b, t in grid}},
                   "eval_step": "CUDA graph replay, one ragged persistent launch per round"},
        "roofline": rl,
        "e2e": {"value": world * S / e2e_s, "unit": "toy fits/s", "h2d_bytes_per_step": int(n_events) * 8,
                "d2h_bytes_per_step": S * (P + 3) * 8},
        "gpu_launches": int(n_launches),
        "clocks": clk.summary(),
        "fits": {"mean_evals": float(ev.mean()), "max_evals": int(ev.max()),
                 "converged_frac": float(np.concatenate(conv).mean())},
    }


def run_learned(args, api, torch, dist, rank, world, local, steps=None):
    """Learned start: train on plain-fitted toys (setup, untimed), then time
    the 1e4 fresh evaluation toys fitted from the network's start (with the
    plain fit as fallback) next to the same toys fitted from the plain start."""
    from paper_2003_12861_gb300 import learned

    spec = W.decay_model()
    model = api.Model.from_spec(spec)
    seed = W.SEED_BASE + 4 + 1000 * rank
    X, Y, tinfo = learned.build_training_set(model, args.train_toys, seed)
    net, ninfo = learned.train(X, Y, epochs=args.epochs, batch=1024, lr=1e-3, seed=seed)
    warm = learned.compare(net, model, 512, seed + 999)
    del warm
    with ClockSampler(local) as clk:
        r = None
        for _ in range(steps or args.steps):
            r = learned.compare(net, model, 10_000, seed + 777, characterise=True)
    if rank != 0:
        return None
    return {
        "value": r["learned"]["toy_fits_per_s"] * world, "unit": "toy fits/s",
        "ms_per_step": 1e3 * r["learned"]["wall_s"], "dtype": "f64 likelihood, bf16 x bf16 -> f32 network",
        "config": {"workload": "learned_start", "train_toys": tinfo["toys"], "train_converged": tinfo["converged"],
                   "eval_toys": 10_000, "sizes": "Poisson(N), N log-uniform in [1e3, 1e5]",
                   "theta": "uniform +-30% around the decay model's values", "network": "64-128-128-128-6 GELU",
                   "labels": "the deeper of the fits from the default start and from the generating values",
                   "tol_edm": r["tol_edm"],
                   "epochs": args.epochs},
        "learned_vs_plain": r,
        "training": {"build_s": tinfo["seconds"], "train_s": ninfo["seconds"], "final_loss": ninfo["final_loss"]},
        "e2e": {"value": r["learned"]["toy_fits_per_s"] * world, "unit": "toy fits/s",
                "h2d_bytes_per_step": 8 * 10_000 * 6, "d2h_bytes_per_step": 10_000 * 9 * 8,
                "note": "histogram, network, fits and fallback through the public API, host results"},
        "gpu_launches": r["learned"]["gpu_launches"], "clocks": clk.summary(),
    }


def binned_flops(spec):
    """Algorithmic FP64 flops of one binned NLL+gradient evaluation: per
    (sample, bin) entry its rate (two multiply-adds per histosys term: a_i
    alpha + b_i g, one product with the factor) and its weighted sum; per
    histosys modifier and bin its two weighted coefficient sums; per bin the
    weight and the Poisson term."""
    n_hs = {}
    for (smp, kind, *_rest) in spec["modifiers"]:
        if kind == 2:
            n_hs[smp] = n_hs.get(smp, 0) + 1
    rate = sum(len(h) * (1 + 4 * n_hs.get(s, 0)) for s, h in enumerate(spec["nominal"]))
    n_entries = sum(len(h) for h in spec["nominal"])
    hs_bins = sum(len(spec["nominal"][smp]) for (smp, kind, *_r) in spec["modifiers"] if kind == 2)
    return rate + 2 * n_entries + 4 * hs_bins + 4 * spec["n_bins"]


def run_binned(args, api, torch, dist, rank, world, local):
    """Binned (HistFactory-style) NLL + gradient of 4096 datasets of the
    28-channel, 253-nuisance model per step (one batched launch)."""
    spec = W.binned_model()
    m = api.BinnedModel(spec)
    S, P, Bn = 4096, spec["n_params"], spec["n_bins"]
    th = torch.as_tensor(W.binned_toy_thetas(S, W.SEED_BASE + 5 + 1000 * rank, P)).cuda()
    nu = torch.zeros((S, Bn), dtype=torch.float64, device="cuda")
    m.expected(th, nu)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(W.SEED_BASE + 6 + 1000 * rank)
    counts = torch.poisson(nu, generator=gen)
    out = torch.zeros((S, 1 + P), dtype=torch.float64, device="cuda")
    flags = torch.zeros(S, dtype=torch.int32, device="cuda")
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            m.nll_grad_async(counts, th, out, flags, stream=stream)
    stream.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    n_launch0 = api.launch_count()
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            for i in range(args.steps):
                flush.zero_()
                starts[i].record(stream)
                m.nll_grad_async(counts, th, out, flags, stream=stream)
                ends[i].record(stream)
        torch.cuda.synchronize()
    n_launches = api.launch_count() - n_launch0
    total_ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends))
    if dist:
        t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms = total_ms / args.steps
    # end to end: host counts and parameters in, host results out
    hc, ht = counts.cpu().numpy(), th.cpu().numpy()
    m.nll_grad(hc, ht)
    t0 = time.perf_counter()
    k = 5
    for _ in range(k):
        m.nll_grad(hc, ht)
    e2e_s = (time.perf_counter() - t0) / k
    if rank != 0:
        return None
    # batched fits of 256 of the datasets from the nominal point (each
    # fit's BFGS state holds a 256 x 256 inverse Hessian on the host)
    n_fit = 256
    lo = np.array([0.01] * 3 + [-5.0] * (P - 3))
    hi = np.array([5.0] * 3 + [5.0] * (P - 3))
    start = np.concatenate([[1.0, 1.0, 1.0], np.zeros(P - 3)])
    m.fit(hc[:8], start, lo, hi, want_cov=False)
    t0 = time.perf_counter()
    r = m.fit(hc[:n_fit], start, lo, hi, want_cov=False)
    fit_s = time.perf_counter() - t0
    fl = binned_flops(spec)
    fp64 = api.probe(0)
    fffma = 2.0 * api.probe(6)  # float-float multiply-adds, counted as 2 flops each
    achieved = S * fl / (ms * 1e-3)
    return {
        "value": world * S / (ms * 1e-3), "unit": "datasets/s", "ms_per_step": ms, "dtype": "f64",
        "config": {"workload": "binned_4096", "datasets": S, "channels": 28, "bins": Bn, "samples": len(spec["nominal"]),
                   "parameters": P, "modifiers": len(spec["modifiers"]),
                   "histograms": len(spec["nominal"]) + 2 * sum(1 for md in spec["modifiers"] if md[1] == 2),
                   "l2": "flushed between steps (256 MiB write); the model's histograms (3.6 MB) are re-read from L2"},
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": fffma / 1e12, "unit": "TFLOP/s",
                     "frac": achieved / fffma, "traffic": None,
                     "peak_basis": f"float-float multiply-add rate measured in-run (the kernel's multiply-add "
                                   f"loops run in float-float); {fl} algorithmic flops per dataset",
                     "fp64_fma_tflops_measured": fp64 / 1e12, "frac_of_fp64_fma": achieved / fp64},
        "e2e": {"value": world * S / e2e_s, "unit": "datasets/s", "h2d_bytes_per_step": S * (Bn + P) * 8,
                "d2h_bytes_per_step": S * (1 + P) * 8 + S * 4},
        "gpu_launches": int(n_launches), "clocks": clk.summary(),
        "fits": {"datasets": n_fit, "fits_per_s": n_fit / fit_s, "mean_evals": float(r["n_evals"].mean()),
                 "max_evals": int(r["n_evals"].max()), "converged_frac": float((r["status"] == 0).mean()),
                 "tol_edm": 1e-7, "start": "nominal (normfactors 1, nuisances 0)"},
    }


def exchange_partials(api, pairs, flags, group=None):
    """The sharded step's one exchange: every rank's compensated partial
    sums ((n_sets, 1 + P, 2) pairs and n_sets flags, host arrays) gathered
    in rank order over torch.distributed and merged exactly on every rank
    (rf_combine_partials).  Returns (NLL and gradient per set, flags)."""
    allp, allf = api.gather_partials(pairs, flags, group)
    return api.combine_partials(allp, allf)


def run_sharded(args, api, torch, dist, rank, world, local):
    """Strong scaling of one dataset: the product model's 1e8 events split
    over the ranks by rf_shard (contiguous 4096-aligned event ranges); per
    step every rank evaluates its shard's compensated partial sums
    (rf_nll_grad_partial: parameter point + event pass), the ranks exchange
    them once (an all_gather of (1 + 12) x 2 doubles per rank) and every rank
    merges them in rank order.  Each rank's shard is generated on its GPU
    (any in-range events serve the timing; the combine's correctness against
    the whole dataset is tested on its own)."""
    ctor, theta_true, n_total, f32, bpe = WORKLOADS["prod3_1e8_f32"]
    spec = W.model_for(ctor)
    model = api.Model.from_spec(spec)
    lo, hi = api.shard(n_total, 4096, rank, world)
    data = api.generate_toys(model, theta_true, W.SEED_BASE + 1 + 1000 * rank, [float(hi - lo)], poisson=False,
                             f32=[f32] * spec.n_obs)
    api.autotune(model, data, passes=2)
    P = model.n_free
    stream = torch.cuda.Stream()
    th = torch.tensor(theta_true * (1 + 0.02 * np.cos(np.arange(P))), dtype=torch.float64, device="cuda")
    pairs = torch.zeros((1, 1 + P, 2), dtype=torch.float64, device="cuda")
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step():
        api.nll_grad_partial(model, data, th, pairs, flags, stream=stream)
        stream.synchronize()
        return exchange_partials(api, pairs.cpu().numpy(), flags.cpu().numpy())

    for _ in range(args.warmup):
        step()
    ts = []
    dist.barrier()
    torch.cuda.synchronize()
    n_launch0 = api.launch_count()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            dist.barrier()
            t0 = time.perf_counter()
            out, fo = step()
            ts.append(time.perf_counter() - t0)
    n_launches = api.launch_count() - n_launch0
    t = torch.tensor([sum(ts)], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_s = float(t.item())
    if rank != 0:
        return None
    return {
        "value": n_total * args.steps / total_s, "unit": "events/s", "ms_per_step": 1e3 * total_s / args.steps,
        "dtype": path_dtype(model, f32),
        "config": {"workload": "prod3_1e8_f32", "mode": "one dataset sharded over the ranks (strong scaling)",
                   "n_events_total": n_total, "shard_events_rank0": hi - lo, "columns": "3 x f32",
                   "free_parameters": P, "l2": "flushed between steps (256 MiB write)",
                   "exchange": "one all_gather of (1 + 12) x 2 doubles per rank, rank-ordered exact merge"},
        "e2e": {"value": n_total * args.steps / total_s, "unit": "events/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": (1 + P) * 16 + 4,
                "note": "the step ends with the combined NLL and gradient on every rank's host"},
        "gpu_launches": int(n_launches), "clocks": clk.summary(), "nll_check": float(out[0, 0]), "scaling": "strong",
    }


def headline_extras(args, api, torch, local):
    """The rest of the metric beside the headline's events/s, each measured
    in this run on its own configuration: the decay model at 1e7 events
    (events/s and its 6-parameter fit), 4096 batched toy fits (toy fits/s)
    and learned-start against plain-start fits (toy fits/s, evaluations,
    identical minima)."""
    ex = {}
    t0 = time.perf_counter()
    d = run_events(args, api, torch, None, 0, 1, local, wl="decay_1e7", steps=100, fit_figure=True)
    ex["decay_1e7"] = {k: d[k] for k in ("value", "unit", "ms_per_step", "dtype", "config", "roofline", "e2e",
                                         "gpu_launches", "clocks", "fit")}
    ex["decay_1e7"]["cpu_baseline"] = {"kind": "oracle", "note": "see --workload decay_1e7"}
    t = run_toys(args, api, torch, None, 0, 1, local, steps=3, warmup=3)
    v, smp = oracle_toy_fits_per_s(8.0)
    t["cpu_baseline"] = {"value": v, "unit": "toy fits/s", "cores": 1, "kind": "oracle", "sample": smp}
    ex["toy_fits_4096"] = t
    ex["learned_vs_plain"] = run_learned(args, api, torch, None, 0, 1, local, steps=1)
    ex["seconds"] = time.perf_counter() - t0
    return ex


def run_ours(args):
    import torch

    from paper_2003_12861_gb300 import _lib as L
    from paper_2003_12861_gb300 import api

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    L.load()
    headline = args.workload == "prod3_1e8_f32" and not args.shard
    if args.shard:
        if dist is None:  # one rank: the same step with a one-rank group
            import torch.distributed as dist

            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            os.environ.setdefault("MASTER_PORT", "29531")
            dist.init_process_group("gloo", rank=0, world_size=1)
        line = run_sharded(args, api, torch, dist, rank, world, local)
    elif args.workload == "decay_toys_4096":
        line = run_toys(args, api, torch, dist, rank, world, local)
    elif args.workload == "learned_start":
        line = run_learned(args, api, torch, dist, rank, world, local)
    elif args.workload == "binned_4096":
        line = run_binned(args, api, torch, dist, rank, world, local)
    else:
        line = run_events(args, api, torch, dist, rank, world, local, fp64_figure=headline and rank == 0,
                          fit_figure=args.workload == "decay_1e7")
    if headline and world == 1 and not args.no_extras:
        line["extras"] = headline_extras(args, api, torch, local)
    if rank == 0:
        full = {"metric": METRIC, "value": line.pop("value"), "unit": line.pop("unit"), "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": line.pop("ms_per_step"),
                "higher_is_better": True, "scaling": line.pop("scaling", "weak"), "vs_baseline": None,
                "dtype": line.pop("dtype"), "data": "synthetic"}
        full.update(line)
        if not args.no_cpu_baseline:
            full["cpu_baseline"] = cpu_baseline(args.workload)
        print(json.dumps(full), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="prod3_1e8_f32", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--shard", action="store_true",
                    help="strong scaling: one 1e8-event dataset sharded over the ranks, one exchange per step")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload: skip the decay, toy-fit and learned-start figures")
    ap.add_argument("--blocks-per-sm", type=int, default=0,
                    help="resident blocks per SM of the event kernel instead of the autotuner's winner (the grid "
                         "is still scanned and reported); for profiling runs, whose timings the profiler distorts")
    ap.add_argument("--train-toys", type=int, default=1_000_000, help="learned_start: training toys")
    ap.add_argument("--epochs", type=int, default=20, help="learned_start: training epochs")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = DEFAULT_STEPS[args.workload] if not args.shard else 20
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
