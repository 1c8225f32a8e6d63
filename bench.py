#!/usr/bin/env python
"""Throughput of the NFFT-like procedure for bandlimited functions on GB300.

Workload (default, the d = 2 configuration the metric is quoted on): d = 2,
M = 256 x 256, sigma = 2 (L = 512 x 512), sinh window, m = 8 (the smallest
m in {4, 6, 8} whose error against the trigonometric sum is <= 1e-6),
N = 2^20 nodes i.i.d. uniform in [-1/2, 1/2)^2 (float32), fhat complex64
N(0,1) times the triangle envelope, adjoint input complex64 N(0,1).  All
inputs are synthetic and seeded (module ``workloads``).

One step = one forward transform (Algorithm 4.2 steps 1-3: precorrection +
oversampled FFT + short sums) and one adjoint transform (spreading +
forward-sign FFT + crop/weight) of the FP32 plan on one batch, with the
nodes already binned (set_nodes is amortised; its time is reported
separately).  value = N nodes / step time (nodes/s through one
forward + adjoint round trip).  The headline step is the pair of C-ABI calls
captured once in a CUDA graph and replayed (the launch mode a serving loop
uses); the same step launched call by call on the stream is timed beside it
(`stream_ms_per_step`).  The L2 cache is flushed (a 256 MiB write) before
every timed step, outside the timed events.

Also reported: the plain FP64 GPU path on the same inputs and its speed
ratio, the FP32 error against the FP64 path, per-kernel device times,
the roofline of the dominant kernel, end-to-end throughput through the
C-ABI with host buffers, the oracle on the host cores (cpu_baseline) and
SM clocks sampled during the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "nodes/s at rel. err <=1e-6 (d=2,3): FP32/learned vs plain FP64; % roofline"
UNIT = "nodes/s"

CONFIGS = {
    # name: (d, M, m, N, batch, node kind)
    "d2_M256_m8_N2^20": (2, 256, 8, 1 << 20, 1, "uniform"),
    "d3_M128_m6_N2^23_spokes": (3, 128, 6, 1 << 23, 1, "spokes"),
    "d2_M512_m6_N4e6_B8": (2, 512, 6, 4_000_000, 8, "uniform"),
    "d1_M256_m8_N1024": (1, 256, 8, 1024, 1, "uniform"),
    # smaller spoke case for profiler captures (same density profile, 1/8 of the nodes)
    "d3_M128_m6_N2^20_spokes": (3, 128, 6, 1 << 20, 1, "spokes"),
}
DEFAULT_CONFIG = "d2_M256_m8_N2^20"
# FP32 flavour of the timed plan: the d = 3 workload is specified with
# compensated accumulation of the tap sums ("f32c"), the others plain FP32.
PRECISION = {"d3_M128_m6_N2^23_spokes": "f32c", "d3_M128_m6_N2^20_spokes": "f32c"}

# GB300 unit counts at the maximum SM clock (2070 MHz): 152 SMs; 128 FP32
# FMA lanes per SM; the special-function unit issues 16 lanes per SM per clock
# for rsqrt / rcp and 32 for ex2 (measured with ``bench.py --unit-rates``).
# The roofline of a short-sum kernel is the largest of its FP32 time, its SFU
# time and its HBM time; the JSON reports the binding one.
SMS = 152
FP32_LANES = 128
SFU_SLOTS = 16           # SFU issue slots per SM per clock (rsqrt, rcp: 1 slot; ex2: 1/2)
SM_MAX_MHZ = 2070.0
# SFU slots per tap weight of the sinh window: rsqrt + rcp + 2 ex2 (1/2 each)
SFU_SLOTS_PER_WEIGHT = 3.0

# DRAM bytes (read + write) per launch of the short-sum kernels from one ncu
# capture of the same workload and kernel version (the launch-list profile
# summary of each workload); absent when not captured for the current code.
NCU_TRAFFIC_BYTES = {
    ("d2_M256_m8_N2^20", "spread"): 21113344,
    ("d2_M256_m8_N2^20", "interp"): 14765824,
}


def short_sum_roofline(d, m, N, B, M, seconds):
    """Roofline of one interpolation or spreading launch (N nodes, batch B):
    algorithmic FP32 flops 5 (2m)^d per node and batch entry, SFU slots
    3 * d * 2m per node (one sinh-window weight per tap and dimension), HBM
    bytes (4d + 8) per node and batch entry plus one pass over the L^d grid.
    Reports the unit whose time bound is largest."""
    f = SM_MAX_MHZ * 1e6
    flops = 5.0 * (2 * m) ** d * N * B
    slots = SFU_SLOTS_PER_WEIGHT * d * 2 * m * N
    hbm_bytes = (4 * d + 8) * N * B + 8 * (2 * M) ** d * B
    peaks = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0)) * 1e9
    t = {"fp32": flops / (SMS * FP32_LANES * 2 * f), "sfu": slots / (SMS * SFU_SLOTS * f),
         "hbm": hbm_bytes / hbm_peak}
    unit = max(t, key=t.get)
    if unit == "fp32":
        out = {"bound": "alu", "achieved": flops / seconds / 1e12, "peak": SMS * FP32_LANES * 2 * f / 1e12,
               "unit": "TFLOP/s", "peak_note": "FP32 FMA: 152 SMs x 128 lanes x 2 flop x 2070 MHz (derived)"}
    elif unit == "sfu":
        out = {"bound": "alu", "achieved": slots / seconds / 1e12, "peak": SMS * SFU_SLOTS * f / 1e12,
               "unit": "Tslot/s (SFU)",
               "peak_note": "SFU: 152 SMs x 16 issue slots x 2070 MHz; rsqrt, rcp 1 slot, ex2 1/2 (measured rates)"}
    else:
        out = {"bound": "hbm", "achieved": hbm_bytes / seconds / 1e9, "peak": hbm_peak / 1e9, "unit": "GB/s",
               "peak_note": "measured copy bandwidth"}
    out["frac"] = out["achieved"] / out["peak"]
    out["bound_unit"] = unit
    out["t_bound_us"] = {k: v * 1e6 for k, v in t.items()}
    out["flops_per_launch"] = flops
    out["sfu_slots_per_launch"] = slots
    out["hbm_bytes_per_launch"] = hbm_bytes
    return out


def aggregate_over_ranks(t_step_ms, units_per_rank, world, device=None):
    """Whole-job figures of N replicas: the step time is the maximum over the
    ranks (every rank processes units_per_rank units per step), the value the
    units of all ranks per second.  Returns (t_max_ms, value)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        tt = torch.tensor([float(t_step_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_step_ms = float(tt.item())
    return t_step_ms, world * units_per_rank / (t_step_ms * 1e-3)


def run_paper(args):
    """The paper's experiments on the GPU (Section 5): Example 5.1 for both
    algorithms in FP64 and FP32, and Fig. 5.1's e(v) at P = 10^5 points for
    961 frequencies (one batched interpolation per curve).  Prints one JSON
    line with the errors and the times."""
    import torch
    from paper_2502_07155_gb300 import build
    build.build()
    from paper_2502_07155_gb300.experiments import example51_errors, fig51_errors
    torch.cuda.set_device(0)
    Ms = [20, 40, 80, 100, 200, 400, 600, 800, 1000]
    ex = {str(M): {f"{meth}_{prec}": example51_errors(M, 5, prec, meth) for meth in ("shannon", "classic")
                   for prec in ("f64", "f32")} for M in Ms}
    for M in Ms:   # ablation: D = I (Section 5's |I_L| psi_hat ~ 1)
        ex[str(M)]["shannon_f64_D=I"] = example51_errors(M, 5, "f64", "shannon", precorrect=False)
    beta_sh = float(np.pi * 5 * 0.5)
    curves = {}
    for name, kw in [("shannon_full", dict(interval="full")), ("shannon_trunc", dict(interval="trunc")),
                     ("classic_full", dict(interval="full", method="classic")),
                     ("classic_trunc", dict(interval="trunc", method="classic")),
                     ("classic_trunc_beta_shannon", dict(interval="trunc", method="classic", beta=beta_sh))]:
        fig51_errors(P=1000, **kw)   # warm-up (builds the plan's kernels)
        v, e, sec = fig51_errors(P=100_000, **kw)
        inner = np.abs(v) <= 9
        nonint = inner & (np.abs(v - np.round(v)) > 1e-9)
        integ = inner & ~nonint
        curves[name] = {"median_nonint_inner": float(np.median(e[nonint])), "max_nonint_inner": float(e[nonint].max()),
                        "max_int_inner": float(e[integ].max()), "interp_seconds": sec,
                        "node_evaluations_per_s": v.size * 100_000 / sec}
    print(json.dumps({"metric": "paper experiments on GPU (Example 5.1 max error; Fig. 5.1 e(v))",
                      "example_5_1": ex, "fig_5_1": {"M": 20, "m": 5, "S": 32, "P": 100_000, "frequencies": 961,
                                                      "curves": curves}}))
    return 0


def run_unit_rates():
    """Build and run the unit-rate microbenchmark (FP32 FMA, ex2, rsqrt, rcp
    lane operations per SM per clock); prints one JSON line per unit."""
    src = os.path.join(ROOT, "paper_2502_07155_gb300", "unit_rates.cu")
    exe = os.path.join(ROOT, "paper_2502_07155_gb300", "_build", "unit_rates")
    os.makedirs(os.path.dirname(exe), exist_ok=True)
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe, src], check=True)
    return subprocess.run([exe]).returncode


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


def make_inputs(cfg):
    d, M, m, N, B, kind = CONFIGS[cfg]
    if kind == "spokes":
        x = W.nodes_spokes(n_spokes=1 << 13, per_spoke=N >> 13)
    else:
        x = W.nodes_uniform(N, d)
    envelope = cfg != "d2_M512_m6_N4e6_B8"
    fh = W.fhat_gaussian(M, d, batch=B, envelope=envelope)
    g = W.adjoint_input(N, batch=B)
    return x, fh, g


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        mhz = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        maxm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for i, nm in enumerate(names):
                if r[5 + i].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": max(maxm) if maxm else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# --------------------------------------------------------------------------- CPU baseline (oracle)

_ORACLE_CHILD = r"""
import json, sys, time, numpy as np
sys.path.insert(0, sys.argv[1])
import oracle as O
z = np.load(sys.argv[2])
d, M, m = int(z["d"]), int(z["M"]), int(z["m"])
p = O.make_plan(d, M, 2.0, m, beta=float(z["beta"]))
fac = O.precorrection_factors(p)
x, fh, g = z["x"], z["fh"], z["g"]
t0 = time.perf_counter()
grid = O.grid_samples(p, fh, fac)
f = O.step3_short_sums(p, grid, x)
h = O.adjoint(p, g, x, fac)
t = time.perf_counter() - t0
out = {"seconds": t, "n": int(x.shape[0])}
if "f_gpu" in z.files:
    fg = z["f_gpu"]
    out["fp32_vs_oracle_rel_l2"] = float(np.linalg.norm(fg - f) / np.linalg.norm(f))
    feas = np.flatnonzero(np.all(np.abs(x) < 0.5 - m / (2.0 * M), axis=1))[:2000]
    if feas.size:
        nd = O.ndft(fh, x[feas])
        out["oracle_vs_ndft_rel_l2_feasible"] = float(np.linalg.norm(f[:, feas] - nd) / np.linalg.norm(nd))
        out["fp32_vs_ndft_rel_l2_feasible"] = float(np.linalg.norm(fg[:, feas] - nd) / np.linalg.norm(nd))
        out["ndft_sample"] = int(feas.size)
print(json.dumps(out))
"""


def run_oracle_sample(cfg, x, fh, g, beta, n_sample, f_gpu=None):
    """Time the oracle (forward + adjoint, single thread) on the first n_sample
    nodes in a child process (no GPU).  Returns its JSON dict."""
    d, M, m, N, B, kind = CONFIGS[cfg]
    fd, path = tempfile.mkstemp(suffix=".npz")
    os.close(fd)
    arrays = dict(d=d, M=M, m=m, beta=beta, x=x[:n_sample], fh=fh, g=g[:, :n_sample])
    if f_gpu is not None:
        arrays["f_gpu"] = f_gpu[:, :n_sample]
    np.savez(path, **arrays)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    try:
        res = subprocess.run([sys.executable, "-c", _ORACLE_CHILD, ROOT, path], capture_output=True, text=True,
                             env=env, timeout=900)
    finally:
        os.unlink(path)
    if res.returncode != 0:
        raise RuntimeError("oracle child failed: " + res.stderr[-2000:])
    return json.loads(res.stdout.strip().splitlines()[-1])


# --------------------------------------------------------------------------- reference arm

def run_reference(args, cfg):
    """The oracle as the reference arm: each step is forward + adjoint of the
    oracle on a bounded sample of the workload's nodes (full grid DFT)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    d, M, m, N, B, kind = CONFIGS[cfg]
    x, fh, g = make_inputs(cfg)
    n_sample = min(1 << 13, N)
    sys.path.insert(0, ROOT)
    times = []
    for i in range(args.warmup + args.steps):
        r = run_oracle_sample(cfg, x, fh, g, float(np.pi * m * 0.5), n_sample)
        if i >= args.warmup:
            times.append(r["seconds"])
    t = float(np.mean(times))
    value = n_sample / t
    sample = f"first {n_sample} of the {N} nodes with the full grid DFT (M={M}^{d}, L={2 * M}^{d}), forward + adjoint"
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": cfg, "d": d, "M": M, "m": m, "N": N, "batch": B, "nodes": kind},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


# --------------------------------------------------------------------------- our arm

def run_ours(args, cfg):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local_rank)
    if local_rank == 0:
        from paper_2502_07155_gb300 import build
        build.build()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
        dist.barrier()
    import paper_2502_07155_gb300 as nb

    d, M, m, N, B, kind = CONFIGS[cfg]
    x, fh, g = make_inputs(cfg)
    dev = torch.device("cuda", local_rank)
    x_d = torch.from_numpy(x).to(dev)
    fh_d = torch.from_numpy(fh).to(dev)
    g_d = torch.from_numpy(g).to(dev)

    plan = nb.Plan(d, M, 2.0, m, precision=PRECISION.get(cfg, "f32"), batch=B)
    t0 = time.perf_counter()
    plan.set_nodes(x_d)
    t_set_first = time.perf_counter() - t0
    f_out = torch.empty((B, N), dtype=torch.complex64, device=dev)
    h_out = torch.empty((B,) + (M,) * d, dtype=torch.complex64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        plan.forward(fh_d, out=f_out)
        plan.adjoint(g_d, out=h_out)

    for _ in range(args.warmup):
        step()
    plan.sync()

    # set_nodes alone (binning, a1), timed with events (it synchronises)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    set_ms = []
    for _ in range(3):
        flush.zero_()
        ev0.record(stream)
        plan.set_nodes(x_d)
        ev1.record(stream)
        ev1.synchronize()
        set_ms.append(ev0.elapsed_time(ev1))

    # ---- per-kernel device times (CUDA events around every launch), in a
    # pass of their own so that the events do not sit inside the timed steps
    plan.kernel_timing(True)
    for _ in range(args.steps):
        flush.zero_()
        step()
    plan.sync()
    ktimes = plan.kernel_times()
    plan.kernel_timing(False)

    # ---- the step captured once in a CUDA graph (replayed in the timed region)
    graph = None
    if not args.no_graph:
        g_stream = torch.cuda.Stream()
        g_stream.wait_stream(stream)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(g_stream):
            step()
            torch.cuda.synchronize()
            with torch.cuda.graph(graph, stream=g_stream):
                step()
        torch.cuda.synchronize()
        for _ in range(3):
            graph.replay()
        torch.cuda.synchronize()

    # ---- timed region: K stream-launched steps, then K graph replays
    def timed_steps(run):
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        for i in range(args.steps):
            flush.zero_()
            starts[i].record(stream)
            run()
            ends[i].record(stream)
        torch.cuda.synchronize()
        return float(np.mean([starts[i].elapsed_time(ends[i]) for i in range(args.steps)]))

    clocks = ClockSampler(local_rank)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = plan.kernel_launches()
    t_stream = timed_steps(step)
    launches_per_step = (plan.kernel_launches() - launches0) / args.steps
    t_graph = timed_steps(graph.replay) if graph is not None else None
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    plan.sync()
    t_step = t_graph if t_graph is not None else t_stream
    launches = int(round(launches_per_step * args.steps))
    t_step, value = aggregate_over_ranks(t_step, N, world, dev)
    launch_mode = "CUDA graph replay of the captured forward + adjoint calls" if graph is not None else "stream launches"
    if args.quick:
        # timed region only (used for profiling captures): no comparison legs
        if rank == 0:
            print(json.dumps({"quick": True, "config": cfg, "ms_per_step": t_step, "value": value,
                              "unit": UNIT, "gpu_launches": launches, "clocks": clk,
                              "set_nodes_ms": float(np.median(set_ms)), "stream_ms_per_step": t_stream,
                              "launch": launch_mode,
                              "kernels": {k: {"ms_total": v[0], "launches": v[1]} for k, v in ktimes.items()}}))
        if world > 1:
            dist.destroy_process_group()
        plan.close()
        return 0

    # ---- per-direction times (same plan, events around each call)
    def timed(fn, reps):
        out = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            out.append(a.elapsed_time(b))
        return float(np.median(out))

    fwd_ms = timed(lambda: plan.forward(fh_d, out=f_out), max(3, args.steps // 2))
    adj_ms = timed(lambda: plan.adjoint(g_d, out=h_out), max(3, args.steps // 2))
    gx = torch.empty((N, d), dtype=torch.float32, device=dev)
    grad_ms = timed(lambda: plan.node_grad(fh_d, g_d, out=gx), 3)
    f32 = plan.forward(fh_d, out=f_out).clone()
    plan.sync()

    # ---- classical NFFT (Algorithm 2.1) on the same inputs, FP32
    cplan = nb.Plan(d, M, 2.0, m, precision="f32", method="classic", batch=B)
    cplan.set_nodes(x_d)
    for _ in range(2):
        cplan.forward(fh_d, out=f_out)
        cplan.adjoint(g_d, out=h_out)
    cls_ms = timed(lambda: (cplan.forward(fh_d, out=f_out), cplan.adjoint(g_d, out=h_out)), 3)
    cplan.sync()
    cplan.close()

    # ---- FP32 with compensated (Neumaier) accumulation of the tap rows
    kplan = nb.Plan(d, M, 2.0, m, precision="f32c", batch=B)
    kplan.set_nodes(x_d)
    for _ in range(2):
        kplan.forward(fh_d, out=f_out)
        kplan.adjoint(g_d, out=h_out)
    comp_ms = timed(lambda: (kplan.forward(fh_d, out=f_out), kplan.adjoint(g_d, out=h_out)), 3)
    f32c = kplan.forward(fh_d, out=f_out).clone()
    kplan.sync()
    kplan.close()

    # ---- plain FP64 GPU path on the same inputs
    plan64 = nb.Plan(d, M, 2.0, m, precision="f64", batch=B)
    x64 = torch.from_numpy(x.astype(np.float64)).to(dev)
    fh64 = torch.from_numpy(fh.astype(np.complex128)).to(dev)
    g64 = torch.from_numpy(g.astype(np.complex128)).to(dev)
    plan64.set_nodes(x64)
    f64o = torch.empty((B, N), dtype=torch.complex128, device=dev)
    h64o = torch.empty((B,) + (M,) * d, dtype=torch.complex128, device=dev)
    plan64.forward(fh64, out=f64o)
    plan64.adjoint(g64, out=h64o)
    plan64.sync()
    reps64 = 2 if N * (2 * m) ** d > 5e9 else 3
    f64_ms = timed(lambda: (plan64.forward(fh64, out=f64o), plan64.adjoint(g64, out=h64o)), reps64)
    f64 = plan64.forward(fh64, out=f64o)
    plan64.sync()
    err_fp32_fp64 = float(torch.linalg.vector_norm(f32.to(torch.complex128) - f64) / torch.linalg.vector_norm(f64))
    err_fp32c_fp64 = float(torch.linalg.vector_norm(f32c.to(torch.complex128) - f64) / torch.linalg.vector_norm(f64))
    plan64.close()

    # ---- end to end through the C-ABI with pinned host buffers
    fh_h = torch.from_numpy(fh).pin_memory()
    g_h = torch.from_numpy(g).pin_memory()
    f_h = torch.empty((B, N), dtype=torch.complex64).pin_memory()
    h_h = torch.empty((B,) + (M,) * d, dtype=torch.complex64).pin_memory()

    # end to end through the host-buffer C-ABI calls: the inputs are uploaded
    # from page-locked host memory and both results downloaded inside the
    # timed region; the plan overlaps the adjoint's upload with the forward
    # transform and the forward's download with the adjoint
    def e2e_step():
        plan.forward_host(fh_h, out=f_h)
        plan.adjoint_host(g_h, out=h_h)
        plan.join()

    for _ in range(2):
        e2e_step()
    plan.sync()
    torch.cuda.synchronize()
    e2e_ms, e2e_wall = [], []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()    # nothing of the step may start before the first event
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        w0 = time.perf_counter()
        a.record(stream)
        e2e_step()
        b.record(stream)
        b.synchronize()
        e2e_wall.append((time.perf_counter() - w0) * 1e3)
        e2e_ms.append(a.elapsed_time(b))
    e2e_t = float(np.mean(e2e_ms))
    e2e_wall_t = float(np.mean(e2e_wall))
    h2d = fh_h.numel() * 8 + g_h.numel() * 8
    d2h = f_h.numel() * 8 + h_h.numel() * 8

    # ---- roofline of the dominant short-sum kernel
    dom = max(("interp", "spread"), key=lambda k: ktimes[k][0])
    dom_ms, dom_n = ktimes[dom]
    per_launch_s = dom_ms / max(dom_n, 1) * 1e-3
    roofline = short_sum_roofline(d, m, N, B, M, per_launch_s)
    roofline["kernel"] = dom
    roofline["traffic"] = NCU_TRAFFIC_BYTES.get((cfg, dom))

    result = None
    if rank == 0:
        # cpu baseline: the oracle on a bounded sample of the same workload
        n_sample = 1 << 18 if d <= 2 else 1 << 13
        n_sample = min(n_sample, N)
        cb = run_oracle_sample(cfg, x, fh, g, plan.beta, n_sample, f_gpu=f32.cpu().numpy())
        cpu_value = cb["n"] / cb["seconds"]
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": cfg, "d": d, "M": M, "sigma": 2.0, "L": 2 * M, "m": m, "N": N, "batch": B,
                       "nodes": kind, "window": "sinh", "beta": plan.beta, "precision": PRECISION.get(cfg, "f32"),
                       "step": "forward + adjoint (nodes binned once)", "l2": "flushed (256 MiB write) before each step",
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                       "launch": launch_mode, "stream_ms_per_step": t_stream},
            "e2e": {"value": world * N / (e2e_t * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_t, "host_wall_ms_per_step": e2e_wall_t,
                    "api": "nfftbl_forward_host + nfftbl_adjoint_host + nfftbl_join (page-locked host buffers)"},
            "gpu_launches": launches,
            "roofline": roofline,
            "cpu_baseline": {"value": cpu_value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"first {cb['n']} of the {N} nodes, full grid DFT, forward + adjoint, "
                                       f"one thread ({cb['seconds']:.1f} s)"},
            "clocks": clk,
            "breakdown_ms": {"forward": fwd_ms, "adjoint": adj_ms, "set_nodes": float(np.median(set_ms)),
                             "set_nodes_first_call_s": t_set_first, "node_grad": grad_ms,
                             "kernels_in_timed_region": {k: {"ms_total": v[0], "launches": v[1]}
                                                         for k, v in ktimes.items()}},
            "fp64": {"ms_per_step": f64_ms, "nodes_per_s": N / (f64_ms * 1e-3), "speedup_fp32": f64_ms / t_step},
            "classic_nfft_fp32": {"ms_per_step": cls_ms, "nodes_per_s": N / (cls_ms * 1e-3)},
            "fp32_compensated": {"ms_per_step": comp_ms, "nodes_per_s": N / (comp_ms * 1e-3),
                                 "fp32c_vs_fp64_gpu_rel_l2": err_fp32c_fp64},
            "accuracy": {"fp32_vs_fp64_gpu_rel_l2": err_fp32_fp64,
                         **{k: v for k, v in cb.items() if k not in ("seconds", "n")}},
        }
        print(json.dumps(result))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    plan.close()
    return 0


def run_ablation(args):
    """Window, method, beta and precorrection ablations at d = 2, M = 256,
    sigma = 2 on 2^20 held-out feasible nodes (Fourier data N(0,1) x
    triangle): relative l2 error against the trigonometric sums (FP64
    classical NFFT at m = 12) for m = 2..8, the FP32 forward time of each
    configuration at the same size, and a sweep of beta around its default."""
    import torch
    from paper_2502_07155_gb300 import build
    build.build()
    import paper_2502_07155_gb300 as nb

    d, M = 2, 256
    L = 2 * M
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    ms = list(range(2, 9))
    x = W.nodes_feasible(1 << 20, d, max(ms) + 1, L, seed=W.SEED_HELDOUT)
    fh = W.fhat_gaussian(M, d, seed=W.SEED_HELDOUT)
    x64 = torch.from_numpy(x.astype(np.float64)).to(dev)
    x32 = torch.from_numpy(x.astype(np.float32)).to(dev)
    fh64 = torch.from_numpy(fh.astype(np.complex128)).to(dev)
    fh32 = torch.from_numpy(fh.astype(np.complex64)).to(dev)
    ref_plan = nb.Plan(d, M, 2.0, 12, precision="f64", method="classic")
    ref_plan.set_nodes(x64)
    ref = ref_plan.forward(fh64)
    ref_plan.close()

    def rel(a):
        return float(torch.linalg.vector_norm(a.to(torch.complex128) - ref) / torch.linalg.vector_norm(ref))

    def error(m, precision="f64", **kw):
        plan = nb.Plan(d, M, 2.0, m, precision=precision, **kw)
        plan.set_nodes(x64 if precision == "f64" else x32)
        e = rel(plan.forward(fh64 if precision == "f64" else fh32))
        plan.close()
        return e

    def fwd_ms(m, **kw):
        plan = nb.Plan(d, M, 2.0, m, precision="f32", **kw)
        plan.set_nodes(x32)
        out = torch.empty((1, x.shape[0]), dtype=torch.complex64, device=dev)
        for _ in range(3):
            plan.forward(fh32, out=out)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(10):
            plan.forward(fh32, out=out)
        b.record()
        b.synchronize()
        plan.close()
        return a.elapsed_time(b) / 10

    variants = {
        "shannon_sinh": dict(method="shannon", window="sinh"),
        "shannon_ckb": dict(method="shannon", window="ckb"),
        "classic_sinh": dict(method="classic", window="sinh"),
        "classic_ckb": dict(method="classic", window="ckb"),
        "shannon_sinh_D=I": dict(method="shannon", window="sinh", precorrect=False),
    }
    table = {}
    for name, kw in variants.items():
        table[name] = {str(m): {"err_f64": error(m, **kw), "fwd_ms_f32": fwd_ms(m, **kw)} for m in ms}
    for m in ms:
        table["shannon_sinh"][str(m)]["err_f32"] = error(m, "f32", method="shannon", window="sinh")
    sweep = {}
    for m in (4, 6, 8):
        b0 = nb.Plan(d, M, 2.0, m, precision="f64").beta
        sweep[str(m)] = {f"{f:.2f}": error(m, method="shannon", window="sinh", beta=f * b0)
                         for f in (0.6, 0.8, 0.9, 1.0, 1.1, 1.2, 1.4)}
        sweep[str(m)]["beta_default"] = b0
    print(json.dumps({"metric": "ablations: relative l2 error against the trigonometric sums, FP32 forward ms",
                      "config": {"workload": "ablation_d2_M256_sigma2", "nodes": x.shape[0],
                                 "nodes_kind": f"uniform feasible for m = {max(ms) + 1}",
                                 "targets": "FP64 classical NFFT m=12"},
                      "by_m": table, "beta_sweep": sweep}))
    return 0


def run_learned(args):
    """Learned window at d = 2, M = 256, sigma = 2: train phi_theta on 2^16
    feasible uniform nodes (Fourier data N(0,1) x triangle), then compare with
    the sinh window on 2^22 held-out nodes at equal m and by the m each needs
    for a given error.  Targets are the trigonometric sums, computed by the
    FP64 classical NFFT at m = 12 (equal to the NDFT to ~1e-14)."""
    import torch
    from paper_2502_07155_gb300 import build
    build.build()
    import paper_2502_07155_gb300 as nb
    from paper_2502_07155_gb300.learned import WindowTrainer

    d, M = 2, 256
    L = 2 * M
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)

    def targets(x, fh):
        ref = nb.Plan(d, M, 2.0, 12, precision="f64", method="classic")
        ref.set_nodes(torch.from_numpy(x.astype(np.float64)).to(dev))
        out = ref.forward(torch.from_numpy(fh.astype(np.complex128)).to(dev))
        ref.close()
        return out

    def rel(a, b):
        return float(torch.linalg.vector_norm(a.to(torch.complex128) - b) / torch.linalg.vector_norm(b))

    def fwd_time(plan, fh_d, out):
        for _ in range(3):
            plan.forward(fh_d, out=out)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(10):
            plan.forward(fh_d, out=out)
        b.record()
        b.synchronize()
        return a.elapsed_time(b) / 10

    results = []
    for m in args.learned_m:
        xt = W.nodes_feasible(1 << 16, d, m, L, seed=W.SEED_TRAIN)
        fht = W.fhat_gaussian(M, d, seed=W.SEED_TRAIN)
        yt = targets(xt, fht).to(torch.complex64)
        tr = WindowTrainer(d, M, m, lr=args.learned_lr)
        tr.set_data(torch.from_numpy(xt).to(dev), torch.from_numpy(fht).to(dev), yt)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hist = tr.train(args.learned_steps, log_every=max(1, args.learned_steps // 5))
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        tab = tr.table_host()
        # held-out nodes feasible for the largest m compared (m + 2)
        xh = W.nodes_feasible(1 << 22, d, m + 2, L, seed=W.SEED_HELDOUT)
        fhh = W.fhat_gaussian(M, d, seed=W.SEED_HELDOUT)
        yh = targets(xh, fhh)
        xh_d = torch.from_numpy(xh).to(dev)
        fhh_d = torch.from_numpy(fhh).to(dev)
        out = torch.empty((1, xh.shape[0]), dtype=torch.complex64, device=dev)
        row = {"m": m, "train_steps": args.learned_steps, "train_seconds": t_train,
               "train_loss": [[i, v] for i, v in hist]}
        pl = nb.Plan(d, M, 2.0, m, window="table", table=tab, precision="f32")
        pl.set_nodes(xh_d)
        row["learned_err"] = rel(pl.forward(fhh_d, out=out), yh)
        row["learned_fwd_ms"] = fwd_time(pl, fhh_d, out)
        pl.close()
        sinh = {}
        for ms in sorted(set([m, m + 1, m + 2])):
            ps = nb.Plan(d, M, 2.0, ms, precision="f32")
            ps.set_nodes(xh_d)
            sinh[ms] = {"err": rel(ps.forward(fhh_d, out=out), yh), "fwd_ms": fwd_time(ps, fhh_d, out)}
            ps.close()
        row["sinh"] = sinh
        row["gain_equal_m"] = sinh[m]["err"] / row["learned_err"]
        results.append(row)
        print(json.dumps(row), file=sys.stderr)
    out = {"metric": "learned window vs sinh window: held-out relative l2 error against the trigonometric sum",
           "config": {"workload": "learned_window_d2_M256_sigma2", "train_nodes": 1 << 16, "heldout_nodes": 1 << 22,
                      "targets": "FP64 classical NFFT m=12", "mlp": "1-64-64-1 tanh, BF16 backward",
                      "table_len": 4097},
           "results": results, "data": "synthetic", "n_gpus": 1}
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", choices=sorted(CONFIGS), default=DEFAULT_CONFIG)
    ap.add_argument("--learned", action="store_true", help="train and evaluate the learned window (d=2, M=256)")
    ap.add_argument("--learned-m", type=int, nargs="+", default=[2, 3, 4], dest="learned_m")
    ap.add_argument("--learned-steps", type=int, default=1500, dest="learned_steps")
    ap.add_argument("--learned-lr", type=float, default=3e-3, dest="learned_lr")
    ap.add_argument("--paper", action="store_true", help="run the paper's experiments (Example 5.1, Fig. 5.1)")
    ap.add_argument("--unit-rates", action="store_true", dest="unit_rates",
                    help="measure FP32 FMA and SFU lane rates per SM (roofline peaks)")
    ap.add_argument("--no-graph", action="store_true", dest="no_graph",
                    help="time stream-launched steps only (default: the headline replays the step as a CUDA graph)")
    ap.add_argument("--ablation", action="store_true",
                    help="window / method / beta / precorrection ablations (d=2, M=256): error and FP32 forward time")
    ap.add_argument("--quick", action="store_true",
                    help="timed region only (no FP64, classical, end-to-end or oracle legs); for profiling")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.unit_rates:
        return run_unit_rates()
    if args.paper:
        return run_paper(args)
    if args.impl == "reference":
        return run_reference(args, args.config)
    if args.learned:
        return run_learned(args)
    if args.ablation:
        return run_ablation(args)
    return run_ours(args, args.config)


if __name__ == "__main__":
    sys.exit(main())
