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

Also reported, on the same line: forward-only and adjoint-only throughput
(N / time of one direction); the plain FP64 GPU path on the same inputs,
timed the same two ways (graph replay against graph replay, stream launches
against stream launches) with both speed ratios; the FP32 error against the
FP64 path and, on feasible sampled nodes, both errors against the
trigonometric sums (FP64 classical NFFT at large m); per-kernel device times;
the roofline of both short-sum kernels; the oversampled FFT against cuFFT
(torch.fft) on the same grid; end-to-end throughput through the C-ABI with
host buffers; the oracle on every host core (cpu_baseline, the same sample
as the reference arm); SM clocks sampled during the timed region; and the
metric's d = 3 half, the radial-spoke workload (M = 128^3, N = 2^23) at
m = 8 (the smallest m at relative error <= 1e-6) and at m = 6, each with the
same timings, ratios and rooflines (key "d3").

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
    "d3_M128_m8_N2^23_spokes": (3, 128, 8, 1 << 23, 1, "spokes"),
    "d2_M512_m6_N4e6_B8": (2, 512, 6, 4_000_000, 8, "uniform"),
    "d1_M256_m8_N1024": (1, 256, 8, 1024, 1, "uniform"),
    # smaller spoke case for profiler captures (same density profile, 1/8 of the nodes)
    "d3_M128_m6_N2^20_spokes": (3, 128, 6, 1 << 20, 1, "spokes"),
    "d3_M128_m8_N2^20_spokes": (3, 128, 8, 1 << 20, 1, "spokes"),
}
DEFAULT_CONFIG = "d2_M256_m8_N2^20"
# FP32 flavour of the timed plan: the d = 3 workload is specified with
# compensated accumulation of the tap sums ("f32c"), the others plain FP32.
PRECISION = {"d3_M128_m6_N2^23_spokes": "f32c", "d3_M128_m8_N2^23_spokes": "f32c",
             "d3_M128_m6_N2^20_spokes": "f32c", "d3_M128_m8_N2^20_spokes": "f32c"}

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


# Nominal dense tensor rates of GB300, TF32 : BF16 (1.1 : 2.25 PFLOP/s); the
# TF32 peak is the measured BF16 GEMM rate times this ratio.
TF32_PER_BF16 = 1.1 / 2.25


def tensor_spread_roofline(x, M, m, seconds):
    """Tensor-pipe view of the d = 3 FP32 spreading launch (spread3t_kernel):
    the MMA flops it issues, per work item ceil(nodes / 8) stages of
    (M tiles) x 3 TF32 MMAs of 128 x NP x 8, with the binning's items (8^3
    tiles of L = 2M, at most 1024 nodes each), against the measured BF16
    peak times the nominal TF32/BF16 ratio.  These flops include the
    padding of the box to whole M tiles and the split-operand products, so
    the fraction says how busy the tensor pipe is, not how close the
    algorithm is to its bound (that is the FP32 roofline beside it)."""
    L, T, K = 2 * M, 8, 1024
    u = (np.float32(L) * x.astype(np.float32)).astype(np.float32)
    cell = np.floor(u).astype(np.int64) + L // 2
    tile = ((cell[:, 0] // T) * (L // T) + cell[:, 1] // T) * (L // T) + cell[:, 2] // T
    counts = np.bincount(tile)
    counts = counts[counts > 0]
    stages = int(((counts // K) * (K // 8)).sum() + ((counts % K + 7) // 8).sum())
    W = 2 * m
    R, B2 = T + W - 1, T + W
    NT = (R * B2 + 127) // 128
    NP = (2 * R + 15) // 16 * 16
    flops = float(stages) * NT * 3 * 128 * NP * 8 * 2
    peak = float(measured_peaks().get("bf16_tflops", 1900.0)) * TF32_PER_BF16
    achieved = flops / seconds / 1e12
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "mma_flops_per_launch": flops, "stages": stages,
            "peak_note": "measured bf16 GEMM burst x 1.1/2.25 (nominal TF32 : BF16), kind::tf32 MMAs"}


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


# FP32 FMA and special-function-unit (ex2, rsqrt, rcp) lane rates per SM, the
# peaks behind the short-sum kernels' ALU / SFU rooflines: each thread runs 8
# independent dependency chains of one instruction, the chains' results feed
# a checksum so that nothing is dead.  Measurement tooling of this script,
# not part of the library; compiled into the package's build folder.
_UNIT_RATES_CU = r"""
#include <cstdio>
#include <cuda_runtime.h>

template <int OP>
__global__ void chains(float* out, int iters) {
    float v[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = 1.0f + 1e-3f * static_cast<float>((threadIdx.x + c) & 63);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            float y;
            if (OP == 0) asm volatile("fma.rn.f32 %0, %1, 0f3F7FF972, 0f38D1B717;" : "=f"(y) : "f"(v[c]));
            if (OP == 1) asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(v[c]));
            if (OP == 2) asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(v[c]));
            if (OP == 3) asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(v[c]));
            v[c] = (OP == 1) ? y * 0.5f : (OP == 3) ? y + 1.0f : y;
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += v[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int OP>
static int run(const char* name, int sms, float* out, float* host) {
    const int blocks = sms * 8, threads = 256, iters = 4096;
    chains<OP><<<blocks, threads>>>(out, 16);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a);
    chains<OP><<<blocks, threads>>>(out, iters);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, a, b);
    if (cudaGetLastError() != cudaSuccess) return 1;
    cudaMemcpy(host, out, sizeof(float) * blocks * threads, cudaMemcpyDeviceToHost);
    double check = 0.0;
    for (int i = 0; i < blocks * threads; ++i) check += host[i];
    int clk_khz = 0;
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, 0);
    const double ops = static_cast<double>(blocks) * threads * iters * 8;
    const double per_clk = ops / (ms * 1e-3) / sms / (clk_khz * 1e3);
    printf("{\"op\": \"%s\", \"ms\": %.4f, \"lane_ops_per_clk_per_sm\": %.2f, \"clock_mhz\": %d, \"checksum\": %.6e}\n",
           name, ms, per_clk, clk_khz / 1000, check);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return 0;
}

int main() {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess) return 1;
    float* out = nullptr;
    const size_t n = static_cast<size_t>(sms) * 8 * 256;
    if (cudaMalloc(&out, sizeof(float) * n) != cudaSuccess) return 1;
    float* host = new float[n];
    int bad = 0;
    bad |= run<0>("ffma", sms, out, host);
    bad |= run<1>("ex2", sms, out, host);
    bad |= run<2>("rsqrt", sms, out, host);
    bad |= run<3>("rcp", sms, out, host);
    delete[] host;
    cudaFree(out);
    return (bad || cudaDeviceSynchronize() != cudaSuccess) ? 1 : 0;
}
"""


def run_unit_rates():
    """Build and run the unit-rate microbenchmark (FP32 FMA, ex2, rsqrt, rcp
    lane operations per SM per clock); prints one JSON line per unit."""
    bdir = os.path.join(ROOT, "paper_2502_07155_gb300", "_build")
    os.makedirs(bdir, exist_ok=True)
    src = os.path.join(bdir, "unit_rates.cu")
    exe = os.path.join(bdir, "unit_rates")
    with open(src, "w") as fh:
        fh.write(_UNIT_RATES_CU)
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

_ORACLE_STATE = {}


def _oracle_init(root, d, M, m, beta, fh):
    """Worker set-up (spawned process, no GPU): the oracle plan and its
    precorrection factors (step 0a, excluded from the timed steps)."""
    if root not in sys.path:
        sys.path.insert(0, root)
    import oracle as O
    p = O.make_plan(d, M, 2.0, m, beta=beta)
    _ORACLE_STATE.update(O=O, p=p, fac=O.precorrection_factors(p), fh=fh)


def _oracle_share(task):
    """One worker's share of an oracle step: the grid of steps 1-2 (direct
    DFT), the short sums at this share's nodes and the adjoint of this
    share's inputs (Psi^T, F^H, D)."""
    x, g = task
    st = _ORACLE_STATE
    O, p, fac = st["O"], st["p"], st["fac"]
    grid = O.grid_samples(p, st["fh"], fac)
    f = O.step3_short_sums(p, grid, x)
    h = O.adjoint(p, g, x, fac)
    return f, h


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OraclePool:
    """The FP64 oracle (forward + adjoint of Algorithm 4.2) on the host
    cores: one spawned worker per core, each computing the grid and the
    short sums and adjoint of its share of the sample's nodes; the adjoint is
    linear in its input, so the shares' adjoints add.  A step's time is the
    wall clock of the parallel section."""

    def __init__(self, d, M, m, beta, fh, procs=None):
        import multiprocessing
        self.procs = procs or min(32, host_cores())
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS",
                                                 "CUDA_VISIBLE_DEVICES")}
        os.environ.update(OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
        try:
            ctx = multiprocessing.get_context("spawn")
            self.pool = ctx.Pool(self.procs, initializer=_oracle_init, initargs=(ROOT, d, M, m, beta, fh))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def step(self, x, g):
        shares = [s for s in np.array_split(np.arange(x.shape[0]), self.procs) if s.size]
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_share, [(x[s], g[:, s]) for s in shares])
        t = time.perf_counter() - t0
        f = np.concatenate([r[0] for r in res], axis=1)
        h = res[0][1]
        for r in res[1:]:
            h = h + r[1]
        return f, h, t

    def close(self):
        self.pool.close()
        self.pool.join()


# Nodes per oracle step (both the reference arm and the GPU line's
# cpu_baseline): the first n nodes of the workload, with the full grid DFT.
ORACLE_SAMPLE = {2: 1 << 18, 3: 1 << 12, 1: 1024}


def oracle_sample_text(cfg, n, procs, steps, seconds):
    d, M, m, N, B, kind = CONFIGS[cfg]
    return (f"first {n} of the {N} nodes per step, full grid DFT (M={M}^{d}, L={2 * M}^{d}), forward + adjoint, "
            f"{procs} worker processes of one thread each ({steps} steps, {seconds:.1f} s)")


def workload_config(cfg, beta, world):
    """The `config` object of both arms' lines: what the workload is."""
    d, M, m, N, B, kind = CONFIGS[cfg]
    return {"workload": cfg, "d": d, "M": M, "sigma": 2.0, "L": 2 * M, "m": m, "N": N, "batch": B,
            "nodes": kind, "window": "sinh", "beta": beta, "precision": PRECISION.get(cfg, "f32"),
            "step": "forward + adjoint (nodes binned once)",
            "l2": "GPU: flushed (256 MiB write) before each timed step",
            "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"}


def default_beta(m):
    return float(np.pi * m * 0.5)   # pi m (1 - 1/sigma) at sigma = 2


# --------------------------------------------------------------------------- reference arm

def run_reference(args, cfg):
    """The oracle as the reference arm: each step is forward + adjoint of the
    oracle on a bounded sample of the workload's nodes (full grid DFT), on
    every host core."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return 0
    d, M, m, N, B, kind = CONFIGS[cfg]
    x, fh, g = make_inputs(cfg)
    n = min(ORACLE_SAMPLE[d], N)
    pool = OraclePool(d, M, m, default_beta(m), fh)
    times = []
    try:
        for i in range(args.warmup + args.steps):
            _, _, t = pool.step(x[:n], g[:, :n])
            if i >= args.warmup:
                times.append(t)
    finally:
        pool.close()
    t = float(np.mean(times))
    value = n / t
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(cfg, default_beta(m), world),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.procs, "kind": "oracle",
                            "sample": oracle_sample_text(cfg, n, pool.procs, args.steps, sum(times))},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


# --------------------------------------------------------------------------- our arm

def traffic_from_profiles(cfg, kernel):
    """DRAM bytes (read + write) per launch of `kernel` on workload `cfg`
    from the ncu summary profiles/traffic.md, whose rows name the source
    digest of the short-sum kernels they were captured with; None when no
    row matches the current source (the counters are stale)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.md")
    src = os.path.join(ROOT, "paper_2502_07155_gb300", "csrc", "taps.cuh")
    try:
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:12]
        rows = open(path).read().splitlines()
    except OSError:
        return None
    for line in rows:
        cells = [c.strip().strip("`") for c in line.strip().strip("|").split("|")]
        if len(cells) >= 4 and cells[0] == cfg and cells[1] == kernel and cells[3] == digest:
            try:
                return int(cells[2])
            except ValueError:
                return None
    return None


def ev_time(stream, fn, reps, flush=None):
    """Median device time (ms) of fn() over reps calls, CUDA events on
    `stream`, L2 flushed before each call."""
    import torch
    out = []
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        out.append(a.elapsed_time(b))
    return float(np.median(out))


def capture_graph(fn):
    """fn() captured once in a CUDA graph (after one eager warm-up on the
    capture stream)."""
    import torch
    stream = torch.cuda.current_stream()
    g_stream = torch.cuda.Stream()
    g_stream.wait_stream(stream)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(g_stream):
        fn()
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=g_stream):
            fn()
    torch.cuda.synchronize()
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    return graph


def cufft_comparison(nb, plan, fh_d, dev, stream, flush, reps=10):
    """The oversampled FFT of step 2 (Eq. 4.7) two ways: the library's
    pruned passes (forward direction, CUDA events around each pass) and
    cuFFT through torch.fft.ifftn on the zero-padded, precorrected L^d array
    (the whole transform, unpruned; building the array is not timed).  Both
    grids are compared."""
    import torch
    d = plan.d
    M, L = plan.M, plan.L
    plan.kernel_timing(True)
    for _ in range(reps):
        flush.zero_()
        plan.forward(fh_d)
    plan.sync()
    kt = plan.kernel_times()
    plan.kernel_timing(False)
    ours_ms = kt["fft"][0] / reps
    plan.forward(fh_d)
    ours_grid = plan.grid_tensor()[0].clone()
    theta = fh_d[0].to(torch.complex64)
    for t in range(d):
        fac = torch.from_numpy(plan.factors(t)).to(dev)
        shape = [1] * d
        shape[t] = M[t]
        theta = theta * fac.reshape(shape).to(torch.float32)
    pad = torch.zeros(tuple(L), dtype=torch.complex64, device=dev)
    sl = tuple(slice(L[t] // 2 - M[t] // 2, L[t] // 2 + M[t] // 2) for t in range(d))
    pad[sl] = theta
    src = torch.fft.ifftshift(pad)
    out = torch.fft.ifftn(src, norm="forward")
    cufft_ms = ev_time(stream, lambda: torch.fft.ifftn(src, norm="forward"), reps, flush)
    cu_grid = torch.fft.fftshift(out)
    err = float(torch.linalg.vector_norm((cu_grid - ours_grid).to(torch.complex128)) /
                torch.linalg.vector_norm(cu_grid.to(torch.complex128)))
    return {"ours_forward_passes_ms": ours_ms, "ours_passes": kt["fft"][1] // reps,
            "cufft_ifftn_ms": cufft_ms, "grid_rel_l2": err, "grid": f"{'x'.join(str(v) for v in L)} complex64",
            "note": "ours: pruned passes with the precorrection fused into the first load; cuFFT: full transform "
                    "of the zero-padded array (building it not timed)"}


def accuracy_vs_ndft(nb, d, M, m, x, f32_full, fh, dev, n_max=1 << 15):
    """Relative l2 error of the FP32 forward (computed at full size) and of
    the FP64 method on feasible sampled nodes against the trigonometric sums
    of Eq. 2.1, computed by the FP64 classical NFFT at m = 12 (m = 8 at
    d = 3), equal to the direct sums to about 1e-14."""
    import torch
    L = 2 * M
    feas = np.flatnonzero(W.feasible_mask(x, m, L))
    if feas.size == 0:
        return None
    rng = np.random.default_rng(7)
    idx = np.sort(rng.choice(feas, size=min(n_max, feas.size), replace=False))
    xs = torch.from_numpy(x[idx].astype(np.float64)).to(dev)
    fh64 = torch.from_numpy(fh.astype(np.complex128)).to(dev)
    m_ref = 12 if d < 3 else 8   # (FP64 d = 3 plans support m <= 8; the classical NFFT is ~1e-15 there)
    ref = nb.Plan(d, M, 2.0, m_ref, precision="f64", method="classic", batch=fh.shape[0])
    ref.set_nodes(xs)
    y = ref.forward(fh64)
    ref.close()
    p64 = nb.Plan(d, M, 2.0, m, precision="f64", batch=fh.shape[0])
    p64.set_nodes(xs)
    y64 = p64.forward(fh64)
    p64.close()
    idx_d = torch.from_numpy(idx).to(dev)
    got = f32_full[:, idx_d].to(torch.complex128)
    nrm = torch.linalg.vector_norm(y)
    return {"fp32_vs_ndft_rel_l2": float(torch.linalg.vector_norm(got - y) / nrm),
            "fp64_vs_ndft_rel_l2": float(torch.linalg.vector_norm(y64 - y) / nrm),
            "feasible_nodes_sampled": int(idx.size),
            "reference": f"FP64 classical NFFT, m = {m_ref} (the trigonometric sums of Eq. 2.1)"}


def measure(nb, cfg, args, dev, flush, full):
    """Every timing of one workload on one GPU.  `full` adds the legs only
    the headline line carries (classical NFFT, compensated FP32, end to end
    through the host-buffer calls)."""
    import torch
    d, M, m, N, B, kind = CONFIGS[cfg]
    x, fh, g = make_inputs(cfg)
    x_d = torch.from_numpy(x).to(dev)
    fh_d = torch.from_numpy(fh).to(dev)
    g_d = torch.from_numpy(g).to(dev)
    stream = torch.cuda.current_stream()
    prec = PRECISION.get(cfg, "f32")
    plan = nb.Plan(d, M, 2.0, m, precision=prec, batch=B)
    t0 = time.perf_counter()
    plan.set_nodes(x_d)
    t_set_first = time.perf_counter() - t0
    f_out = torch.empty((B, N), dtype=torch.complex64, device=dev)
    h_out = torch.empty((B,) + (M,) * d, dtype=torch.complex64, device=dev)

    def step():
        plan.forward(fh_d, out=f_out)
        plan.adjoint(g_d, out=h_out)

    for _ in range(args.warmup):
        step()
    plan.sync()
    set_ms = ev_time(stream, lambda: plan.set_nodes(x_d), 3, flush)

    # per-kernel device times (CUDA events around every launch), in a pass of their own
    plan.kernel_timing(True)
    for _ in range(args.steps):
        flush.zero_()
        step()
    plan.sync()
    ktimes = plan.kernel_times()
    plan.kernel_timing(False)

    graph = None if args.no_graph else capture_graph(step)

    def timed_steps(run, reps):
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
        for i in range(reps):
            flush.zero_()
            starts[i].record(stream)
            run()
            ends[i].record(stream)
        torch.cuda.synchronize()
        return float(np.mean([starts[i].elapsed_time(ends[i]) for i in range(reps)]))

    res = {"cfg": cfg, "N": N, "B": B, "d": d, "M": M, "m": m, "beta": plan.beta, "precision": prec}
    res["timed_region"] = {}
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    torch.cuda.synchronize()
    launches0 = plan.kernel_launches()
    res["t_stream"] = timed_steps(step, args.steps)
    res["launches"] = plan.kernel_launches() - launches0
    res["t_graph"] = timed_steps(graph.replay, args.steps) if graph is not None else None
    res["clocks"] = clocks.stop()
    plan.sync()
    res["t_step"] = res["t_graph"] if res["t_graph"] is not None else res["t_stream"]
    res["launch_mode"] = ("CUDA graph replay of the captured forward + adjoint calls" if graph is not None
                          else "stream launches")
    res["set_nodes_ms"] = set_ms
    res["set_nodes_first_call_s"] = t_set_first
    res["ktimes"] = ktimes
    reps_dir = max(3, args.steps // 2)
    res["fwd_ms"] = ev_time(stream, lambda: plan.forward(fh_d, out=f_out), reps_dir, flush)
    res["adj_ms"] = ev_time(stream, lambda: plan.adjoint(g_d, out=h_out), reps_dir, flush)
    gx = torch.empty((N, d), dtype=torch.float32, device=dev)
    res["grad_ms"] = ev_time(stream, lambda: plan.node_grad(fh_d, g_d, out=gx), 3, flush)
    f32 = plan.forward(fh_d, out=f_out).clone()
    plan.sync()

    # roofline of the dominant short-sum kernel
    dom = max(("interp", "spread"), key=lambda k: ktimes[k][0])
    dom_ms, dom_n = ktimes[dom]
    roofline = short_sum_roofline(d, m, N, B, M, dom_ms / max(dom_n, 1) * 1e-3)
    roofline["kernel"] = dom
    roofline["traffic"] = traffic_from_profiles(cfg, dom)
    res["roofline"] = roofline
    other = "spread" if dom == "interp" else "interp"
    o_ms, o_n = ktimes[other]
    res["roofline_other"] = dict(short_sum_roofline(d, m, N, B, M, o_ms / max(o_n, 1) * 1e-3), kernel=other,
                                 traffic=traffic_from_profiles(cfg, other))
    if d == 3 and B == 1 and 2 <= m <= 8 and PRECISION.get(cfg, "f32") in ("f32", "f32c"):
        sp = res["roofline"] if dom == "spread" else res["roofline_other"]
        sp["tensor"] = tensor_spread_roofline(x, M, m, ktimes["spread"][0] / max(ktimes["spread"][1], 1) * 1e-3)

    # plain FP64 GPU path on the same inputs, timed both ways
    plan64 = nb.Plan(d, M, 2.0, m, precision="f64", batch=B)
    x64 = torch.from_numpy(x.astype(np.float64)).to(dev)
    fh64 = torch.from_numpy(fh.astype(np.complex128)).to(dev)
    g64 = torch.from_numpy(g.astype(np.complex128)).to(dev)
    plan64.set_nodes(x64)
    f64o = torch.empty((B, N), dtype=torch.complex128, device=dev)
    h64o = torch.empty((B,) + (M,) * d, dtype=torch.complex128, device=dev)

    def step64():
        plan64.forward(fh64, out=f64o)
        plan64.adjoint(g64, out=h64o)

    step64()
    plan64.sync()
    reps64 = 2 if N * (2 * m) ** d > 5e9 else 3
    f64_stream = timed_steps(step64, reps64)
    f64_graph = None
    if graph is not None:
        graph64 = capture_graph(step64)
        f64_graph = timed_steps(graph64.replay, reps64)
        del graph64
    f64 = plan64.forward(fh64, out=f64o)
    plan64.sync()
    res["fp64"] = {"ms_per_step_graph": f64_graph, "ms_per_step_stream": f64_stream,
                   "nodes_per_s": N / ((f64_graph or f64_stream) * 1e-3),
                   "speedup_fp32_graph": (f64_graph / res["t_graph"]) if f64_graph else None,
                   "speedup_fp32_stream": f64_stream / res["t_stream"],
                   "basis": "FP32 and FP64 steps timed the same way: CUDA-graph replay against CUDA-graph replay, "
                            "stream launches against stream launches"}
    res["err_fp32_fp64"] = float(torch.linalg.vector_norm(f32.to(torch.complex128) - f64) /
                                 torch.linalg.vector_norm(f64))
    plan64.close()
    del x64, g64, h64o
    res["accuracy_ndft"] = accuracy_vs_ndft(nb, d, M, m, x, f32, fh, dev)
    res["fft_vs_cufft"] = cufft_comparison(nb, plan, fh_d, dev, stream, flush) if B == 1 else None

    if full:
        # classical NFFT (Algorithm 2.1) on the same inputs, FP32
        cplan = nb.Plan(d, M, 2.0, m, precision="f32", method="classic", batch=B)
        cplan.set_nodes(x_d)
        for _ in range(2):
            cplan.forward(fh_d, out=f_out)
            cplan.adjoint(g_d, out=h_out)
        res["cls_ms"] = ev_time(stream, lambda: (cplan.forward(fh_d, out=f_out), cplan.adjoint(g_d, out=h_out)), 3,
                                flush)
        cplan.sync()
        cplan.close()
        # FP32 with compensated (Neumaier) accumulation of the tap rows
        kplan = nb.Plan(d, M, 2.0, m, precision="f32c", batch=B)
        kplan.set_nodes(x_d)
        for _ in range(2):
            kplan.forward(fh_d, out=f_out)
            kplan.adjoint(g_d, out=h_out)
        res["comp_ms"] = ev_time(stream, lambda: (kplan.forward(fh_d, out=f_out), kplan.adjoint(g_d, out=h_out)),
                                 3, flush)
        f32c = kplan.forward(fh_d, out=f_out).clone()
        kplan.sync()
        kplan.close()
        res["err_fp32c_fp64"] = float(torch.linalg.vector_norm(f32c.to(torch.complex128) - f64) /
                                      torch.linalg.vector_norm(f64))
        # end to end through the host-buffer C-ABI calls: inputs uploaded from
        # page-locked host memory and both results downloaded inside the timed region
        fh_h = torch.from_numpy(fh).pin_memory()
        g_h = torch.from_numpy(g).pin_memory()
        f_h = torch.empty((B, N), dtype=torch.complex64).pin_memory()
        h_h = torch.empty((B,) + (M,) * d, dtype=torch.complex64).pin_memory()

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
        res["e2e_ms"] = float(np.mean(e2e_ms))
        res["e2e_wall_ms"] = float(np.mean(e2e_wall))
        res["h2d"] = fh_h.numel() * 8 + g_h.numel() * 8
        res["d2h"] = f_h.numel() * 8 + h_h.numel() * 8
    res["f32_host"] = f32.cpu().numpy()
    res["inputs"] = (x, fh, g)
    del f64, f64o
    plan.close()
    return res


def summary(res):
    """The per-workload object of the JSON line (without the inputs)."""
    N, B = res["N"], res["B"]
    out = {"workload": res["cfg"], "m": res["m"], "precision": res["precision"],
           "ms_per_step": res["t_step"], "nodes_per_s": N / (res["t_step"] * 1e-3),
           "stream_ms_per_step": res["t_stream"], "launch": res["launch_mode"],
           "forward_ms": res["fwd_ms"], "adjoint_ms": res["adj_ms"],
           "forward_nodes_per_s": N / (res["fwd_ms"] * 1e-3), "adjoint_nodes_per_s": N / (res["adj_ms"] * 1e-3),
           "set_nodes_ms": res["set_nodes_ms"], "node_grad_ms": res["grad_ms"],
           "roofline": res["roofline"], "roofline_other_kernel": res["roofline_other"],
           "fp64": res["fp64"], "fp32_vs_fp64_gpu_rel_l2": res["err_fp32_fp64"],
           "accuracy_vs_ndft": res["accuracy_ndft"], "fft_vs_cufft": res["fft_vs_cufft"],
           "kernels_in_timed_region": {k: {"ms_total": v[0], "launches": v[1]} for k, v in res["ktimes"].items()},
           "clocks": res["clocks"]}
    if B > 1:
        out["nodes_per_s_note"] = f"N nodes per step for each of {B} vectors"
    return out


def run_ours(args, cfg):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local_rank)
    # the oracle's worker pool is spawned (not forked) and started before any GPU work
    pool = None
    d, M, m, N, B, kind = CONFIGS[cfg]
    if rank == 0 and not args.quick:
        x0, fh0, g0 = make_inputs(cfg)
        pool = OraclePool(d, M, m, default_beta(m), fh0)
    if local_rank == 0:
        from paper_2502_07155_gb300 import build
        build.build()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
        dist.barrier()
    import paper_2502_07155_gb300 as nb

    dev = torch.device("cuda", local_rank)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    if world > 1:
        dist.barrier()
    res = measure(nb, cfg, args, dev, flush, full=not args.quick)
    if world > 1:
        dist.barrier()
    t_step, value = aggregate_over_ranks(res["t_step"], N, world, dev)
    if args.quick:
        if rank == 0:
            print(json.dumps({"quick": True, "config": cfg, "ms_per_step": t_step, "value": value, "unit": UNIT,
                              "gpu_launches": res["launches"], "clocks": res["clocks"],
                              "set_nodes_ms": res["set_nodes_ms"], "stream_ms_per_step": res["t_stream"],
                              "launch": res["launch_mode"], "forward_ms": res["fwd_ms"], "adjoint_ms": res["adj_ms"],
                              "node_grad_ms": res["grad_ms"],
                              "fp64": res["fp64"], "fp32_vs_fp64_gpu_rel_l2": res["err_fp32_fp64"],
                              "accuracy_vs_ndft": res["accuracy_ndft"], "fft_vs_cufft": res["fft_vs_cufft"],
                              "roofline": res["roofline"], "roofline_other_kernel": res["roofline_other"],
                              "kernels": {k: {"ms_total": v[0], "launches": v[1]}
                                          for k, v in res["ktimes"].items()}}))
        if world > 1:
            dist.destroy_process_group()
        return 0

    # the metric's d = 3 half: the spoke workload at m = 8 (the smallest m at
    # relative error <= 1e-6) and at m = 6 (its configured truncation)
    d3 = {}
    if cfg == DEFAULT_CONFIG and not args.no_d3:
        for c3 in ("d3_M128_m8_N2^23_spokes", "d3_M128_m6_N2^23_spokes"):
            r3 = measure(nb, c3, args, dev, flush, full=False)
            d3[c3] = summary(r3)
            del r3
            torch.cuda.empty_cache()

    result = None
    if rank == 0:
        # cpu baseline: the oracle on the host cores, same sample as the reference arm
        x, fh, g = res["inputs"]
        n = min(ORACLE_SAMPLE[d], N)
        reps = 3
        ts = []
        for _ in range(reps):
            f_or, h_or, t = pool.step(x[:n], g[:, :n])
            ts.append(t)
        pool.close()
        cpu_value = n / float(np.mean(ts))
        f32h = res["f32_host"]
        acc = {"fp32_vs_fp64_gpu_rel_l2": res["err_fp32_fp64"],
               "fp32_vs_oracle_rel_l2_sample": float(np.linalg.norm(f32h[:, :n] - f_or) / np.linalg.norm(f_or)),
               "oracle_sample_nodes": n}
        if res["accuracy_ndft"]:
            acc.update(res["accuracy_ndft"])
        s = summary(res)
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(cfg, res["beta"], world),
            "launch": res["launch_mode"], "stream_ms_per_step": res["t_stream"],
            "e2e": {"value": world * N / (res["e2e_ms"] * 1e-3), "unit": UNIT, "h2d_bytes_per_step": res["h2d"],
                    "d2h_bytes_per_step": res["d2h"], "ms_per_step": res["e2e_ms"],
                    "host_wall_ms_per_step": res["e2e_wall_ms"],
                    "api": "nfftbl_forward_host + nfftbl_adjoint_host + nfftbl_join (page-locked host buffers)"},
            "gpu_launches": res["launches"],
            "roofline": res["roofline"],
            "roofline_other_kernel": res["roofline_other"],
            "cpu_baseline": {"value": cpu_value, "unit": UNIT, "cores": pool.procs, "kind": "oracle",
                             "sample": oracle_sample_text(cfg, n, pool.procs, reps, sum(ts))},
            "clocks": res["clocks"],
            "forward_nodes_per_s": s["forward_nodes_per_s"], "adjoint_nodes_per_s": s["adjoint_nodes_per_s"],
            "breakdown_ms": {"forward": res["fwd_ms"], "adjoint": res["adj_ms"], "set_nodes": res["set_nodes_ms"],
                             "set_nodes_first_call_s": res["set_nodes_first_call_s"], "node_grad": res["grad_ms"],
                             "kernels_in_timed_region": s["kernels_in_timed_region"]},
            "fp64": res["fp64"],
            "classic_nfft_fp32": {"ms_per_step": res["cls_ms"], "nodes_per_s": N / (res["cls_ms"] * 1e-3)},
            "fp32_compensated": {"ms_per_step": res["comp_ms"], "nodes_per_s": N / (res["comp_ms"] * 1e-3),
                                 "fp32c_vs_fp64_gpu_rel_l2": res["err_fp32c_fp64"]},
            "accuracy": acc,
            "fft_vs_cufft": res["fft_vs_cufft"],
            "d3": d3,
        }
        print(json.dumps(result))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
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
    # equal error: the smallest measured m of each window whose held-out error
    # is <= 1e-6, with its forward time (held-out nodes are feasible for m + 2
    # of the trained m, so the sinh entries of different rows differ slightly)
    def smallest(entries):
        ok = sorted((mm, e, t) for mm, e, t in entries if e <= 1e-6)
        return {"m": ok[0][0], "err": ok[0][1], "fwd_ms": ok[0][2]} if ok else None
    eq = {"learned": smallest([(r["m"], r["learned_err"], r["learned_fwd_ms"]) for r in results]),
          "sinh": smallest([(mm, v["err"], v["fwd_ms"]) for r in results for mm, v in r["sinh"].items()])}
    out = {"metric": "learned window vs sinh window: held-out relative l2 error against the trigonometric sum",
           "config": {"workload": "learned_window_d2_M256_sigma2", "train_nodes": 1 << 16, "heldout_nodes": 1 << 22,
                      "targets": "FP64 classical NFFT m=12", "mlp": "1-64-64-1 tanh, BF16 backward",
                      "table_len": 4097, "trained_m": list(args.learned_m)},
           "results": results, "equal_error_1e-6": eq, "data": "synthetic", "n_gpus": 1}
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
                    help="one workload without the classical, compensated, end-to-end and oracle legs")
    ap.add_argument("--no-d3", action="store_true", dest="no_d3",
                    help="leave the d = 3 workloads out of the default line")
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
