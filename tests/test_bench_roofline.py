"""The roofline arithmetic of bench.py (host logic, no GPU): algorithmic
counts per launch of a short-sum kernel and the choice of the binding unit.

Per node and batch entry: 5 (2m)^d FP32 flops (a complex-times-real tap is
two FMAs, the tensor-product weight one multiply); per node: 3 d 2m SFU slots
(one sinh-window weight per tap and dimension at three slots); HBM: (4d + 8)
bytes per node and batch entry plus one pass over the 8-byte L^d grid."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

bench = pytest.importorskip("bench")


def test_counts_and_sfu_bound_at_d2_m8():
    N, M = 1 << 20, 256
    r = bench.short_sum_roofline(2, 8, N, 1, M, 144.4e-6)
    assert r["flops_per_launch"] == 5 * 16 ** 2 * N
    assert r["sfu_slots_per_launch"] == 3 * 2 * 16 * N
    assert r["hbm_bytes_per_launch"] == (4 * 2 + 8) * N + 8 * (2 * M) ** 2
    f = bench.SM_MAX_MHZ * 1e6
    sfu_peak = bench.SMS * bench.SFU_SLOTS * f
    fp32_peak = bench.SMS * bench.FP32_LANES * 2 * f
    assert r["t_bound_us"]["sfu"] == pytest.approx(3 * 2 * 16 * N / sfu_peak * 1e6)
    assert r["t_bound_us"]["fp32"] == pytest.approx(5 * 256 * N / fp32_peak * 1e6)
    # at m = 8 the weights' SFU slots bound the kernel, not its FMAs or HBM
    assert r["bound_unit"] == "sfu" and r["bound"] == "alu"
    assert r["frac"] == pytest.approx(r["t_bound_us"]["sfu"] * 1e-6 / 144.4e-6)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])


def test_fp32_bound_at_d3_and_batch_scaling():
    N = 1 << 23
    r1 = bench.short_sum_roofline(3, 6, N, 1, 128, 11.9e-3)
    assert r1["bound_unit"] == "fp32"
    assert r1["flops_per_launch"] == 5 * 12 ** 3 * N
    # a batch multiplies the flops and the node bytes, not the weights
    r8 = bench.short_sum_roofline(3, 6, N, 8, 128, 11.9e-3)
    assert r8["flops_per_launch"] == 8 * r1["flops_per_launch"]
    assert r8["sfu_slots_per_launch"] == r1["sfu_slots_per_launch"]


def test_hbm_bound_when_the_grid_dominates():
    # few nodes on a large grid: one pass over the grid outweighs the taps
    r = bench.short_sum_roofline(1, 2, 1 << 10, 1, 1 << 22, 1e-3)
    assert r["bound_unit"] == "hbm" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert max(r["t_bound_us"], key=r["t_bound_us"].get) == "hbm"


def test_tensor_spreading_stage_count_by_direct_binning():
    """The tensor-pipe figure of the d = 3 spreading counts its stages: per
    work item (8^3-cell tile of L = 2M, at most 1024 nodes) ceil(nodes / 8)
    stages, each (M tiles) x 3 TF32 MMAs of 128 x N_P x 8.  Checked against
    the tiles and items counted one node at a time."""
    import numpy as np
    rng = np.random.default_rng(4)
    M, m = 32, 8
    L = 2 * M
    x = rng.uniform(-0.5, 0.5, size=(6000, 3)).astype(np.float32)
    x[:2500] = np.float32(0.01)                                        # one tile of 2500 nodes: 3 items
    per_tile = {}
    for p in x:
        cell = [int(np.floor(np.float32(L) * p[t])) + L // 2 for t in range(3)]
        key = tuple(c // 8 for c in cell)
        per_tile[key] = per_tile.get(key, 0) + 1
    stages = 0
    for n in per_tile.values():
        while n > 0:
            k = min(n, 1024)
            stages += (k + 7) // 8
            n -= k
    r = bench.tensor_spread_roofline(x, M, m, 1e-3)
    assert r["stages"] == stages
    W = 2 * m
    R, B2 = 8 + W - 1, 8 + W
    NT, NP = (R * B2 + 127) // 128, (2 * R + 15) // 16 * 16
    assert (NT, NP) == (5, 48)
    assert r["mma_flops_per_launch"] == stages * NT * 3 * 128 * NP * 8 * 2
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])


def test_traffic_rows_follow_the_source_digest(tmp_path, monkeypatch):
    """A traffic row is reported only while its digest matches the current
    short-sum kernel source; any change to the source makes the key null."""
    import hashlib
    src = tmp_path / "paper_2502_07155_gb300" / "csrc"
    src.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (src / "taps.cuh").write_bytes(b"// kernels\n")
    dig = hashlib.sha256(b"// kernels\n").hexdigest()[:12]
    (tmp_path / "profiles" / "traffic.md").write_text(
        "| workload | kernel | bytes | digest |\n|---|---|---|---|\n"
        f"| d2_M256_m8_N2^20 | spread | 123 | {dig} |\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_from_profiles("d2_M256_m8_N2^20", "spread") == 123
    assert bench.traffic_from_profiles("d2_M256_m8_N2^20", "interp") is None
    (src / "taps.cuh").write_bytes(b"// kernels, changed\n")
    assert bench.traffic_from_profiles("d2_M256_m8_N2^20", "spread") is None
