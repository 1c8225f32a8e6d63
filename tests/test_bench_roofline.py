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
