"""The benchmark's roofline arithmetic on CPU: the algorithmic work per unit
it divides by, and the bound it picks, against hand-computed values."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402
import synth  # noqa: E402


def test_mlp_flops_per_query():
    # 2 * sum of layer products: 32-64-64-64-32 -> 24,576; 4-32-32-16 -> 3,328.
    assert bench.mlp_flops(synth.PAPER_HASH) == 2 * (32 * 64 + 64 * 64 + 64 * 64 + 64 * 32) == 24576
    assert bench.mlp_flops(synth.TINY_BF16) == 2 * (4 * 32 + 32 * 32 + 32 * 16) == 3328


def test_tc_roofline_picks_the_smallest_bound():
    pk = {"hbm_gbs": 8000.0, "bf16_tflops": 2000.0}
    up = {"mufu_gops": 10000.0}
    r = bench.tc_roofline(10e9, synth.TINY_BF16, pk, up, sms=152, sm_mhz=2000.0)
    expect = {"hbm": 8000e9 / 40, "tensor": 2000e12 / 3328, "mufu": 10000e9 / 63,
              "fp32_lanes": 152 * 128 * 2000e6 / 300}
    for k, v in expect.items():
        assert r["bounds"][k] == pytest.approx(v)
    assert r["limiting_unit"] == "fp32_lanes" and r["bound"] == "alu"
    assert r["frac"] == pytest.approx(10e9 / expect["fp32_lanes"])


def test_train_roofline_adds_adam_and_scatter_time():
    w = synth.PRODUCT_BF16
    pk = {"hbm_gbs": 7000.0}
    up = {"l2_atomic_v2_gops": 200.0, "l2_atomic_v4_gops": 180.0}
    n_params = 10_000_000
    # Upper bound: every corner one two-wide atomic.
    r = bench.train_roofline(5e8, w, n_params, pk, up)
    step = 34.0 * n_params / 7000e9 + w.n_train * len(w.level_res) * 8 / 200e9
    assert r["peak"] == pytest.approx(w.n_train / step)
    assert r["frac"] == pytest.approx(5e8 * step / w.n_train)
    assert r["atomics_per_step"]["per_sample"] == 128
    # Counted operations: four-wide at their own rate.
    n4, n2 = 3_000_000, 40_000_000
    r = bench.train_roofline(5e8, w, n_params, pk, up, (n4, n2))
    step = 34.0 * n_params / 7000e9 + n4 / 180e9 + n2 / 200e9
    assert r["peak"] == pytest.approx(w.n_train / step)
    assert r["bound_ms"]["scatter_l2_atomics"] == pytest.approx((n4 / 180e9 + n2 / 200e9) * 1e3)


def test_serving_roofline_sums_queries_compaction_and_training():
    w = synth.TINY_BF16
    pk = {"hbm_gbs": 8000.0, "bf16_tflops": 2000.0}
    up = {"mufu_gops": 10000.0}
    sv = {"queries": 64 * 6_500_000, "frame_ms_mean": 0.7}
    r = bench.serving_roofline(sv, w, 64, pk, up, sms=152, sm_mhz=2000.0, train_bound_s=20e-6)
    q_s = 6_500_000 / (152 * 128 * 2000e6 / 300)
    c_s = 8 * 6_500_000 / 8000e9
    assert r["bound_ms_per_frame"] == pytest.approx((q_s + c_s + 20e-6) * 1e3)
    assert r["frac"] == pytest.approx((q_s + c_s + 20e-6) / 0.7e-3)


class _FakeIdx:
    """Stands in for a model: grid_indices returns fixed corner indices."""

    def __init__(self, idx):
        self.idx = idx

    def grid_indices(self, pos):
        import torch
        return torch.as_tensor(self.idx)


def test_gather_sector_counts_by_hand():
    torch = pytest.importorskip("torch")
    w = synth.PAPER_HASH  # two FP32 features: 8-byte entries, four to a sector
    L = len(w.level_res)
    offs = np.cumsum([0] + synth.grid_sizes(w)[:-1])
    idx = np.zeros((L, 8, 2), np.int64)
    # Query 0: every level's corners are entries 0..7 (two sectors when the
    # level starts on a sector boundary). Query 1: eight corners 64 entries
    # apart (eight sectors).
    idx[:, :, 0] = np.arange(8)[None, :]
    idx[:, :, 1] = 64 * np.arange(8)[None, :]
    expect = 0
    for l in range(L):
        s0 = {((offs[l] + e) * 8) // 32 for e in range(8)}
        expect += len(s0) + 8
    got = bench.gather_sector_counts(_FakeIdx(idx), w, torch.zeros((3, 2)))
    assert got == expect


def test_gather_roofline_arithmetic():
    r = bench.gather_roofline(2e9, 96.0, {"l2_sector_read_gbs": 9600.0})
    assert r["peak"] == pytest.approx(9600e9 / (32 * 96.0))
    assert r["frac"] == pytest.approx(2e9 / r["peak"])
