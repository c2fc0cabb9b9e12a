"""Unit-peak microbenchmarks (npm_measure_unit_peaks): the measured rates
are finite and within an order of magnitude of the GB300's unit counts
(152 SMs; 128 FP32 lanes and 16 MUFU lanes per SM at ~2 GHz)."""
import math

import pytest

pytestmark = pytest.mark.gpu


def test_unit_peaks_plausible():
    import paper_2504_04315_gb300 as npm
    p = npm.measure_unit_peaks()
    for k, v in p.items():
        assert math.isfinite(v) and v > 0, (k, v)
    nominal_fma = p["sm_count"] * 128 * 2 * p["max_sm_clock_mhz"] * 1e6 / 1e12
    nominal_mufu = p["sm_count"] * 16 * p["max_sm_clock_mhz"] * 1e6 / 1e9
    assert 0.3 * nominal_fma < p["fp32_fma_tflops"] < 1.5 * nominal_fma, p
    assert 0.1 * nominal_mufu < p["mufu_gops"] < 4.0 * nominal_mufu, p
    assert 500 < p["l2_sector_read_gbs"] < 100000, p
    assert 1 < p["l2_atomic_gops"] < 10000 and 1 < p["l2_atomic_v2_gops"] < 10000, p
