"""The benchmark's roofline arithmetic (host logic, no GPU): the tensor-core shape is held to the
lower of its tensor bound (measured sustained bf16 rate over 8 flop per pair) and its one-compare
epilogue bound (SMs x 128 FP32 lanes x the sampled clock), the float32 shapes to SMs x 128 lanes x
clock over 4 lane operations per pair; frac = achieved / peak."""
import math

import pytest

import bench


@pytest.fixture
def peaks(monkeypatch):
    monkeypatch.setattr(bench, "measured_peaks", lambda: {"bf16_tflops_sustained": 1694.0, "hbm_gbs": 6728.7})


def _ms(match_ms, exact_ms=0.0):
    # per-kind device time of a step: match, collide, collide_nn, finalize, stein, exact
    return [match_ms, 5.0, 8.0, 3.0, 1.4, exact_ms]


def test_tensor_core_roofline_is_the_epilogue_bound(peaks):
    pairs = 3 * 256 * 2048 * 8192
    r = bench.roofline_entry(True, pairs, 0.6963e-3, 0.0861e-3, _ms(70.3, 8.7), 152, {"sm_mhz": 2070.0})
    epi = 152 * 128 * 2070e6
    tensor = 1694.0e12 / 8
    assert r["bound"] == "alu" and r["unit"] == "Gpairs/s"
    assert math.isclose(r["peak"], min(epi, tensor) / 1e9, rel_tol=1e-12)
    assert math.isclose(r["achieved"], pairs / 0.6963e-3 / 1e9, rel_tol=1e-12)
    assert math.isclose(r["frac"], r["achieved"] / r["peak"], rel_tol=1e-12)
    assert 0.45 < r["frac"] < 0.47
    assert math.isclose(r["frac_of_tensor_bound"], pairs / 0.6963e-3 / tensor, rel_tol=1e-12)
    assert math.isclose(r["executed_mma_tflops"], pairs / 0.6963e-3 * 32 / 1e12, rel_tol=1e-12)
    assert math.isclose(r["matching_pairs_per_s"], pairs / (0.6963e-3 + 0.0861e-3), rel_tol=1e-12)
    assert math.isclose(r["kernel_share"], 70.3 / sum(_ms(70.3, 8.7)), rel_tol=1e-12)


def test_tensor_bound_wins_when_the_clock_is_high(peaks):
    # a clock at which the one-compare epilogue would outrun the tensor pipe: the tensor bound rules
    sms, mhz = 152, 20000.0
    r = bench.roofline_entry(True, 1e10, 1e-3, 1e-4, _ms(1.0, 0.1), sms, {"sm_mhz": mhz})
    assert r["bound"] == "tensor"
    assert math.isclose(r["peak"], 1694.0e12 / 8 / 1e9, rel_tol=1e-12)


def test_float32_roofline_counts_four_lane_operations_per_pair(peaks):
    pairs = 3 * 256 * 2048 * 8192
    r = bench.roofline_entry(False, pairs, 1.70e-3, 0.0, _ms(170.0), 148, {"sm_mhz": 1900.0})
    lanes = 148 * 128 * 1900e6
    assert r["bound"] == "alu" and r["kernel"] == "fwd_match_kernel"
    assert math.isclose(r["peak"], lanes / 4 / 1e9, rel_tol=1e-12)
    assert math.isclose(r["frac"], pairs / 1.70e-3 / (lanes / 4), rel_tol=1e-12)
    assert math.isclose(r["frac_fma_pipe"], pairs / 1.70e-3 / (lanes / 3), rel_tol=1e-12)


def test_nominal_clock_without_samples(peaks):
    r = bench.roofline_entry(True, 1e10, 1e-3, 0.0, _ms(1.0), 152, {"sm_mhz": None})
    assert math.isclose(r["sm_mhz"], bench.SM_MAX_MHZ_NOMINAL)
    assert "nominal" in r["peak_basis"]
