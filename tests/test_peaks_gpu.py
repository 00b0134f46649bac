"""vrs_measure_peaks: the measured throughputs that serve as roofline denominators are
plausible for the device (no microbenchmark was optimised away, none is off by a unit)."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def peaks():
    from paper_2505_10144_gb300 import build
    build.build()
    from paper_2505_10144_gb300 import api
    return api.measure_peaks()


def test_device_attributes(peaks):
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    assert peaks["sm_count"] == props.multi_processor_count
    assert peaks["l2_bytes"] == props.L2_cache_size
    assert 500_000 < peaks["max_sm_clock_khz"] < 4_000_000


def test_fp32_fma_rate_is_bounded_by_the_lanes(peaks):
    # 128 FP32 lanes per SM, 2 flop per FMA, at most the maximum clock
    nominal = peaks["sm_count"] * 128 * 2 * peaks["max_sm_clock_khz"] * 1e3 / 1e12
    assert 0.5 * nominal < peaks["fp32_tflops"] <= 1.02 * nominal


def test_rates_are_ordered(peaks):
    fma_gops = peaks["fp32_tflops"] / 2 * 1e3
    assert fma_gops / 64 < peaks["exp2_gops"] < fma_gops
    assert fma_gops / 8 < peaks["logic_gops"] <= 1.02 * fma_gops
    assert peaks["l2_read_gbs"] > peaks["dram_read_gbs"] > 1000.0
