"""The FP64 throughput measurement that gives the roofline its denominator: a plausible rate for a
GPU whose FP64 pipe issues about two fused multiply-adds per SM per cycle, and a stable one."""
import pytest

pytestmark = pytest.mark.gpu


def test_fp64_peak_measurement():
    import torch
    import paper_2208_01260_gb300 as hw
    assert torch.cuda.is_available()
    best, median, ms = hw.hw_measure_fp64_peak(5)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    # between a quarter and four times 2 fma per SM per cycle at 1-2.1 GHz
    assert 0.25 * 2 * sms * 1.0e9 <= best <= 4 * 2 * sms * 2.1e9, best
    assert median <= best and median >= 0.8 * best and ms > 1.0
    with pytest.raises(hw.HwError):
        hw.hw_measure_fp64_peak(0)
