"""The measured FP64 ceiling (hweno_measure_fp64_peak): a DFMA-only loop
lands between half and 1.1 times the nominal rate (152 SMs x 2 DFMA per clock
x 2 flops at up to 2.07 GHz = 1.26 TFLOP/s)."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hw():
    from paper_2207_05258_gb300 import build
    build.build()
    from paper_2207_05258_gb300 import hweno
    return hweno


def test_fp64_loop_rate_is_plausible(hw):
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nominal = sms * 2 * 2 * 2.07e9 / 1e12
    r = hw.measure_fp64_peak()
    assert 0.5 * nominal < r < 1.1 * nominal, (r, nominal)
