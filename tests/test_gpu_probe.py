"""The FP32 FMA throughput probe behind the ALU roofline."""
import pytest

pytestmark = pytest.mark.gpu


def test_fp32_peak_probe_is_plausible(tg):
    """GB300: 152 SMs x 128 FP32 lanes x 2 FLOP x about 2 GHz, 80 TFLOP/s nominal; the probe must land near it
    and agree with itself."""
    a, b = tg.tg_measure_fp32_peak(), tg.tg_measure_fp32_peak()
    assert 20.0 < a < 200.0, a
    assert abs(a - b) <= 0.1 * max(a, b), (a, b)
