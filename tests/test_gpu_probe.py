"""rsi_fp32_peak, the FP32 ceiling the benchmark compares the traversal's
arithmetic with: the measured rate must be plausible for the device (well
above zero, not above its FP32 units at the maximum clock)."""
import pytest
import torch

import paper_2209_02878_gb300 as rsi

pytestmark = pytest.mark.gpu


def test_fp32_peak_is_plausible():
    props = torch.cuda.get_device_properties(0)
    # 128 FP32 lanes per SM, 2 flops per FMA, at most 2.2 GHz
    ceiling = props.multi_processor_count * 128 * 2 * 2.2e9 / 1e12
    v = rsi.fp32_peak(1 << 16)
    assert 0.2 * ceiling < v <= ceiling, (v, ceiling)
    # the rate does not depend on the length of the run
    v2 = rsi.fp32_peak(1 << 17)
    assert abs(v2 - v) <= 0.15 * v, (v, v2)
