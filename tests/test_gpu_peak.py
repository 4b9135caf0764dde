"""The measured FP32 FMA throughput used as the FP32 form's roofline peak:
positive, repeatable, and within the range of the GPU's unit counts."""

import pytest
import torch

pytestmark = pytest.mark.gpu


def test_fp32_fma_peak_is_plausible(nsdf_lib):
    import paper_2110_01614_gb300 as nsdf
    a = nsdf.nsdf_debug_fp32_fma_peak()
    b = nsdf.nsdf_debug_fp32_fma_peak()
    props = torch.cuda.get_device_properties(0)
    # 128 FP32 lanes per SM, 2 FLOP per FMA, at most ~2.2 GHz
    bound = props.multi_processor_count * 128 * 2 * 2.2e9 / 1e12
    assert 0.3 * bound < a <= 1.05 * bound, (a, bound)
    assert abs(a - b) / a < 0.1
