"""The FMA throughput probe that gives the FP32 path's roofline its arithmetic peak.

Physical bounds: 128 FP32 lanes per SM, one fused multiply-add (2 flops) per lane per clock, so the
measured FP32 rate cannot exceed SMs x 128 x 2 x the maximum SM clock; it must reach a large part of
it (the probe issues nothing but independent FMAs).  The FP64 rate is positive and far below FP32.
"""
import pytest
import torch

from paper_2202_04486_gb300 import binding, build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    build.build()
    binding.load_library()


def test_flop_count_and_sink():
    sink = torch.full((3 * 256,), float("nan"), device="cuda")
    fl = binding.mdc_alu_probe(0, 3, 32, sink)
    torch.cuda.synchronize()
    assert fl == 2.0 * 3 * 256 * 8 * 32
    assert torch.isfinite(sink).all()


def test_fp32_peak_within_physical_bounds():
    props = torch.cuda.get_device_properties(0)
    # upper bound at 2.2 GHz: above any SM clock this part runs at
    ceiling = props.multi_processor_count * 128 * 2 * 2.2e9 / 1e12
    t32 = binding.alu_peak_tflops(0)
    t64 = binding.alu_peak_tflops(1)
    assert 0.3 * ceiling < t32 <= ceiling, (t32, ceiling)
    assert 0.0 < t64 < t32, (t64, t32)
