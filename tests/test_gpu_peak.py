"""The FMA-rate measurement aid (neno6_pipe_peak) behind the roofline figures:
both pipes give a finite rate, FP32 well above FP64 (GB300 runs FP64 at a
small fraction of its FP32 rate), and FP64 not above its nominal ceiling
(2 DFMA per clock per SM at the maximum clock, with 10 % slack)."""
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_pipe_peaks():
    import paper_2207_08500_gb300 as p
    from paper_2207_08500_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    f64 = p.pipe_peak("fp64")
    f32 = p.pipe_peak("fp32")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    print("FMA rates: fp64 %.3f TFLOP/s, fp32 %.1f TFLOP/s" % (f64 / 1e12, f32 / 1e12))
    assert 0 < f64 <= 1.1 * 2 * 2 * sms * 2.07e9
    assert f32 > 10 * f64
