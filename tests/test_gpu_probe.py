"""The FP32 FMA throughput probe (a measurement aid): its rate lies near the
FP32 peak implied by the SM count, the FMA lanes and the clock, and bad
arguments are refused without a launch."""
import pytest

from tests.test_gpu_parity import _gpu

pytestmark = pytest.mark.gpu


def test_probe_rate_is_near_the_fp32_peak():
    _gpu()
    from paper_2602_15883_b300 import binding
    ms, flop = binding.probe_fp32(4000)
    tflops = flop / (ms * 1e-3) / 1e12
    nominal = 148 * 128 * 2 * 2.032e9 / 1e12        # 77.0 TFLOP/s at the maximum SM clock
    assert 0.5 * nominal <= tflops <= 1.05 * nominal, tflops


def test_probe_rejects_bad_arguments():
    _gpu()
    from paper_2602_15883_b300 import binding
    for bps, iters in ((0, 10), (9, 10), (4, 0)):
        with pytest.raises(binding.DpinnError):
            binding.probe_fp32(iters, blocks_per_sm=bps)
