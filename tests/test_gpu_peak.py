"""lb_measure_fp32_peak: the measured FP32 FMA throughput is consistent with
the device's own shape, each SM issuing at most one warp-instruction per
scheduler (four per SM) and cycle at the clock the kernel saw, and reaching
most of that with independent chains."""
import pytest

pytestmark = pytest.mark.gpu


def test_fma_peak_is_bounded_by_the_issue_rate():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_01126_gb300 import build

    build.build()
    from paper_2505_01126_gb300 import lbgb

    p = lbgb.measure_fp32_peak()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert 500.0 < p["sm_mhz"] < 3000.0
    issue_max = sms * 4 * p["sm_mhz"] * 1e6
    assert p["warp_inst_per_s"] <= 1.02 * issue_max
    assert p["warp_inst_per_s"] >= 0.8 * issue_max
    assert p["fp32_flops"] == pytest.approx(64 * p["warp_inst_per_s"], rel=1e-12)
    # packed two-lane FMAs: at least the scalar FLOP rate from half the instructions
    assert p["fp32_flops_paired"] == pytest.approx(128 * p["paired_warp_inst_per_s"], rel=1e-12)
    assert p["paired_warp_inst_per_s"] <= 1.02 * issue_max
    assert p["fp32_flops_paired"] >= 0.8 * p["fp32_flops"]
