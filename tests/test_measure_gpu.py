"""The measured FP32 SIMT peak (lbf_measure_fp32_peak), the denominator of the FP32 kernels'
roofline: positive, and below what the SMs' FMA lanes can deliver at the highest clock."""

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_fp32_peak_is_physical():
    from paper_1105_0661_gb300 import build_lib
    build_lib.build()
    from paper_1105_0661_gb300 import lbf
    torch.cuda.set_device(0)
    r = lbf.measure_fp32_peak(3)
    # 128 FP32 lanes per SM, 2 flop per FMA, at most ~2.1 GHz; packed FP32x2 at most twice that
    lane_bound = r["sms"] * 128 * 2 * 2.2e9 / 1e12
    print(f"FP32 peak: FFMA {r['ffma_tflops']:.1f}, FP32x2 {r['ffma2_tflops']:.1f} TFLOP/s on {r['sms']} SMs")
    assert r["sms"] > 0
    assert 0.2 * lane_bound < r["ffma_tflops"] <= lane_bound
    assert 0.2 * lane_bound < r["ffma2_tflops"] <= 2 * lane_bound
