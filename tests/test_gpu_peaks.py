"""The measured arithmetic peaks (pat_measure_peaks) against the unit counts
and clocks of the device: each measured rate lies between 60 % and 105 % of
units x lanes x clock for FP32 (128 lanes per SM, 2 flops per FMA); FP64 and
the special-function unit, whose unit counts differ between parts, only get
order-of-magnitude bounds below FP32."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_measured_peaks():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_29253_gb300 import _lib

    pk = _lib.pat_measure_peaks()
    props = torch.cuda.get_device_properties(0)
    nsm = props.multi_processor_count
    # the maximum SM clock in kHz, as the driver reports it
    clk_hz = getattr(props, "clock_rate", 0) * 1e3 or 2.07e9
    fp32_nominal = nsm * 128 * 2 * clk_hz
    print({k: f"{v:.4g}" for k, v in pk.items()}, f"nominal FP32 {fp32_nominal:.4g}")
    assert 0.6 * fp32_nominal <= pk["fp32_ffma_flops"] <= 1.05 * fp32_nominal
    assert 0.6 * fp32_nominal <= pk["fp32_ffma2_flops"] <= 2.1 * fp32_nominal
    assert 1e11 <= pk["fp64_dfma_flops"] <= pk["fp32_ffma_flops"]
    assert 1e11 <= pk["sfu_rsqrt_ops"] <= pk["fp32_ffma_flops"]
