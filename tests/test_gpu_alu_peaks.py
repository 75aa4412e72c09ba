"""The measured FMA throughput the benchmark reports its FP64-bound kernels against (mg_alu_peaks): FP64 and scalar
FP32 rates of the device, each from one timed launch of independent FMA chains.  The values must be plausible for
the part (GB300: FP64 issues about two FMAs per SM and clock, FP32 128 lanes per SM) and FP32 well above FP64."""
import pytest

pytestmark = pytest.mark.gpu


def test_alu_peaks_are_plausible_and_repeatable():
    from paper_2403_08063_gb300 import alu_peaks
    a64, a32 = alu_peaks()
    b64, b32 = alu_peaks()
    print(f"FMA throughput: FP64 {a64:.3f} / {b64:.3f} TFLOP/s, FP32 {a32:.1f} / {b32:.1f} TFLOP/s")
    assert 0.3 < a64 < 10.0 and 10.0 < a32 < 300.0
    assert a32 > 10.0 * a64
    assert abs(a64 - b64) <= 0.1 * a64 and abs(a32 - b32) <= 0.1 * a32
