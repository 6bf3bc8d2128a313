"""gc_fma_peak, the measured FMA throughput the push kernels' rooflines divide by: the FP32
rate lies between 60 % and 105 % of the unit-count peak at the maximum SM clock (152 SMs x 128
lanes x 2 flop x 2.07 GHz = 80.5 TFLOP/s), the FP64 rate near the GPU's nominal FP64 rate and
far below the FP32 one, and a bad device is refused."""
import pytest

pytestmark = pytest.mark.gpu
gcpush = pytest.importorskip("paper_2403_06706_gb300.gcpush")


def test_fma_peak_is_plausible():
    f32, f64 = gcpush.fma_peak(0)
    print(f"FP32 {f32:.1f} TFLOP/s, FP64 {f64:.3f} TFLOP/s")
    derived = 152 * 128 * 2 * 2.07e9 / 1e12
    assert 0.6 * derived < f32 < 1.05 * derived
    assert 0.3 < f64 < 5.0
    assert f32 > 16 * f64
    with pytest.raises(gcpush.GcError):
        gcpush.fma_peak(999)
