"""Measured multiply-add peaks (wmg_measure_peak), the roofline denominators
of the ALU-bound operator kernels: positive and bounded by the unit counts
at the SM clock (152 SMs x 128 FP32 lanes x 2 FLOP x 2.07 GHz = 80.5 TFLOP/s
for one multiply-add per lane and cycle; the paired instruction can at most
double it), FP64 below FP32, and unknown kinds refused."""
import pytest

torch = pytest.importorskip("torch")
import paper_1310_0956_gb300 as wmg  # noqa: E402

pytestmark = pytest.mark.gpu


def test_measured_peaks_are_plausible():
    f32 = wmg.wmg_measure_peak(wmg.PEAK_FP32_FMA)
    f32x2 = wmg.wmg_measure_peak(wmg.PEAK_FP32_FMA2)
    f64 = wmg.wmg_measure_peak(wmg.PEAK_FP64_FMA)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    bound = sms * 128 * 2 * 2.2e9 / 1e12
    assert 0.3 * bound < f32 <= 1.05 * bound
    assert 0.3 * bound < f32x2 <= 2.1 * bound
    assert 0.0 < f64 < f32


def test_unknown_kind_is_refused():
    with pytest.raises(wmg.WmgError) as e:
        wmg.wmg_measure_peak(7)
    assert e.value.code == wmg.WMG_ERR_INVALID_ARG
