"""The library's arithmetic-pipe microbenchmarks (roofline denominators).

The FP32 FMA rate must lie near what the SM count and the clock allow (128
FP32 lanes per SM, one FMA per lane and clock, clock between 1 and 2.2 GHz),
and the ex2.approx rate below it (the special function unit is narrower)."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_measured_peaks_are_plausible():
    import paper_1009_1351_gb300 as tn
    from paper_1009_1351_gb300 import build
    build.build()
    tn.load_library()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    r = tn.tnlm_measure_peaks(0)
    lanes = sms * 128
    assert lanes * 1.0e9 * 0.7 <= r["fp32_ops"] <= lanes * 2.2e9
    assert 0 < r["ex2_ops"] < r["fp32_ops"]
