"""The FP32 throughput probe (sp_fp32_peak), the measured denominator of the
projector's roofline: plausible values for this GPU (at most the SM count x
128 FP32 lanes x 2 flops x the maximum clock, by a small margin, and well
above a tenth of it), and the packed FMA form at least as fast as half the
scalar one (two FMAs per instruction)."""
import pytest

torch = pytest.importorskip("torch")
sp = pytest.importorskip("paper_2503_20907_gb300")

pytestmark = pytest.mark.gpu


def test_fp32_peak_probe():
    props = torch.cuda.get_device_properties(0)
    t1, ms1 = sp.fp32_peak(False)
    t2, ms2 = sp.fp32_peak(True)
    print(f"\nFP32 FMA chains: scalar {t1:.1f} TFLOP/s ({ms1:.2f} ms), packed {t2:.1f} TFLOP/s ({ms2:.2f} ms)")
    ceiling = props.multi_processor_count * 128 * 2 * 2.2e9 / 1e12   # 2.2 GHz: above any boost clock here
    for t, ms in ((t1, ms1), (t2, ms2)):
        assert ms > 0.0
        assert 0.1 * ceiling < t < 2.05 * ceiling
    assert t2 > 0.5 * t1
