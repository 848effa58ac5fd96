"""The FP32 FMA-rate probe that supplies the FP32 roofline's denominator: it runs, it scales with the work
it is given, and it lands between a plausible floor and the device's derived ceiling (SMs x 128 FP32 lanes
x 2 flops x the maximum clock the device reports)."""
import pytest

from gpu_common import need_gpu, torch
from paper_1810_02821_gb300 import build, wf

pytestmark = pytest.mark.gpu


def test_fp32_peak_probe():
    need_gpu()
    build.build()
    props = torch.cuda.get_device_properties(0)
    for paired in (False, True):
        wf.wf_measure_fp32_peak(paired, 2048)
        tf1, ms1 = wf.wf_measure_fp32_peak(paired, 8192)
        tf2, ms2 = wf.wf_measure_fp32_peak(paired, 32768)
        assert ms2 > 2.5 * ms1, (ms1, ms2)
        derived = props.multi_processor_count * 128 * 2 * 2.2e9 / 1e12   # above any GB300 boost clock
        assert 0.3 * derived < tf2 < derived, (paired, tf2, derived)
    with pytest.raises(wf.WFError):
        wf.wf_measure_fp32_peak(False, 0)
