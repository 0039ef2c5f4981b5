"""Peak-rate probes (the roofline denominators) run, finish their bounded waits and measure
rates within the unit counts of the part: FP32 FMA at most 2 x 128 lanes x SMs x clock."""
import pytest

from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def _rate(torch, nv, kind, reps, err):
    s = torch.cuda.current_stream()
    nv.vfmm_probe_peak(kind, max(1, reps // 10), s.cuda_stream, err.data_ptr())
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(s)
    ops = nv.vfmm_probe_peak(kind, reps, s.cuda_stream, err.data_ptr())
    b.record(s)
    torch.cuda.synchronize()
    return ops / (a.elapsed_time(b) / 1e3)


def test_probe_rates_are_physical():
    torch = torch_cuda()
    from paper_1110_2921_gb300 import _native as nv
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    fp32_max = 2 * 128 * sms * 2.2e9          # above the 2070 MHz maximum clock
    ffma = _rate(torch, nv, nv.VFMM_PROBE_FFMA, 4000, err)
    print("FFMA %.1f TFLOP/s" % (ffma / 1e12))
    assert 0.3 * fp32_max < ffma < fp32_max
    for kind in (nv.VFMM_PROBE_EX2, nv.VFMM_PROBE_RSQRT):
        r = _rate(torch, nv, kind, 500, err)
        print("MUFU %d: %.0f Gop/s" % (kind, r / 1e9))
        assert 0 < r < fp32_max / 2            # MUFU is narrower than the FMA pipe
    d = _rate(torch, nv, nv.VFMM_PROBE_DFMA, 60, err)
    print("DFMA %.2f TFLOP/s" % (d / 1e12))
    assert 0 < d < fp32_max
    for kind in (nv.VFMM_PROBE_MMA_TF32, nv.VFMM_PROBE_MMA_BF16):
        r = _rate(torch, nv, kind, 40000, err)
        print("MMA %d: %.0f TFLOP/s" % (kind, r / 1e12))
        assert 1e14 < r < 3e15
    assert int(err.item()) == 0
