"""pcm_pipe_peak: the measured FMA rates sit below the nominal unit-count
peaks of the device (152 SMs x 128 FP32 lanes or 2 FP64 units x 2 flop x
clock) and well above a tenth of them, so that the roofline fractions the
bench reports against them are meaningful."""
import pytest

pytestmark = pytest.mark.gpu


def test_pipe_peaks_in_range():
    import torch
    import paper_1505_07851_gb300 as pcm
    p = torch.cuda.get_device_properties(0)
    nsm = p.multi_processor_count
    fmax = 2.07e9   # highest SM clock of the part
    nominal = {"fp32": nsm * 128 * 2 * fmax / 1e12, "fp64": nsm * 2 * 2 * fmax / 1e12}
    nominal["fp32x2"] = nominal["fp32"] * 2
    for k in ("fp32", "fp32x2", "fp64"):
        v = pcm.pipe_peak(k)
        assert 0.1 * nominal[k] < v < 1.05 * nominal[k], (k, v, nominal[k])


def test_pipe_peak_rejects_bad_kind():
    import paper_1505_07851_gb300 as pcm
    import ctypes
    out = ctypes.c_double()
    assert pcm.pcm_pipe_peak(0, 7, ctypes.byref(out)) == pcm.PCM_ERR_ARG
    assert pcm.pcm_pipe_peak(0, 0, None) == pcm.PCM_ERR_ARG
