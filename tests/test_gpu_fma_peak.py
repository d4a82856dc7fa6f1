"""The FMA throughput measurement behind the matrix-element rooflines: FP32
near 152 SMs x 128 lanes x 2 FLOP per clock, FP64 far below it, and argument
errors."""
import pytest

from paper_2105_10529_gb300._lib import MF_FP64, MF_MIXED, MfError

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_fma_peak_is_plausible():
    from paper_2105_10529_gb300.api import measure_fma_peak
    props = torch.cuda.get_device_properties(0)
    nominal32 = props.multi_processor_count * 128 * 2 * 2.07e9 / 1e12   # at the maximum SM clock
    f32 = measure_fma_peak(MF_MIXED)
    f64 = measure_fma_peak(MF_FP64)
    assert 0.4 * nominal32 < f32 < 1.1 * nominal32, (f32, nominal32)
    assert 0.0 < f64 < f32 / 4, (f64, f32)


def test_fma_peak_arguments():
    import ctypes as C
    from paper_2105_10529_gb300 import _lib
    out = C.c_double(0.0)
    assert _lib.lib().mf_measure_fma_peak(7, None, C.byref(out)) == 1
    assert _lib.lib().mf_measure_fma_peak(MF_MIXED, None, None) == 1
    with pytest.raises(MfError):
        from paper_2105_10529_gb300.api import measure_fma_peak
        measure_fma_peak(3)
