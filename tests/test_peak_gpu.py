"""The library's arithmetic-peak probe (the roofline denominators of the
sweeps): the FP64 FMA loop and the packed two-float FMA loop run, return a
finite positive rate, and the FP32 pipe is the faster one by a wide margin on
a part whose FP64 rate is a small fraction of its FP32 rate (GB300: 1/64)."""
import math

import pytest

torch = pytest.importorskip("torch")

from paper_2305_19400_gb300 import bte

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2305_19400_gb300 import build as B
    B.build()


def test_fma_loops_measure_both_pipes():
    f64, ms64 = bte.bte_measure_peak(bte.BTE_PEAK_FP64_FMA)
    f32, ms32 = bte.bte_measure_peak(bte.BTE_PEAK_FP32X2_FMA)
    print(f"FP64 FMA {f64 / 1e12:.3f} TFLOP/s ({ms64:.1f} ms), packed FP32 FMA {f32 / 1e12:.2f} TFLOP/s ({ms32:.1f} ms)")
    assert math.isfinite(f64) and f64 > 0 and ms64 > 1.0
    assert math.isfinite(f32) and f32 > 0 and ms32 > 1.0
    assert f32 > 8 * f64


def test_unknown_kind_is_refused():
    with pytest.raises(bte.BTEError):
        bte.bte_measure_peak(7)
