"""The FP64 rate probe (hfx_probe_fp64): DFMA on CUDA cores and the FP64
tensor-core product measured on this GPU.  The FP64 build runs on DFMA; the
probe checks the rates are in the range that choice rests on (both near the
part's FP64 rate, about 1.26 TFLOP/s at 2.07 GHz) and prints them."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_fp64_rates():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_12505_gb300 import hfx
    dfma, dmma = hfx.probe_fp64()
    print(f"FP64 DFMA {dfma:.3f} TFLOP/s, FP64 tensor-core mma.sync {dmma:.3f} TFLOP/s")
    assert 0.2 < dfma < 10.0 and 0.2 < dmma < 10.0
