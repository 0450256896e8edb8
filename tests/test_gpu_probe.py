"""The tensor-core DFT probe: one radix-8 stage of the product's FFTs on FP32 butterflies and as
split-TF32 tensor-core matrix products, on the same data.  Checks both against FP64 (the split keeps
the error at the FP32 level, below the product's 1e-5 bar; a single TF32 product would not) and
reports the two timings (whether tensor cores pay for the FFT stages)."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_tensor_core_dft_stage_probe():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1002_1505_gb300 import dda as D
    # accuracy: four stages (an FFT of the product's lengths has two to four), against FP64
    a = D.dda_probe_tc_dft(0, nvec=1 << 12, reps=4)
    assert a["fp32_err"] < 1e-6 and a["tensor_err"] < 1e-5, a
    # speed: 256 stages on 16M complex values held in registers
    r = D.dda_probe_tc_dft(0, nvec=1 << 21, reps=256)
    print("DFT-8 stage probe (4 stages):", a, "(256 stages):", r)
    assert r["fp32_ms"] > 0 and r["tensor_ms"] > 0
