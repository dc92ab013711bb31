"""The measured FP64 FMA rate that the FP64 forms' arithmetic roofline is
reported against: positive, repeatable, and of the order of GB300's nominal
FP64 rate (1.25 TFLOP/s; a narrow FP64 pipe next to its FP32 one)."""
import pytest

pytestmark = pytest.mark.gpu


def test_fp64_fma_rate():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1003_4548_gb300 import capi
    r1 = capi.measure_fp64_fma_rate(torch.cuda.current_stream().cuda_stream)
    r2 = capi.measure_fp64_fma_rate(torch.cuda.current_stream().cuda_stream)
    assert 0.2 < r1 < 5.0 and 0.2 < r2 < 5.0
    assert abs(r1 - r2) < 0.2 * max(r1, r2)
