"""Measurement entry point: arithmetic-pipe rates of the device (gpe_alu_peak).
Sanity bounds only (GB300: FP64 ~1.2 TFLOP/s nominal, FP32 ~75 TFLOP/s): the
rates are finite, positive, ordered, and the FP64 pipe is far below FP32."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G(built_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_02045_gb300 import gpe
    return gpe


def test_alu_peak_rates(G):
    fp64 = G.alu_peak("fp64_fma")
    fp32 = G.alu_peak("fp32_fma")
    fp32x2 = G.alu_peak("fp32x2_fma")
    assert 1e2 < fp64 < 1e5, fp64          # GFLOP/s
    assert 1e4 < fp32 < 3e5, fp32
    assert 1e4 < fp32x2 < 6e5, fp32x2
    assert fp32 > 8 * fp64
    assert G.lib().gpe_alu_peak(3, None, None) == G.GPE_ERR_ARG
