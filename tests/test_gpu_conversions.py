"""The library's integer-pipe IEEE 754 conversions (binary64 -> binary32
round-to-nearest-even, binary32 -> binary64, finite test), which the FP32
path's FP64 stage epilogue uses instead of GB300's FP64-unit conversions,
checked against the hardware conversions bit for bit on generated values
(raw bit patterns over every exponent, rounding ties and their neighbours,
exponents at the edges of the binary32 range)."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1602_09079_gb300 as m
    m.load()
    return m


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_ieee_conversions_match_hardware(dg, seed):
    assert dg.dg_selftest_conversions(1 << 24, seed) == 0
