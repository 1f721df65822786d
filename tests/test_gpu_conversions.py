"""The integer-arithmetic float <-> double conversions that the mixed-precision
kernels use agree with the hardware conversions: bit for bit for normal values,
zeros and infinities (every float for the widening, 2^30 sampled doubles for the
round-to-nearest-even narrowing), subnormals flushed to a signed zero, NaN kept
NaN.  The kernels' integer halving, doubling and sign tests agree with the FP64
arithmetic, and the mixed update's float-float sums convert to a double within
one ulp of the FP64 add."""
import pytest

pytestmark = pytest.mark.gpu


def test_conversions_match_hardware():
    from paper_1410_4194_gb300 import hydro
    widen, narrow = hydro.check_conversions()
    assert widen == 0, "float -> double mismatches: %d" % widen
    assert narrow == 0, "double -> float mismatches: %d" % narrow


def test_integer_scaling_matches_the_fp64_multiply():
    from paper_1410_4194_gb300 import hydro
    halving, doubling, signs, ffsums = hydro.check_scaling()
    assert halving == 0, "x/2 mismatches: %d" % halving
    assert doubling == 0, "2x mismatches: %d" % doubling
    assert signs == 0, "product sign mismatches: %d" % signs
    assert ffsums == 0, "float-float sum mismatches: %d" % ffsums


def test_fp64_rate_probe_is_the_fp64_pipe():
    """The FP64 throughput probe (the denominator the benchmark reports beside
    the unit-count peak) measures between half and 1.05 times GB300's two FP64
    FMA a clock an SM at the maximum clock (152 SMs x 2070 MHz x 2 x 2 flops):
    a kernel whose chains the compiler folded, or a float pipe measured by
    mistake, would fall outside."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    from paper_1410_4194_gb300 import hydro
    rate = hydro.probe_fp64_rate()
    nominal = 152 * 2070e6 * 2 * 2
    assert 0.5 * nominal < rate < 1.05 * nominal, rate
