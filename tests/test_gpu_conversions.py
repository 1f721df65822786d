"""The integer-arithmetic float <-> double conversions that the mixed-precision
kernels use agree with the hardware conversions: bit for bit for normal values,
zeros and infinities (every float for the widening, 2^30 sampled doubles for the
round-to-nearest-even narrowing), subnormals flushed to a signed zero, NaN kept
NaN.  The kernels' integer halving, doubling and sign tests agree with the FP64
arithmetic, and the mixed update's float-float sums convert to a double within
one ulp of the FP64 add.  The Newton-refined FP64 reciprocal, quotient, square
root, reciprocal square root and the pressure function's reciprocal roots stay
within an ulp or two of the correctly rounded values."""
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


def test_newton_refined_operations_within_their_ulp_bounds():
    """The fast FP64 path's reciprocal, quotient and square root (a seed and
    Newton-type steps) differ from CUDA's correctly rounded operations by at
    most one ulp, and the reciprocal square root by at most one ulp from the
    nearest double to the exact value: what is left after the steps is the
    final rounding plus a fraction of an ulp.  The pressure function's
    reciprocal roots sigma^(-1/5) and sigma^(-1/2), from a float log2/exp2 seed
    and one third-order step, stay within two ulps over sigma in
    [1e-30, 1e30]: the residual 1 - sigma t^5 carries the rounding of three
    products (up to ~0.6 ulp in t), and the seed's error at the range's ends
    (~2^-19) leaves 11 delta^3 < 0.2 ulp after the step.  A dropped
    correction term or a wrong series coefficient would leave an error of the
    order of e or e^2 (2^-19 to 2^-38 relative: thousands of ulps or more)."""
    from paper_1410_4194_gb300 import hydro
    rcp, div, sqrt, rsqrt, root5, root2 = hydro.check_newton()
    assert rcp <= 1, "reciprocal: %d ulp" % rcp
    assert div <= 1, "quotient: %d ulp" % div
    assert sqrt <= 1, "square root: %d ulp" % sqrt
    assert rsqrt <= 1, "reciprocal square root: %d ulp" % rsqrt
    assert root5 <= 2, "sigma^(-1/5): %d ulp" % root5
    assert root2 <= 2, "sigma^(-1/2): %d ulp" % root2
