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
