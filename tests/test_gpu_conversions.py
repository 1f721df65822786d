"""The integer-arithmetic float <-> double conversions that the mixed-precision
kernels use agree bit for bit with the hardware conversions (every float for
the widening, 2^30 sampled doubles for the round-to-nearest-even narrowing)."""
import pytest

pytestmark = pytest.mark.gpu


def test_conversions_match_hardware_bit_for_bit():
    from paper_1410_4194_gb300 import hydro
    widen, narrow = hydro.check_conversions()
    assert widen == 0, "float -> double mismatches: %d" % widen
    assert narrow == 0, "double -> float mismatches: %d" % narrow
