"""The benchmark's algorithmic flop table is the one the operation-counting
oracle measures (so the roofline's numerator is not a hand-typed guess)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("name", ["sedov", "sod512"])
def test_flop_table_matches_counting_oracle(name):
    sys.path.insert(0, ROOT)
    import bench
    from oracle import count_ops
    measured = count_ops.counts(name)["flops_per_unit"]
    table = bench.ALGORITHMIC_FLOPS[name]
    assert sorted(measured) == sorted(table)
    for stage, v in measured.items():
        assert table[stage] == pytest.approx(v, abs=1e-3), stage


def test_mixed_fp64_flops_by_construction():
    sys.path.insert(0, ROOT)
    import bench
    f3 = bench.mixed_fp64_flops(3)
    assert f3["riemann2"] == 88 and f3["update"] == 45
    assert bench.mixed_fp64_flops(1)["riemann2"] == 48
