"""The benchmark's algorithmic flop table is the one the operation-counting
oracle measures (so the roofline's numerator is not a hand-typed guess)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("name", ["sedov", "sod512", "noh"])
def test_flop_table_matches_counting_oracle(name):
    sys.path.insert(0, ROOT)
    import bench
    from oracle import count_ops
    measured = count_ops.counts(name)["flops_per_unit"]
    table = bench.ALGORITHMIC_FLOPS[name]
    assert sorted(measured) == sorted(table)
    for stage, v in measured.items():
        assert table[stage] == pytest.approx(v, abs=1e-3), stage


def test_mixed_tables_by_construction():
    """Mixed precision: FP64 only in the primitives (12 flops) and the update
    (10); the step's algorithmic HBM bytes per cell update add up the stages'."""
    sys.path.insert(0, ROOT)
    import bench
    f3 = bench.mixed_fp64_flops(3)
    assert f3["riemann2"] == 0 and f3["update"] == 10 and f3["prims"] == 12
    b = bench.ALGORITHMIC_BYTES["mixed"]
    assert bench.mixed_bytes_per_cell_update(3) == (b["prims"] + b["update"]
                                                    + 3 * (b["ppmc"] + b["riemann1"]
                                                           + b["riemann2"]))
    assert bench.mixed_bytes_per_cell_update(3) == 908


def test_ncu_traffic_table_is_consistent():
    """Each captured per-unit DRAM traffic sits just below the stage's
    algorithmic bytes (nothing re-read; part of the last writes still in L2
    when a kernel ends), and names the sources its digest covers."""
    sys.path.insert(0, ROOT)
    import bench
    for key, info in bench.NCU_TRAFFIC.items():
        assert 0.75 < info["bytes_per_unit"] / bench.ALGORITHMIC_BYTES[key[0]][key[1]] < 1.05, key
        assert len(bench.source_digest(info["sources"])) == 16
