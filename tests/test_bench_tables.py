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
    """Mixed precision: FP64 only in the primitives (8 flops) and the update
    (10); the step's algorithmic HBM bytes per cell update add up the stages'."""
    sys.path.insert(0, ROOT)
    import bench
    f3 = bench.mixed_fp64_flops(3)
    assert f3["riemann2"] == 0 and f3["update"] == 10 and f3["prims"] == 8
    b = bench.ALGORITHMIC_BYTES["mixed"]
    assert bench.mixed_bytes_per_cell_update(3) == (b["prims"] + b["update"]
                                                    + 3 * (b["ppmc"] + b["riemann1"]
                                                           + b["riemann2"]))
    assert bench.mixed_bytes_per_cell_update(3) == 908


def test_ncu_traffic_table_is_consistent():
    """Each captured per-unit DRAM traffic sits near the stage's algorithmic
    bytes (below them where part of the last writes is still in L2 when a
    kernel ends), and names the sources its digest covers.  Above by at most
    5%, except the FP64 PPMC and second Riemann set, whose y and z sweeps by
    four-cell segments read the halo rows of the neighbouring segments again
    (PPMC 200.7 B a cell against 184, the three sweeps averaging 195.1; the
    second set 213.3 B a face against 200, averaging 211.4) in kernels bound by
    their FP64 pipe with DRAM 8-16% busy."""
    sys.path.insert(0, ROOT)
    import bench
    for key, info in bench.NCU_TRAFFIC.items():
        hi = 1.10 if key in (("fp64", "ppmc"), ("fp64", "riemann2")) else 1.05
        assert 0.75 < info["bytes_per_unit"] / bench.ALGORITHMIC_BYTES[key[0]][key[1]] < hi, key
        assert len(bench.source_digest(info["sources"])) == 16


def test_l1_helper_and_scaled_turbulence_recipe():
    """bench.l1_rel: the relative L1 difference per field, the momenta against
    their group's largest L1 norm; the small turbulence boxes keep the 512^3
    recipe's 32 cells across the shortest wavelength (shells scaled with n)."""
    sys.path.insert(0, ROOT)
    import numpy as np

    import bench
    ref = np.ones((5, 2, 2, 2))
    ref[1:4] = 0.0
    ref[2] = 2.0  # the momenta's common scale: sum |m_y| = 16
    a = ref.copy()
    a[0, 0, 0, 0] += 0.5   # rho: 0.5 / 8
    a[3, 1, 1, 1] += 1.0   # m_z: 1 / 16
    l1 = bench.l1_rel(a, ref)
    assert l1 == pytest.approx([0.5 / 8, 0.0, 0.0, 1.0 / 16, 0.0])
    assert bench.workload_shape("turbulence128") == (128, 128, 128)
    assert "shells 1..4" in bench.workload_desc("turbulence128")


def test_fp64_slot_table_matches_the_traffic_capture():
    """The FP64 lane-slot counts and the DRAM bytes per unit come from the same
    ncu captures of the same kernel sources."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.NCU_FP64_SLOTS_DIGEST == bench.NCU_TRAFFIC[("fp64", "riemann2")]["digest"]
    for (wl, stage), v in bench.NCU_FP64_SLOTS.items():
        assert wl in ("sedov", "turbulence") and stage in bench.ALGORITHMIC_FLOPS["sedov"]
        assert 0 < v < 400


def test_single_roofline_of_a_synthetic_fp64_step():
    """The FP64 roofline from a per-stage split: the dominant stage (the second
    Riemann set, its x and y, z kernels named), its algorithmic flops per launch
    over its average launch time against the unit-count peak, the captured
    traffic scaled to the launch's units while the sources match the capture,
    and the FP64 issue fraction from the captured lane-slots (Sedov 256^3
    shapes: 257 x 256 x 256 faces a launch, three launches)."""
    sys.path.insert(0, ROOT)
    import bench
    faces = 257 * 256 * 256
    stages = {"prims": (2.4, 3, 3 * 264 ** 3), "riemann2": (16.2, 3, 3 * faces),
              "riemann1": (9.9, 3, 3 * 257 * 258 * 258)}
    r = bench.single_roofline(stages, "fp64", "sedov", "ppmc", "exact", 3, 128, None, 2070.0)
    assert r["kernel"] == "kb_riemann2 (x) / kb_riemann2_seg (y, z)"
    assert r["units_per_launch"] == faces and abs(r["avg_launch_ms"] - 5.4) < 1e-12
    flops = bench.ALGORITHMIC_FLOPS["sedov"]["riemann2"] * faces / 5.4e-3
    assert abs(r["achieved"] / flops - 1) < 1e-12
    assert abs(r["frac"] - flops / bench.FP64_FLOPS_PEAK) < 1e-12
    info = bench.NCU_TRAFFIC[("fp64", "riemann2")]
    assert abs(r["traffic"] - info["bytes_per_unit"] * faces) < 1e-3
    slots = bench.NCU_FP64_SLOTS[("sedov", "riemann2")]
    assert abs(r["fp64_issue_frac"] - slots * faces / 5.4e-3 / (2 * 152 * 2070e6)) < 1e-12
    # a 1D grid names the one-face kernel; the Roe solver its own kernel
    r1 = bench.single_roofline(stages, "fp64", "sedov", "ppmc", "exact", 1, 128, None, 2070.0)
    assert r1["kernel"] == "kb_riemann2"
    rr = bench.single_roofline(stages, "fp64", "sedov", "ppmc", "roe", 3, 128, None, 2070.0)
    assert rr["kernel"] == "kb_riemann2_roe" and rr["traffic"] is None
