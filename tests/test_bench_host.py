"""Host-side arithmetic of bench.py: the algorithmic FLOP counts add up from their parts, the
roofline and traffic figures follow from them, whole-job aggregation without ranks, and the
secondary capacity of a batch."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402
from paper_1410_5323_gb300 import inputs as I  # noqa: E402


def test_flop_counts_add_up():
    # per attempt: 5 field evaluations (lookup 69 + Lorentz 12), stage sums, 5th-order update,
    # error estimate, squared norms + (h tol)^2, h x factor and clamp
    assert bench.FLOP_PER_ATTEMPT == 5 * (69 + 12) + 210 + 54 + 60 + (10 + 2) + 2
    # per accepted step: the next step's first field evaluation and kappa
    assert bench.FLOP_PER_ACCEPTED == (69 + 12) + 2
    # modulation: 42 per field evaluation, 5 per attempt and 1 per accepted step
    assert bench.MOD_FLOP_PER_ATTEMPT == 5 * 42 and bench.MOD_FLOP_PER_ACCEPTED == 42
    assert bench.FP64_PEAK_TFLOPS == pytest.approx(152 * 2 * 2.070e9 * 2 / 1e12)


@pytest.mark.parametrize("tables,modulated", [(False, False), (True, False), (True, True)])
def test_fp64_roofline(tables, modulated):
    att, acc, t = 1.0e9, 6.0e8, 0.5
    r = bench.roofline_for("fp64", att, acc, tables, t, calls=1, workload="fp64_256cube_1M_nuclei",
                           modulated=modulated)
    per_att = 743 + (210 if modulated else 0)
    per_acc = 83 + (42 if modulated else 0) + (30 if tables else 0)
    ach = (per_att * att + per_acc * acc) / t / 1e12
    assert r["achieved"] == pytest.approx(ach)
    assert r["frac"] == pytest.approx(ach / bench.FP64_PEAK_TFLOPS)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["traffic"] == pytest.approx(140.5 * att)


def test_traffic_per_call():
    assert bench.traffic_for("fp64_256cube_1M_nuclei", "fp64", 2.0e9, 2) == pytest.approx(140.5 * 1.0e9)
    assert bench.traffic_for("fp64_256cube_1M_nuclei", "mixed", 1.0e9, 1) == pytest.approx(99.4e9)
    assert bench.traffic_for("no_such_workload", "fp64", 1.0e9, 1) is None
    assert bench.traffic_for("fp64_256cube_1M_nuclei", "fp64", 1.0e9, 0) is None


def test_mixed_roofline_counts_residual_fp64_ops():
    r = bench.roofline_for("mixed", 1.0e9, 6.0e8, True, 0.25)
    ops = bench.MIXED_FP64_OPS_PER_ATTEMPT * 1.0e9 + bench.MIXED_FP64_OPS_PER_ACCEPTED * 6.0e8
    assert r["achieved"] == pytest.approx(ops / 0.25 / 1e12)
    assert r["fp32_achieved_tflops"] == pytest.approx(bench.MIXED_FP32_FLOP_PER_ATTEMPT * 1.0e9 / 0.25 / 1e12)
    assert r["traffic"] is None                          # no workload named: no measured bytes


def test_aggregate_single_process_and_capacity():
    assert bench.aggregate(None, 12.5, 3.0, 5.0, None) == (12.5, 3.0, 5.0)
    p = I.make_particles(1000, 3, species=(("H", .5), ("Fe", .5)), energy=("fixed", 1e19))
    assert bench.capacity_for(p) == 1000 + int(np.sum(p.A - 1))
