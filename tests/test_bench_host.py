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
    assert bench.ADJ_FLOP_PER_STEP_BACKWARD == (5 * 81 + 186) + 6 * 276 + 36 + 180 + 36
    # per attempt: 5 field evaluations (lookup 69 + Lorentz 12), stage sums, 5th-order update,
    # error estimate, squared norms + (h tol)^2, h x factor and clamp
    assert bench.FLOP_PER_ATTEMPT == 5 * (69 + 12) + 210 + 54 + 60 + (10 + 2) + 2
    # per accepted step: the next step's first field evaluation and kappa
    assert bench.FLOP_PER_ACCEPTED == (69 + 12) + 2
    # modulation: 42 per field evaluation, 5 per attempt and 1 per accepted step
    assert bench.MOD_FLOP_PER_ATTEMPT == 5 * 42 and bench.MOD_FLOP_PER_ACCEPTED == 42
    assert bench.FP64_PEAK_TFLOPS == pytest.approx(152 * 2 * 2.070e9 * 2 / 1e12)


PEAKS = {"hbm_gbs": 6794.1, "hbm_source": "test", "l2_gbs": 20000.0}


@pytest.mark.parametrize("tables,modulated", [(False, False), (True, False), (True, True)])
def test_fp64_roofline(tables, modulated):
    att, acc, t = 1.0e9, 6.0e8, 0.5
    r = bench.roofline_for("fp64", att, acc, tables, t, calls=1, workload="fp64_256cube_1M_nuclei",
                           modulated=modulated, grid_bytes=537_000_000, peaks=PEAKS)
    per_att = 743 + (210 if modulated else 0)
    per_acc = 83 + (42 if modulated else 0) + (10 if tables else 0)
    ach = (per_att * att + per_acc * acc) / t / 1e12
    T = r["terms"]
    assert T["fp64"]["achieved"] == pytest.approx(ach)
    assert T["fp64"]["frac"] == pytest.approx(ach / bench.FP64_PEAK_TFLOPS)
    # gathered FP64 values: 5 lookups per attempt + 1 per accepted step, 8 corners x 3 x 8 B
    gb = (5 * att + acc) * (192 + (32 if modulated else 0))
    assert T["gather"]["achieved"] == pytest.approx(gb / t / 1e9)
    assert T["gather"]["level"] == "hbm" and T["gather"]["peak"] == PEAKS["hbm_gbs"]
    assert T["fp32"]["achieved"] == pytest.approx((74 * att + (92 * acc if tables else 0)) / t / 1e12)
    # this work at this time is FP64-bound: the headline fields are the FP64 term's
    assert r["term"] == "fp64" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["frac"] == pytest.approx(T["fp64"]["frac"]) and r["achieved"] == T["fp64"]["achieved"]
    assert r["traffic"] == pytest.approx(139.1 * att)


def test_roofline_bound_is_the_max_term_not_the_sum():
    """The precision form's gathered bytes (6 lookups x 96 B per attempt) beat its residual
    FP64 ops against their peaks: the gather term binds; a grid that fits in L2 is measured
    against the L2 copy bandwidth."""
    att, acc, t = 1.0e10, 6.0e9, 1.0
    r = bench.roofline_for("mixed", att, acc, False, t, grid_bytes=1_600_000_000, peaks=PEAKS)
    T = r["terms"]
    assert T["gather"]["achieved"] == pytest.approx(6 * att * 96 / t / 1e9)
    ops = bench.MIXED_FP64_OPS_PER_ATTEMPT * att + bench.MIXED_FP64_OPS_PER_ACCEPTED * acc
    assert T["fp64"]["achieved"] == pytest.approx(ops / t / 1e12)
    assert T["fp32"]["achieved"] == pytest.approx(bench.MIXED_FP32_FLOP_PER_ATTEMPT * att / t / 1e12)
    fr = {k: v["frac"] for k, v in T.items()}
    assert r["term"] == max(fr, key=fr.get) == "gather" and r["bound"] == "hbm"
    assert r["frac"] == pytest.approx(max(fr.values())) and r["frac"] < sum(fr.values())
    b = bench.roofline_for("mixed", att, acc, False, t, grid_dtype="bf16", grid_bytes=1_600_000_000, peaks=PEAKS)
    assert b["terms"]["gather"]["achieved"] == pytest.approx(T["gather"]["achieved"] / 2)
    small = bench.roofline_for("mixed", att, acc, False, t, grid_bytes=50_000_000, peaks=PEAKS)
    assert small["terms"]["gather"]["level"] == "l2" and small["terms"]["gather"]["peak"] == PEAKS["l2_gbs"]
    # at a tenth of the rate the FP64 ops still are a smaller fraction than the gather
    slow = bench.roofline_for("mixed", att, acc, False, 10 * t, grid_bytes=1_600_000_000, peaks=PEAKS)
    assert slow["frac"] == pytest.approx(r["frac"] / 10)


def test_traffic_per_call():
    assert bench.traffic_for("fp64_256cube_1M_nuclei", "fp64", 2.0e9, 2) == pytest.approx(139.1 * 1.0e9)
    assert bench.traffic_for("fp64_256cube_1M_nuclei", "mixed", 1.0e9, 1) == pytest.approx(99.3e9)
    assert bench.traffic_for("no_such_workload", "fp64", 1.0e9, 1) is None
    assert bench.traffic_for("fp64_256cube_1M_nuclei", "fp64", 1.0e9, 0) is None


def test_aggregate_single_process_and_capacity():
    assert bench.aggregate(None, 12.5, 3.0, 5.0, None) == (12.5, 3.0, 5.0)
    p = I.make_particles(1000, 3, species=(("H", .5), ("Fe", .5)), energy=("fixed", 1e19))
    assert bench.capacity_for(p) == 1000 + int(np.sum(p.A - 1))
