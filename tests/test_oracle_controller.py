"""Pins of the oracle's accept test and step-size controller (Sec. 3.1: the step is kept when
its estimated error is within the requested accuracy, and the next step is sized from it).
r = max(|dx|/h, |du|)/tol; accept iff r <= 1, compared as squares in FP64; the factor
0.95 r^p (p = -1/5 after an accepted step, -1/4 after a rejected one) is evaluated in FP32.
References: the square-root definition of r in FP64 (away from r = 1 by more than its
rounding), numpy's log2 and powers, exact powers of two, and the special cases."""
import math

import numpy as np
import pytest

U32 = 2.0 ** -24


def test_accept_is_r_at_most_one(oracle_lib):
    rng = np.random.default_rng(71)
    n_checked = 0
    for _ in range(20000):
        h = 10 ** rng.uniform(16, 22)
        tol = 10 ** rng.uniform(-6, -2)
        dx = rng.standard_normal(3) * h * tol * 10 ** rng.uniform(-1.5, 1.5)
        du = rng.standard_normal(3) * tol * 10 ** rng.uniform(-1.5, 1.5)
        sx, su = oracle_lib.error_sums(np.concatenate([dx, du]))
        r = max(math.sqrt(sx) / h, math.sqrt(su)) / tol
        if abs(r - 1.0) < 1e-12:
            continue
        n_checked += 1
        assert oracle_lib.error_accept(sx, su, h, tol) == (r <= 1.0)
    assert n_checked > 19000


def test_accept_boundary_and_special_cases(oracle_lib):
    tol = 0.5
    assert oracle_lib.error_accept(4.0, 0.25, 4.0, tol)          # |dx| = h tol and |du| = tol exactly
    assert not oracle_lib.error_accept(np.nextafter(4.0, 5.0), 0.0, 4.0, tol)
    assert not oracle_lib.error_accept(0.0, np.nextafter(0.25, 1.0), 4.0, tol)
    assert oracle_lib.error_accept(1e300, 1e300, 0.0, tol)       # zero-length step: r = 0
    assert not oracle_lib.error_accept(float("nan"), 0.0, 4.0, tol)
    assert not oracle_lib.error_accept(0.0, float("inf"), 4.0, tol)


def test_ctrl_log2_against_numpy(oracle_lib):
    rng = np.random.default_rng(72)
    v = 10 ** rng.uniform(-300, 300, 20000)
    got = np.array([oracle_lib.ctrl_log2(x) for x in v])
    ref = np.log2(v)
    # 23 truncated significand bits (1.7e-7), series and FP32 rounding, plus half an ulp of
    # the FP32 result
    assert np.all(np.abs(got - ref) <= 4e-7 + np.abs(ref) * U32)
    # near the reduction boundary sqrt(2) and at 1
    for x in [math.sqrt(2) * (1 - 1e-7), math.sqrt(2) * (1 + 1e-7), 1.0 + 2 ** -20, 1.0 - 2 ** -20, 3.0, 0.75]:
        assert abs(oracle_lib.ctrl_log2(x) - math.log2(x)) <= 4e-7


def test_ctrl_log2_exact_powers_and_specials(oracle_lib):
    for k in range(-1022, 1024, 37):
        assert oracle_lib.ctrl_log2(2.0 ** k) == float(k)
    assert oracle_lib.ctrl_log2(0.0) == -math.inf
    assert oracle_lib.ctrl_log2(5e-324) == -math.inf                # subnormal: no error
    assert oracle_lib.ctrl_log2(math.inf) == math.inf
    assert oracle_lib.ctrl_log2(math.nan) == math.inf                # NaN: an infinite error


def test_ctrl_factor_against_power(oracle_lib):
    for p, lo, hi in [(-0.2, 0.2, 5.0), (-0.25, 0.1, 1.0)]:
        for l2 in np.linspace(-45.0, 45.0, 1801):
            got = oracle_lib.ctrl_factor(l2, p, lo, hi)
            y = min(max(float(np.float32(p) * np.float32(l2)), -8.0), 8.0)
            ref = min(max(0.95 * 2.0 ** y, float(np.float32(lo))), float(np.float32(hi)))
            assert abs(got - ref) <= 4 * U32 * ref, (p, l2, got, ref)


def test_ctrl_factor_special_cases(oracle_lib):
    assert oracle_lib.ctrl_factor(0.0, -0.2, 0.2, 5.0) == float(np.float32(0.95))   # r = 1
    assert oracle_lib.ctrl_factor(math.inf, -0.25, 0.1, 1.0) == float(np.float32(0.1))
    assert oracle_lib.ctrl_factor(math.nan, -0.25, 0.1, 1.0) == float(np.float32(0.1))
    assert oracle_lib.ctrl_factor(-math.inf, -0.2, 0.2, 5.0) == 5.0
    # y is clamped to [-8, 8] before the power (seen only with bounds wider than the step's)
    assert oracle_lib.ctrl_factor(-50.0, -0.2, 0.0, 1000.0) == float(np.float32(0.95 * 256.0))
    assert oracle_lib.ctrl_factor(50.0, -0.2, 0.0, 1000.0) == float(np.float32(np.float32(0.95) * np.float32(2.0 ** -8)))
    # exact powers of two: r = 2^(5k) gives 0.95 2^-k after an accepted step
    for k in range(-1, 3):
        assert oracle_lib.ctrl_factor(5.0 * k, -0.2, 0.0, 100.0) == float(np.float32(np.float32(0.95) * np.float32(2.0 ** -k)))


def test_controller_is_the_power_law(oracle_lib):
    """From the error sums to the factor: 0.95 r^p with r from the square-root definition,
    to a few FP32 rounding errors of log2 values up to ~200 in size."""
    rng = np.random.default_rng(73)
    for _ in range(5000):
        h = 10 ** rng.uniform(16, 22)
        tol = 10 ** rng.uniform(-6, -2)
        dx = rng.standard_normal(3) * h * tol * 10 ** rng.uniform(-3, 3)
        du = rng.standard_normal(3) * tol * 10 ** rng.uniform(-3, 3)
        sx, su = oracle_lib.error_sums(np.concatenate([dx, du]))
        r = max(math.sqrt(sx) / h, math.sqrt(su)) / tol
        l2 = oracle_lib.ctrl_log2r(sx, su, h, tol)
        assert abs(l2 - math.log2(r)) <= 3e-5
        for p, lo, hi in [(-0.2, 0.2, 5.0), (-0.25, 0.1, 1.0)]:
            ref = min(max(0.95 * r ** p, lo), hi)
            assert oracle_lib.ctrl_factor(l2, p, lo, hi) == pytest.approx(ref, rel=2e-5)
