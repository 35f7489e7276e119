"""Pins of the oracle's exp/log (Cody-Waite reduction + truncated series): accuracy
against the C library over the ranges the method uses, and IEEE special cases."""
import math

import numpy as np


def _ulp_err(got, ref):
    if ref == 0.0:
        return 0.0 if got == 0.0 else float("inf")
    return abs(got - ref) / math.ulp(ref)


def test_exp_within_one_ulp(oracle_lib):
    rng = np.random.default_rng(1)
    xs = np.concatenate([rng.uniform(-745, 709, 20000), rng.uniform(-1, 1, 20000),
                         rng.uniform(-1e-6, 1e-6, 2000), [0.0, -0.0, 1.0, -1.0, 700.0, -700.0]])
    worst = max(_ulp_err(oracle_lib.exp(float(x)), math.exp(float(x))) for x in xs)
    assert worst <= 1.0


def test_log_within_two_ulp(oracle_lib):
    rng = np.random.default_rng(2)
    xs = np.concatenate([np.exp(rng.uniform(-740, 709, 20000)), rng.uniform(0.5, 2.0, 20000),
                         1.0 + rng.uniform(-1e-9, 1e-9, 2000), [5e-324, 1e-310, 1.7e308]])
    worst = max(_ulp_err(oracle_lib.log(float(x)), math.log(float(x))) for x in xs)
    assert worst <= 2.0
    assert oracle_lib.log(1.0) == 0.0


def test_special_values(oracle_lib):
    inf = float("inf")
    assert oracle_lib.exp(-inf) == 0.0 and oracle_lib.exp(inf) == inf
    assert oracle_lib.exp(710.0) == inf and oracle_lib.exp(-746.0) == 0.0
    assert math.isnan(oracle_lib.exp(float("nan")))
    assert oracle_lib.log(0.0) == -inf and oracle_lib.log(inf) == inf
    assert math.isnan(oracle_lib.log(-1.0)) and math.isnan(oracle_lib.log(float("nan")))


def test_pow_through_exp_log(oracle_lib):
    """Powers through exp(p log r) stay within 4 ulp (the loss and table paths use both)."""
    for r in [1e-12, 1e-3, 0.37, 1.0, 2.5, 1e3]:
        for p in (-0.2, -0.25):
            got = oracle_lib.exp(p * oracle_lib.log(r))
            assert abs(got - r ** p) <= 4 * math.ulp(r ** p)
