"""The order facts behind the FP64 kernels' integer compares (crp_fp64.cuh: le_sum, le_pos,
lt_pos, eq_num, max_pos, clampd, is_zero): on the operand domains those helpers state, a
comparison of IEEE-754 binary64 bit patterns as integers gives the IEEE result. Checked here
on every pair from a set of special and random values, against numpy's IEEE operations."""
import numpy as np
import pytest

SPECIAL = [0.0, -0.0, 5e-324, 2.2250738585072014e-308, 1e-300, 0.5, 1.0, 1.5, 2.0, 1e300,
           np.finfo(np.float64).max, np.inf, -5e-324, -1.0, -1e300, -np.inf]


def bits(v):
    return np.asarray(v, dtype=np.float64).view(np.int64)


def nans():
    pos = np.array([0x7FF8000000000000, 0x7FF0000000000001, 0x7FFFFFFFFFFFFFFF], dtype=np.int64)
    return np.concatenate([pos, pos | np.int64(-0x8000000000000000)]).view(np.float64)


@pytest.fixture(scope="module")
def values():
    rng = np.random.default_rng(7)
    r = rng.standard_normal(200) * 10.0 ** rng.integers(-300, 300, 200)
    return np.concatenate([np.array(SPECIAL), r])


def test_le_sum_unsigned_order(values):
    # a in [+0, +inf] or NaN of either sign, b in [+0, +inf]
    a = np.concatenate([values[(values >= 0) & ~np.signbit(values)], nans()])
    b = values[(values >= 0) & ~np.signbit(values)]
    A, B = np.meshgrid(a, b, indexing="ij")
    got = bits(A).view(np.uint64) <= bits(B).view(np.uint64)
    with np.errstate(invalid="ignore"):
        assert np.array_equal(got, A <= B)


def test_le_lt_pos_signed_order(values):
    # a not NaN; le: b in [+0, +inf]; lt: b in (+0, +inf]
    a = values
    for strict in (False, True):
        b = values[(values > 0) if strict else ((values >= 0) & ~np.signbit(values))]
        A, B = np.meshgrid(a, b, indexing="ij")
        got = bits(A) < bits(B) if strict else bits(A) <= bits(B)
        assert np.array_equal(got, A < B if strict else A <= B), strict


def test_eq_num_and_is_zero(values):
    A, B = np.meshgrid(values, values, indexing="ij")
    x, y = bits(A), bits(B)
    got = (x == y) | (((x | y) << 1) == 0)
    assert np.array_equal(got, A == B)
    v = np.concatenate([values, nans()])
    with np.errstate(invalid="ignore"):
        assert np.array_equal((bits(v) << 1) == 0, v == 0.0)


def test_max_pos_and_clamp(values):
    b = values[values > 0]
    A, B = np.meshgrid(values, b, indexing="ij")
    got = np.where(bits(A) < bits(B), B, A)
    assert np.array_equal(got, np.fmax(A, B))
    lo, hi = 1e-3, 1e3
    quiet = nans()[(bits(nans()) & np.int64(1 << 51)) != 0]   # fmax of a signaling NaN varies
    v = np.concatenate([values, quiet])
    x = bits(v)
    nan = (x & np.int64(0x7FFFFFFFFFFFFFFF)) > np.int64(0x7FF0000000000000)
    got = np.where(nan | (x < bits(lo)), lo, np.where(x > bits(hi), hi, v))
    assert np.array_equal(got, np.fmin(np.fmax(v, lo), hi))
