"""The precision form's accept decision is the FP64 one: outside a 2^-18 guard band around
tol^2 the FP32 squared norm of the error components certifies it. Checked here against the
FP64 squared norm on random FP32 components concentrated near the threshold, for both FP32
summation orders the compiler may produce (plain sums, or fused multiply-adds)."""
import numpy as np


def _band(tol2):
    lo = np.nextafter(np.float32(tol2 * (1.0 - 2.0 ** -18)), np.float32(0))    # rounded down (at least)
    hi = np.nextafter(np.float32(tol2 * (1.0 + 2.0 ** -18)), np.float32(np.inf))
    return lo, hi


def _q64(a, b, c):
    # fma(c, c, fma(b, b, a * a)) in FP64: FP32 squares are exact in FP64
    a, b, c = (x.astype(np.float64) for x in (a, b, c))
    return (a * a + b * b) + c * c


def _q32_plain(a, b, c):
    return (a * a + b * b) + c * c                       # float32 arithmetic


def _q32_fma(a, b, c):
    # fma(c, c, fma(b, b, a * a)) in FP32: each fused step rounds once
    t = (a * a).astype(np.float64)
    t = np.float32(t + b.astype(np.float64) ** 2)
    return np.float32(t.astype(np.float64) + c.astype(np.float64) ** 2)


def test_fp32_certificate_agrees_with_the_fp64_decision():
    rng = np.random.default_rng(7)
    n = 2_000_000
    for tol in (1e-4, 3.3e-7, 1e-2, 2.0 ** -40):
        tol2 = tol * tol
        lo, hi = _band(tol2)
        d = rng.standard_normal((n, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        # squared norms spread over +-2^-14 (relative) around tol^2, plus some far away
        s = np.sqrt(tol2 * (1.0 + rng.uniform(-2.0 ** -14, 2.0 ** -14, n)))
        s[: n // 10] *= rng.uniform(0.0, 3.0, n // 10)
        v = (d * s[:, None]).astype(np.float32)
        a, b, c = v[:, 0], v[:, 1], v[:, 2]
        q64 = _q64(a, b, c)
        for q32 in (_q32_plain(a, b, c), _q32_fma(a, b, c)):
            acc = q32 <= lo
            rej = q32 >= hi
            assert not np.any(acc & rej)
            assert np.all(q64[acc] <= tol2)
            assert np.all(q64[rej] > tol2)
            # the band is narrow: even with the norms packed within 2^-14 of tol^2, only the
            # ~1/16 of them inside the 2^-18 band are left to FP64
            assert np.mean(acc | rej) > 0.92
