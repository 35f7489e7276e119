"""Pins of the oracle's periodic trilinear field lookup (regular grid, paper Sec. 3.2)."""
import numpy as np
import pytest
from scipy.interpolate import RegularGridInterpolator

import oracle as O


def _field(grid, spacing=0.25, origin=(0.0, 0.0, 0.0)):
    return O.OracleField(np.ascontiguousarray(grid), spacing, origin)


def test_constant_field_exact_everywhere(oracle_lib):
    g = np.zeros((5, 6, 7, 3))
    g[...] = [1.5e-13, -2.25e-13, 0.75e-13]
    f = _field(g)
    rng = np.random.default_rng(3)
    for x in rng.uniform(-50, 50, (200, 3)):
        B = oracle_lib.field_value(f, x)
        # weights sum to one; with dyadic weights the sum is exact, else within 4 ulp
        assert np.allclose(B, g[0, 0, 0], rtol=4e-16, atol=0)


def test_node_values_reproduced(oracle_lib):
    rng = np.random.default_rng(4)
    g = rng.standard_normal((6, 5, 4, 3))
    f = _field(g, spacing=0.5, origin=(-1.0, 2.0, 0.5))
    for (i, j, k) in [(0, 0, 0), (5, 4, 3), (2, 3, 1)]:
        x = np.array([-1.0 + 0.5 * i, 2.0 + 0.5 * j, 0.5 + 0.5 * k])
        assert np.array_equal(oracle_lib.field_value(f, x), g[i, j, k])


def test_affine_field_exact_inside(oracle_lib):
    """Trilinear interpolation reproduces an affine field inside the non-wrapping region."""
    n = 8
    idx = np.arange(n, dtype=np.float64)
    I, J, K = np.meshgrid(idx, idx, idx, indexing="ij")
    M = np.array([[0.3, -1.2, 0.7], [2.0, 0.1, -0.4], [-0.9, 0.5, 1.1]])
    b0 = np.array([0.2, -0.3, 0.4])
    pos = np.stack([I, J, K], -1) * 0.25
    g = pos @ M.T + b0
    f = _field(g)
    rng = np.random.default_rng(5)
    for x in rng.uniform(0, 0.25 * (n - 1), (300, 3)):
        B = oracle_lib.field_value(f, x)
        assert np.allclose(B, M @ x + b0, rtol=1e-13, atol=1e-14)


def test_matches_scipy_regular_grid_interpolator(oracle_lib):
    """Library routine on the grid padded by one periodic layer (the wrap made explicit)."""
    rng = np.random.default_rng(6)
    nx, ny, nz = 7, 5, 6
    g = rng.standard_normal((nx, ny, nz, 3))
    sp = 0.3
    origin = (-0.4, 0.1, 0.25)
    f = _field(g, spacing=sp, origin=origin)
    gp = np.pad(g, ((0, 1), (0, 1), (0, 1), (0, 0)), mode="wrap")
    axes = [origin[a] + sp * np.arange(gp.shape[a]) for a in range(3)]
    ref = RegularGridInterpolator(axes, gp, method="linear")
    L = np.array([nx, ny, nz]) * sp
    for x in rng.uniform(-20, 20, (400, 3)):
        xin = origin + np.mod(x - origin, L)     # same point inside the first period
        B = oracle_lib.field_value(f, x)
        assert np.allclose(B, ref(xin[None])[0], rtol=0, atol=1e-12)


def test_periodic_wrap_bitwise(oracle_lib):
    """With dyadic spacing and positions, x and x + N*spacing*e_i give identical bits."""
    rng = np.random.default_rng(8)
    n = (4, 8, 16)
    g = rng.standard_normal(n + (3,))
    f = _field(g, spacing=0.25)
    for _ in range(100):
        x = np.round(rng.uniform(-8, 8, 3) * 1024) / 1024
        B0 = oracle_lib.field_value(f, x)
        for a in range(3):
            for m in (-2, -1, 1, 3):
                y = x.copy()
                y[a] += m * n[a] * 0.25
                assert np.array_equal(oracle_lib.field_value(f, y), B0)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_storage_widening(oracle_lib, dtype):
    """FP32 storage is widened exactly; BF16 storage is value*scale."""
    g = np.zeros((4, 4, 4, 3), dtype=np.float32)
    g[...] = [0.5, -0.25, 3.0]
    if dtype == "f32":
        f = O.OracleField(g, 1.0)
        assert np.array_equal(oracle_lib.field_value(f, np.array([1.25, 2.75, 0.125])), [0.5, -0.25, 3.0])
    else:
        bits = (g.view(np.uint32) >> 16).astype(np.uint16)   # exact: these values fit in bf16
        f = O.OracleField(bits, 1.0, scale=2e-13, dtype=O.BF16)
        assert np.allclose(oracle_lib.field_value(f, np.array([1.25, 2.75, 0.125])),
                           np.array([0.5, -0.25, 3.0]) * 2e-13, rtol=1e-15)


@pytest.mark.parametrize("scale", [1.0, 2e-13, -3.5])
def test_f16_widening_every_pattern(oracle_lib, scale):
    """F16 storage (Sec. 3.2 grids; the F16 storage type is this project's reading): every
    one of the 65 536 half-precision bit patterns -- normals, subnormals, +-0, +-inf, NaN --
    widens to numpy's float16 value in float64, times the FP32 scale in FP64."""
    bits = np.arange(65536, dtype=np.uint32).astype(np.uint16)
    g = np.empty((16, 16, 256, 3), dtype=np.uint16)
    g[..., 0] = bits.reshape(16, 16, 256)
    g[..., 1] = np.roll(bits, 1).reshape(16, 16, 256)
    g[..., 2] = np.roll(bits, 12345).reshape(16, 16, 256)
    f = O.OracleField(g, 1.0, scale=scale, dtype=O.F16)
    got = O.grid_values(f)
    with np.errstate(invalid="ignore"):
        want = g.view(np.float16).astype(np.float64) * np.float64(np.float32(scale))
    nan = np.isnan(want)
    assert nan.sum() == 3 * 2 * 1023                 # 1023 NaN payloads of either sign
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan], want[~nan])
    # signs of zero and infinity are kept
    assert np.array_equal(np.signbit(got[~nan]), np.signbit(want[~nan]))
