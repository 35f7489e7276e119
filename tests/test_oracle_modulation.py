"""Pins of the oracle's modulated field (paper Sec. 3.2 modulated grids, used so in Sec. 4):
B(x) = M(x) b(x), with b a periodic vector grid and M a periodic scalar grid, each
interpolated trilinearly over its own extent. Independent references: scipy's
RegularGridInterpolator, affine fields, periodicity and the gyration closed form."""
import math

import numpy as np
import pytest
from scipy.interpolate import RegularGridInterpolator

import oracle as O
from paper_1410_5323_gb300 import inputs as I
from _oracle_helpers import C_LIGHT, particles


def _field(grid, spacing, origin, mod, mspacing, morigin):
    return O.OracleField(np.ascontiguousarray(grid), spacing, origin, modulation=mod,
                         mod_spacing=mspacing, mod_origin=morigin)


def _wrap_interp(g, spacing, origin):
    """scipy interpolator over one period with the wrap layer made explicit."""
    gp = np.pad(g, [(0, 1)] * 3 + [(0, 0)] * (g.ndim - 3), mode="wrap")
    axes = [origin[a] + spacing * np.arange(gp.shape[a]) for a in range(3)]
    period = np.array(g.shape[:3]) * spacing
    ref = RegularGridInterpolator(axes, gp, method="linear")
    return lambda x: ref(np.asarray(origin) + np.mod(x - np.asarray(origin), period))[0]


def test_unit_modulation_leaves_the_field_unchanged(oracle_lib):
    rng = np.random.default_rng(11)
    g = rng.standard_normal((6, 5, 4, 3))
    plain = O.OracleField(g, 0.5, (0.1, -0.2, 0.3))
    f = _field(g, 0.5, (0.1, -0.2, 0.3), np.ones((3, 4, 5), np.float32), 0.7, (-1.0, 0.0, 2.0))
    # dyadic positions on both grids (spacings 1/2 and 0.7 are not both dyadic): M = sum of
    # weights, within 2 ulp of one; with modulation spacing 1/4 and dyadic x the sum is exact
    f2 = _field(g, 0.5, (0.1, -0.2, 0.3), np.ones((3, 4, 5), np.float32), 0.25, (0.0, 0.0, 0.0))
    for x in rng.uniform(-20, 20, (200, 3)):
        B0 = oracle_lib.field_value(plain, x)
        assert np.allclose(oracle_lib.field_value(f, x), B0, rtol=5e-16, atol=0)
        xd = np.round(x * 64) / 64
        assert np.array_equal(oracle_lib.field_value(f2, xd), oracle_lib.field_value(plain, xd))


def test_matches_scipy_product_of_two_periodic_interpolators(oracle_lib):
    """Different shapes (non-cubic, to catch a transposed index), spacings and origins for the
    two grids; positions over several periods of each, negative ones included."""
    rng = np.random.default_rng(12)
    g = rng.standard_normal((5, 7, 6, 3))
    m = rng.uniform(0.1, 3.0, (4, 3, 5)).astype(np.float32)
    sp, org = 0.3, (-0.4, 0.1, 0.25)
    msp, morg = 1.1, (0.35, -2.0, 0.6)
    f = _field(g, sp, org, m, msp, morg)
    b_ref = _wrap_interp(g, sp, org)
    m_ref = _wrap_interp(m.astype(np.float64), msp, morg)
    for x in rng.uniform(-15, 15, (400, 3)):
        assert oracle_lib.modulation_value(f, x) == pytest.approx(m_ref(x), rel=1e-12, abs=1e-13)
        B = oracle_lib.field_value(f, x)
        assert np.allclose(B, m_ref(x) * b_ref(x), rtol=1e-12, atol=1e-12)


def test_affine_modulation_times_constant_vector_exact_inside(oracle_lib):
    n = 6
    idx = np.arange(n, dtype=np.float64)
    msp = 0.5
    P = np.stack(np.meshgrid(idx, idx, idx, indexing="ij"), -1) * msp
    a, c = np.array([0.25, -0.5, 0.125]), 2.0
    m = (P @ a + c).astype(np.float32)               # exactly representable (dyadic)
    b0 = np.array([1.5, -0.75, 0.25])
    g = np.broadcast_to(b0, (4, 4, 4, 3)).copy()
    f = _field(g, 1.0, (0.0, 0.0, 0.0), m, msp, (0.0, 0.0, 0.0))
    rng = np.random.default_rng(13)
    for x in rng.uniform(0, msp * (n - 1), (300, 3)):
        assert np.allclose(oracle_lib.field_value(f, x), (a @ x + c) * b0, rtol=1e-14, atol=1e-14)


def test_modulation_is_periodic_over_its_own_extent(oracle_lib):
    rng = np.random.default_rng(14)
    m = rng.uniform(0.5, 2.0, (3, 4, 5)).astype(np.float32)
    msp = 0.75
    f = _field(np.ones((2, 2, 2, 3)), 0.5, (0, 0, 0), m, msp, (0.2, 0.3, -0.1))
    L = np.array(m.shape) * msp
    for x in rng.uniform(-5, 5, (100, 3)):
        v = oracle_lib.modulation_value(f, x)
        for a in range(3):
            e = np.zeros(3)
            e[a] = L[a]
            assert oracle_lib.modulation_value(f, x + 3 * e) == pytest.approx(v, rel=1e-12)
            assert oracle_lib.modulation_value(f, x - 2 * e) == pytest.approx(v, rel=1e-12)


def test_node_values_of_the_modulation_reproduced(oracle_lib):
    rng = np.random.default_rng(15)
    m = rng.uniform(0.5, 2.0, (4, 3, 5)).astype(np.float32)
    morg, msp = np.array([-1.0, 0.5, 2.0]), 0.25
    f = _field(np.ones((2, 2, 2, 3)), 1.0, (0, 0, 0), m, msp, morg)
    for (i, j, k) in [(0, 0, 0), (3, 2, 4), (1, 2, 3), (2, 0, 1)]:
        x = morg + msp * np.array([i, j, k])
        assert oracle_lib.modulation_value(f, x) == float(m[i, j, k])


@pytest.mark.parametrize("M", [0.25, -1.0])
def test_constant_modulation_gyration_closed_form(oracle_lib, M):
    """Uniform b = B0 z-hat times a constant modulation M: a circle of radius E/(Z c |M| B0),
    clockwise for M > 0 (proton) and counter-clockwise for M < 0."""
    B0, E = 1e-13, 1e19
    rg = E / (C_LIGHT * abs(M) * B0)
    dmax = 0.5 * 2 * math.pi * rg
    g = np.zeros((4, 4, 4, 3))
    g[..., 2] = B0
    m = np.full((3, 3, 3), M, dtype=np.float32)
    f = _field(g, I.MPC, (0, 0, 0), m, 7.0 * I.MPC, (0, 0, 0))
    st = O.OracleState(1)
    O.inject(st, particles([1, 0, 0], E), 1, None)
    tol = 1e-7
    rc, _ = O.propagate(st, [f], None, tol, I.KPC, 10 * I.MPC, dmax, seed=1, n_threads=1)
    assert rc == 0 and st.status[0] == O.DONE
    th = dmax / rg
    sgn = 1.0 if M > 0 else -1.0
    xe = np.array([rg * math.sin(th), sgn * rg * (math.cos(th) - 1.0), 0.0])
    x = np.array([st.x[0], st.y[0], st.z[0]])
    assert np.linalg.norm(x - xe) <= tol * dmax
