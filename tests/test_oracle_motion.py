"""Pins of the oracle's equation of motion and Cash-Karp integrator against closed forms
(charged-particle gyration, straight lines, integrator order; paper Sec. 2 deflections)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1410_5323_gb300 import inputs as I
from _oracle_helpers import C_LIGHT, particles, run, uniform_grid

B0 = 1e-13           # 1 nG
E19 = 1e19


def gyro_radius(E, Z, B):
    return E / (Z * C_LIGHT * B)


def circle(s, rg):
    """Proton (Z>0) launched along +x in B = B0 z-hat: clockwise circle seen from +z."""
    th = s / rg
    return (np.array([rg * math.sin(th), rg * (math.cos(th) - 1.0), 0.0]),
            np.array([math.cos(th), -math.sin(th), 0.0]))


def test_gyroradius_value():
    """Textbook: r_g = E/(Z c B); 10^19 eV proton in 1 nG is 10.81 Mpc."""
    assert abs(gyro_radius(E19, 1, B0) / I.MPC - 10.81) < 0.005


@pytest.mark.parametrize("frac", [0.1, 0.5, 1.0])
@pytest.mark.parametrize("tol", [1e-4, 1e-7])
def test_uniform_field_gyration(oracle_lib, frac, tol):
    rg = gyro_radius(E19, 1, B0)
    dmax = frac * 2 * math.pi * rg
    st, rc, _ = run(particles([1, 0, 0], E19), uniform_grid([0, 0, B0]), I.MPC, dmax, tol=tol,
                    hmax=10 * I.MPC)
    assert rc == 0 and st.status[0] == O.DONE and st.s[0] == dmax
    xe, ue = circle(dmax, rg)
    x = np.array([st.x[0], st.y[0], st.z[0]])
    u = np.array([st.ux[0], st.uy[0], st.uz[0]])
    # the accepted solution's global error is bounded by the tolerance per unit length
    assert np.linalg.norm(x - xe) <= tol * dmax
    assert np.linalg.norm(u - ue) <= tol * dmax / rg
    # after a full turn the particle is back at the start; centre stays at (0, -rg, 0)
    if frac == 1.0:
        assert np.linalg.norm(x) <= tol * dmax
    assert abs(np.linalg.norm(x - [0.0, -rg, 0.0]) - rg) <= tol * dmax


def test_tighter_tolerance_is_more_accurate(oracle_lib):
    rg = gyro_radius(E19, 1, B0)
    dmax = 2 * math.pi * rg
    errs = []
    for tol in (1e-3, 1e-5, 1e-7):
        st, _, _ = run(particles([1, 0, 0], E19), uniform_grid([0, 0, B0]), I.MPC, dmax, tol=tol,
                       hmax=10 * I.MPC)
        errs.append(np.linalg.norm(np.array([st.x[0], st.y[0], st.z[0]]) - circle(dmax, rg)[0]))
    assert errs[0] > errs[1] > errs[2]


def test_charge_sign_and_rigidity(oracle_lib):
    """Iron (Z=26) at 26x the energy has the proton's gyro-radius: same trajectory."""
    rg = gyro_radius(E19, 1, B0)
    dmax = 0.3 * rg
    a, _, _ = run(particles([1, 0, 0], E19), uniform_grid([0, 0, B0]), I.MPC, dmax)
    b, _, _ = run(particles([1, 0, 0], 26 * E19, A=56, Z=26), uniform_grid([0, 0, B0]), I.MPC, dmax)
    assert np.allclose([a.x[0], a.y[0]], [b.x[0], b.y[0]], rtol=1e-12, atol=1e-9 * rg)
    assert a.y[0] < 0          # positive charge turns clockwise about +z


def test_parallel_motion_is_straight(oracle_lib):
    dmax = 37.5 * I.MPC
    st, _, _ = run(particles([0, 0, 1], E19), uniform_grid([0, 0, B0]), I.MPC, dmax)
    assert st.ux[0] == 0 and st.uy[0] == 0 and st.uz[0] == 1.0
    assert st.x[0] == 0 and st.y[0] == 0
    assert abs(st.z[0] - dmax) <= 1e-12 * dmax


def test_neutral_particle_straight_at_max_step(oracle_lib):
    rng = np.random.default_rng(0)
    g = rng.standard_normal((8, 8, 8, 3)) * B0
    dmax = 20 * I.MPC
    st, _, _ = run(particles([0.6, 0.8, 0.0], E19, A=1, Z=0), g, 0.25 * I.MPC, dmax)
    assert st.status[0] == O.DONE
    assert np.allclose([st.x[0], st.y[0], st.z[0]], [0.6 * dmax, 0.8 * dmax, 0.0], rtol=1e-13, atol=1.0)
    # the error estimate vanishes, so steps are h_max at once (plus a last sliver from
    # rounding in the accumulated path length)
    assert st.n_steps[0] in (20, 21)


def test_speed_drift_bounded(oracle_lib):
    """|u| is not renormalised; its drift stays below tol per accepted step."""
    rng = np.random.default_rng(1)
    n = 16
    g = I.kolmogorov_grid(n, 0.25 * I.MPC, 2, 8, B0, 3)
    u = rng.standard_normal((32, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    st, _, _ = run(particles(u, E19), g, 0.25 * I.MPC, 50 * I.MPC)
    speed = np.sqrt(st.ux ** 2 + st.uy ** 2 + st.uz ** 2)
    assert np.all(np.abs(speed - 1) <= 1e-4 * st.n_steps)


def _one_attempt(h_over_rg):
    rg = gyro_radius(E19, 1, B0)
    f = O.OracleField(uniform_grid([0, 0, B0]), I.MPC)
    kappa = C_LIGHT / E19
    y0 = np.array([0, 0, 0, 1, 0, 0.0])
    h = h_over_rg * rg
    y5, err = O.ck_attempt(f, kappa, y0, h)
    xe, ue = circle(h, rg)
    return h, np.linalg.norm(err[3:]), np.linalg.norm(y5[3:] - ue)


def test_embedded_error_scales_as_h5(oracle_lib):
    """Cash & Karp: y5 - y4 = O(h^5) (a wrong tableau entry breaks an order condition)."""
    hs, es, ls = zip(*[_one_attempt(q) for q in (0.2, 0.1, 0.05, 0.025, 0.0125)])
    slope = np.polyfit(np.log(hs), np.log(es), 1)[0]
    assert abs(slope - 5.0) < 0.2


def test_fifth_order_solution_local_error_h6(oracle_lib):
    hs, es, ls = zip(*[_one_attempt(q) for q in (0.2, 0.1, 0.05, 0.025)])
    slope = np.polyfit(np.log(hs), np.log(ls), 1)[0]
    assert abs(slope - 6.0) < 0.3


def test_error_sums_definition(oracle_lib):
    """sx = |dx|^2, su = |du|^2 (Euclidean norms, kept squared)."""
    assert oracle_lib.error_sums([3.0, 4.0, 0.0, 0.0, 0.0, 2e-3]) == (25.0, 2e-3 * 2e-3)
    assert oracle_lib.error_sums([0.0, 0.0, 12.0, 1.0, 2.0, 2.0]) == (144.0, 9.0)


def test_fixed_step_global_error_is_fifth_order(oracle_lib):
    """Steps forced to a fixed h (h_min = h_max = h: every attempt is accepted) over one full
    gyration: the error of the returned position against the closed-form circle falls as h^5
    (fitted slope 5 +- 0.3), the global order of the propagated 5th-order solution."""
    rg = gyro_radius(E19, 1, B0)
    dmax = 2 * math.pi * rg
    hs, errs = [], []
    for n_steps in (20, 40, 80, 160):
        h = dmax / n_steps
        st, rc, _ = run(particles([1, 0, 0], E19), uniform_grid([0, 0, B0]), I.MPC, dmax, tol=1.0,
                        hmin=h, hmax=h)
        assert rc == 0 and st.status[0] == O.DONE
        assert abs(int(st.n_steps[0]) - n_steps) <= 1
        hs.append(h)
        errs.append(math.hypot(math.hypot(st.x[0], st.y[0]), st.z[0]))
    slope = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert abs(slope - 5.0) < 0.3, (slope, errs)
