"""Pins of the oracle's reflective boundary (Sec. 4: reflective boundary conditions) and of
backward tracking with antiparticles (Sec. 3.3 galactic propagation: cosmic rays propagated
backwards from Earth). References: the triangle wave of a straight line folded into a box,
time reversal of the Lorentz force, the gyration closed form, and invariants."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1410_5323_gb300 import inputs as I
from _oracle_helpers import C_LIGHT, particles, uniform_grid

MPC = I.MPC
BOX_O = np.array([-1.0, 2.0, 0.5]) * MPC
BOX_L = np.array([3.0, 4.0, 5.0]) * MPC


def _run(parts, grid, spacing, dmax, box=None, tol=1e-4, hmax=MPC, max_steps=0, calls=1, tables=None):
    f = O.OracleField(grid, spacing)
    st = O.OracleState(len(parts))
    O.inject(st, parts, 1, None if tables is None else O.OracleTables(tables))
    rc = 0
    for _ in range(calls):
        rc, _ = O.propagate(st, [f], None, tol, I.KPC, hmax, dmax, seed=1, max_steps=max_steps,
                            n_threads=2, box=box)
    return st, rc


def _triangle(z, o, L):
    """Straight line z(s) folded into [o, o + L] by mirrors: position and direction sign."""
    m = np.mod((z - o) / L, 2.0)
    return np.where(m < 1.0, o + m * L, o + (2.0 - m) * L), np.where(m < 1.0, 1.0, -1.0)


def test_neutral_particles_bounce_like_the_triangle_wave(oracle_lib):
    rng = np.random.default_rng(21)
    n = 64
    u = I.isotropic_directions(n, rng)
    x0 = BOX_O + rng.uniform(0.05, 0.95, (n, 3)) * BOX_L
    p = particles(u, 1e19, A=1, Z=0, x=x0)
    dmax = 37.3 * MPC
    st, rc = _run(p, uniform_grid([0, 0, 0]), MPC, dmax, box=(BOX_O, BOX_L))
    assert rc == 0 and np.all(st.status[:n] == O.DONE)
    x = np.stack([st.x, st.y, st.z], 1)[:n]
    uu = np.stack([st.ux, st.uy, st.uz], 1)[:n]
    u0 = np.stack([st.u0x, st.u0y, st.u0z], 1)[:n]
    for a in range(3):
        xe, sgn = _triangle(x0[:, a] + dmax * u[:, a], BOX_O[a], BOX_L[a])
        assert np.allclose(x[:, a], xe, rtol=0, atol=1e-9 * MPC)
        assert np.array_equal(uu[:, a], sgn * u[:, a])
        assert np.array_equal(u0[:, a], sgn * u[:, a])       # u0 flips with u: no deflection
    assert np.all((x >= BOX_O) & (x <= BOX_O + BOX_L))


def test_box_that_is_never_reached_changes_nothing(oracle_lib):
    B0, E = 1e-13, 1e19
    rg = E / (C_LIGHT * B0)
    g = uniform_grid([0, 0, B0])
    p = particles([1, 0, 0], E)
    dmax = 2 * math.pi * rg
    big = (np.array([-5 * rg, -5 * rg, -5 * rg]), np.array([10 * rg, 10 * rg, 10 * rg]))
    a, _ = _run(p, g, MPC, dmax, box=big, hmax=10 * MPC)
    b, _ = _run(p, g, MPC, dmax, box=None, hmax=10 * MPC)
    for k in ("x", "y", "z", "ux", "uy", "uz", "s", "n_steps", "n_att"):
        assert np.array_equal(getattr(a, k)[:1], getattr(b, k)[:1]), k


def test_charged_particles_stay_in_the_box_with_unit_speed(oracle_lib):
    g = I.kolmogorov_grid(16, 0.25 * MPC, 2, 8, 1e-12, 3)      # 10 nG: strongly deflected
    rng = np.random.default_rng(22)
    n = 200
    x0 = BOX_O + rng.uniform(0.0, 1.0, (n, 3)) * BOX_L
    p = particles(I.isotropic_directions(n, rng), 10 ** rng.uniform(17, 19, n), x=x0)
    f = O.OracleField(g, 0.25 * MPC)
    st = O.OracleState(n)
    O.inject(st, p, 1, None)
    for _ in range(30):                       # positions sampled every 7 accepted steps
        rc, _ = O.propagate(st, [f], None, 1e-4, I.KPC, MPC, 60 * MPC, max_steps=7, n_threads=2,
                            box=(BOX_O, BOX_L))
        assert rc == 0
        x = np.stack([st.x, st.y, st.z], 1)[:n]
        assert np.all(x >= BOX_O - 1e-9 * MPC) and np.all(x <= BOX_O + BOX_L + 1e-9 * MPC)
        # |u| is not renormalised: mirror flips keep it, the integrator drifts below tol a step
        speed = np.sqrt(st.ux[:n] ** 2 + st.uy[:n] ** 2 + st.uz[:n] ** 2)
        assert np.all(np.abs(speed - 1.0) <= 1e-4 * st.n_steps[:n])


def test_box_validation(oracle_lib):
    p = particles([1, 0, 0], 1e19)
    _, rc = _run(p, uniform_grid([0, 0, 1e-13]), MPC, MPC, box=(BOX_O, np.array([1.0, 0.0, 1.0])))
    assert rc == O.ERR_INVALID_ARG


def test_antiproton_gyrates_the_other_way(oracle_lib):
    B0, E = 1e-13, 1e19
    rg = E / (C_LIGHT * B0)
    dmax = 0.5 * 2 * math.pi * rg
    tol = 1e-7
    st, rc = _run(particles([1, 0, 0], E, Z=-1), uniform_grid([0, 0, B0]), MPC, dmax, tol=tol,
                  hmax=10 * MPC)
    assert rc == 0
    th = dmax / rg
    xe = np.array([rg * math.sin(th), -rg * (math.cos(th) - 1.0), 0.0])
    assert np.linalg.norm(np.array([st.x[0], st.y[0], st.z[0]]) - xe) <= tol * dmax


def test_backtracking_retraces_the_forward_trajectory(oracle_lib):
    """Time reversal of the Lorentz force: from the end point, direction reversed and charge
    negated, the particle returns to its start (to the integrator's error bound)."""
    g = I.kolmogorov_grid(16, 0.25 * MPC, 2, 8, 1e-13, 4)
    rng = np.random.default_rng(23)
    n = 100
    p = particles(I.isotropic_directions(n, rng), 1e19, A=4, Z=2, x=rng.uniform(0, 4 * MPC, (n, 3)))
    d = 3.0 * MPC
    tol = 1e-10
    fw, rc = _run(p, g, 0.25 * MPC, d, tol=tol)
    assert rc == 0
    xe = np.stack([fw.x, fw.y, fw.z], 1)[:n]
    ue = np.stack([fw.ux, fw.uy, fw.uz], 1)[:n]
    back = particles(-ue, 1e19, A=4, Z=-2, x=xe)
    bw, rc = _run(back, g, 0.25 * MPC, d, tol=tol)
    assert rc == 0
    xb = np.stack([bw.x, bw.y, bw.z], 1)[:n]
    ub = np.stack([bw.ux, bw.uy, bw.uz], 1)[:n]
    assert np.max(np.linalg.norm(xb - p.x, axis=1)) < 1e-6 * d
    assert np.max(np.linalg.norm(ub + p.u, axis=1)) < 1e-6
    # a charge that is not negated does not come back
    wrong, _ = _run(particles(-ue, 1e19, A=4, Z=2, x=xe), g, 0.25 * MPC, d, tol=tol)
    xw = np.stack([wrong.x, wrong.y, wrong.z], 1)[:n]
    assert np.median(np.linalg.norm(xw - p.x, axis=1)) > 1e-3 * d


def test_antiparticles_need_no_tables(oracle_lib):
    p = particles([1, 0, 0], 1e19, A=4, Z=-2)
    st = O.OracleState(1)
    with pytest.raises(ValueError):
        O.inject(st, p, 1, O.OracleTables(I.synthetic_tables()))
    with pytest.raises(ValueError):
        O.inject(st, particles([1, 0, 0], 1e19, A=4, Z=-5), 1, None)
    O.inject(st, p, 1, None)
