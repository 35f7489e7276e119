"""Pins of the oracle's frozen-step adjoint: central finite differences of the frozen
forward map (grid values, initial position and direction, kappa), and consistency of the
recorded forward with the propagation module."""
import numpy as np
import pytest

import oracle as O
from paper_1410_5323_gb300 import inputs as I

C_LIGHT = 299792458.0


@pytest.fixture(scope="module")
def case(oracle_lib):
    g = I.kolmogorov_grid(8, 0.25 * I.MPC, 2, 4, 1e-13, 4)        # float64 grid
    f = O.OracleField(g, 0.25 * I.MPC)
    E = 10 ** 19.5
    kappa = C_LIGHT / E
    rng = np.random.default_rng(2)
    u = rng.standard_normal(3)
    u /= np.linalg.norm(u)
    y0 = np.concatenate([rng.uniform(0, 2 * I.MPC, 3), u])
    h, yT = O.record_steps(f, kappa, y0, 1e-4, I.KPC, I.MPC, 60)
    return g, f, kappa, y0, h, yT


def _loss(yT, t):
    u = yT[3:] / np.linalg.norm(yT[3:])
    return float(np.sum((u - t) ** 2))


def _lam(yT, t):
    un = np.linalg.norm(yT[3:])
    uh = yT[3:] / un
    gu = 2 * (uh - t)
    return np.concatenate([np.zeros(3), (gu - uh * np.dot(uh, gu)) / un])


def test_recorded_forward_matches_propagation_module(case):
    g, f, kappa, y0, h, yT = case
    assert np.all(h > 0) and np.all(h <= I.MPC)
    assert np.array_equal(O.frozen_forward(f, kappa, y0, h), yT)
    p = I.Particles(y0[None, :3].copy(), y0[None, 3:].copy(), np.array([C_LIGHT / kappa]),
                    np.array([1], np.int32), np.array([1], np.int32), np.array([0], np.int64),
                    np.array([0], np.int32))
    st = O.OracleState(1)
    O.inject(st, p, 1)
    O.propagate(st, [f], None, 1e-4, I.KPC, I.MPC, 1e30, max_steps=len(h), n_threads=1)
    assert np.array_equal([st.x[0], st.y[0], st.z[0], st.ux[0], st.uy[0], st.uz[0]], yT)


def test_adjoint_matches_finite_differences(case):
    g, f, kappa, y0, h, yT = case
    t = yT[3:] / np.linalg.norm(yT[3:]) + np.array([0.01, -0.02, 0.015])
    gbar = np.zeros_like(g)
    y0b, kb = O.adjoint(f, kappa, y0, h, _lam(yT, t), gbar)
    L = lambda gg=g, yy=y0, kk=kappa: _loss(O.frozen_forward(O.OracleField(gg, 0.25 * I.MPC), kk, yy, h), t)
    # grid entries with the largest gradients, plus one never touched (gradient exactly 0)
    flat = np.argsort(np.abs(gbar).ravel())[::-1][:8]
    for idx in flat:
        e = np.zeros(g.size)
        eps = 1e-4 * 1e-13
        e[idx] = eps
        fd = (L(g + e.reshape(g.shape)) - L(g - e.reshape(g.shape))) / (2 * eps)
        assert fd == pytest.approx(gbar.ravel()[idx], rel=1e-4, abs=1e-8 * np.abs(gbar).max())
    assert np.sum(gbar == 0) > 0
    for a in range(6):
        e = np.zeros(6)
        eps = 1e3 if a < 3 else 1e-7
        e[a] = eps
        fd = (L(yy=y0 + e) - L(yy=y0 - e)) / (2 * eps)
        assert fd == pytest.approx(y0b[a], rel=1e-4, abs=1e-6 * np.abs(y0b).max())
    eps = 1e-6 * kappa
    fd = (L(kk=kappa + eps) - L(kk=kappa - eps)) / (2 * eps)
    assert fd == pytest.approx(kb, rel=1e-4)
