"""Reflective box (paper Sec. 4) and backward tracking with antiparticles (Sec. 3.3) on the
GPU: the FP64 form bit for bit against the oracle (every column, u0 included), the precision
form against closed forms and by two-sample KS."""
import numpy as np
import pytest
from scipy import stats

import oracle as O
from paper_1410_5323_gb300 import inputs as I
from _parity import assert_bit_identical, by_uid, run_gpu, run_oracle

pytestmark = pytest.mark.gpu
MIXED = 1
MPC = I.MPC
MIX = (("H", .4), ("He", .3), ("N", .2), ("Fe", .1))
BOX = (np.array([-1.0, 2.0, 0.5]) * MPC, np.array([3.0, 4.0, 5.0]) * MPC)


def _inside(n, seed):
    rng = np.random.default_rng(seed)
    return BOX[0] + rng.uniform(0.0, 1.0, (n, 3)) * BOX[1]


def _grid(seed=1, n=32):
    return I.kolmogorov_grid(n, 0.25 * MPC, 2, 16, 1e-13, seed).astype(np.float32)


def test_fp64_reflective_box_with_interactions_bit_identical(oracle_lib):
    g = _grid(1)
    p = I.make_particles(2000, 41, species=MIX, energy=("power", 1e18, 10 ** 20.5, 2.0))
    p.x[:] = _inside(len(p), 41)
    t = I.synthetic_tables()
    args = ([g], p, t, 1e-4, I.KPC, MPC, 30 * MPC)
    kw = dict(seed=5, capacity=2000 * 56, box=BOX)
    sim, rc = run_gpu(*args, **kw)
    assert rc == 0
    st, orc = run_oracle(*args, **kw)
    assert orc == 0
    a = sim.state()
    assert_bit_identical(a, st.snapshot())
    x = np.stack([a["x"], a["y"], a["z"]], 1)
    assert np.all((x >= BOX[0]) & (x <= BOX[0] + BOX[1]))
    assert sim.counts()["secondaries"] > 0


@pytest.mark.parametrize("max_steps", [37, 300])
def test_fp64_reflective_box_budgeted_calls_bit_identical(oracle_lib, max_steps):
    g = _grid(2)
    p = I.make_particles(800, 42, energy=("loguniform", 1e17, 1e20))
    p.x[:] = _inside(len(p), 42)
    args = ([g], p, None, 1e-4, I.KPC, MPC, 25 * MPC)
    kw = dict(max_steps=max_steps, calls=3, box=BOX)
    sim, rc = run_gpu(*args, **kw)
    assert rc == 0
    st, _ = run_oracle(*args, **kw)
    assert_bit_identical(sim.state(), st.snapshot())


def test_fp64_reflective_box_graph_loop_bit_identical(oracle_lib):
    import paper_1410_5323_gb300 as crp

    g = _grid(3)
    p = I.make_particles(600, 43, energy=("loguniform", 1e17, 1e20))
    p.x[:] = _inside(len(p), 43)
    sim = crp.Simulation([crp.Field(g, 0.25 * MPC)], None, seed=1, capacity=len(p))
    sim.set_boundary(BOX)
    sim.inject(p)
    sim.propagate_loop(1e-4, I.KPC, MPC, 20 * MPC, max_steps=50, form=crp.FORM_FP64)
    assert sim.sync(timeout_s=300.0, raise_on_error=False) == 0
    st, _ = run_oracle([g], p, None, 1e-4, I.KPC, MPC, 20 * MPC, box=BOX)
    assert_bit_identical(sim.state(), st.snapshot())


def test_fp64_antiparticles_bit_identical_and_time_reversal(oracle_lib):
    """Backward tracking: antinuclei bit for bit against the oracle; and the GPU's own end
    states, reversed, come back to the start."""
    g = _grid(4)
    rng = np.random.default_rng(44)
    p = I.make_particles(1000, 44, species=(("He", .5), ("Fe", .5)), energy=("loguniform", 1e18, 1e20))
    p.x[:] = rng.uniform(0, 8 * MPC, (len(p), 3))
    d = 3 * MPC
    hmin = 1e-3 * I.KPC          # low rigidities need steps below 1 kpc to meet tol = 1e-10
    fw, rc = run_gpu([g], p, None, 1e-10, hmin, MPC, d)
    assert rc == 0
    a = by_uid(fw.state())
    back = p.take(np.arange(len(p)))
    back.x[:] = np.stack([a["x"], a["y"], a["z"]], 1)
    back.u[:] = -np.stack([a["ux"], a["uy"], a["uz"]], 1)
    back.Z[:] = -p.Z
    bw, rc = run_gpu([g], back, None, 1e-10, hmin, MPC, d)
    assert rc == 0
    st, _ = run_oracle([g], back, None, 1e-10, hmin, MPC, d)
    b = by_uid(bw.state())
    assert_bit_identical(b, st.snapshot())
    xb = np.stack([b["x"], b["y"], b["z"]], 1)
    assert np.max(np.linalg.norm(xb - p.x, axis=1)) < 1e-6 * d


def test_antiparticles_with_tables_rejected_at_injection():
    import paper_1410_5323_gb300 as crp

    p = I.make_particles(4, 45, species=(("He", 1.0),))
    p.Z[:] = -2
    sim = crp.Simulation([crp.Field(_grid(5, 8), 0.25 * MPC)], crp.Tables(I.synthetic_tables()), capacity=8)
    with pytest.raises(crp.CrpError):
        sim.inject(p)


def test_mixed_neutral_particles_bounce_like_the_triangle_wave():
    rng = np.random.default_rng(46)
    n = 256
    u = I.isotropic_directions(n, rng)
    p = I.Particles(_inside(n, 46), u, np.full(n, 1e19), np.ones(n, np.int32), np.zeros(n, np.int32),
                    np.arange(n, dtype=np.int64), np.zeros(n, np.int32))
    g = np.zeros((4, 4, 4, 3), np.float32)
    dmax = 37.3 * MPC
    sim, rc = run_gpu([g], p, None, 1e-4, I.KPC, MPC, dmax, spacing=MPC, form=MIXED, box=BOX)
    assert rc == 0
    a = by_uid(sim.state())
    for ax, c in enumerate("xyz"):
        z = p.x[:, ax] + dmax * u[:, ax]
        m = np.mod((z - BOX[0][ax]) / BOX[1][ax], 2.0)
        xe = np.where(m < 1.0, BOX[0][ax] + m * BOX[1][ax], BOX[0][ax] + (2.0 - m) * BOX[1][ax])
        sgn = np.where(m < 1.0, 1.0, -1.0)
        assert np.allclose(a[c], xe, rtol=0, atol=1e-5 * MPC)
        assert np.allclose(a["u" + c], sgn * u[:, ax], atol=1e-6)
        assert np.allclose(a["u0" + c], sgn * u[:, ax], atol=1e-6)


def test_mixed_reflective_box_statistics(oracle_lib):
    g = _grid(6)
    p = I.make_particles(3000, 47, species=MIX, energy=("power", 1e18, 10 ** 20.5, 2.0))
    p.x[:] = _inside(len(p), 47)
    t = I.synthetic_tables()
    args = ([g], p, t, 1e-4, I.KPC, MPC, 40 * MPC)
    kw = dict(seed=6, capacity=3000 * 56, box=BOX)
    sim, rc = run_gpu(*args, form=MIXED, **kw)
    assert rc == 0
    st, _ = run_oracle(*args, **kw)
    a, b = sim.state(), st.snapshot()
    x = np.stack([a["x"], a["y"], a["z"]], 1)
    assert np.all((x >= BOX[0] - 1e-9 * MPC) & (x <= BOX[0] + BOX[1] + 1e-9 * MPC))
    pa, pb = a["uid"] < 2 ** 32, b["uid"] < 2 ** 32
    for c in ("x", "y", "z"):
        assert stats.ks_2samp(a[c][pa], b[c][pb]).pvalue > 0.01, c
    assert stats.ks_2samp(np.log10(a["E"][pa]), np.log10(b["E"][pb])).pvalue > 0.01


def test_mixed_backtracking_returns_close_to_the_start():
    g = _grid(7)
    rng = np.random.default_rng(48)
    p = I.make_particles(500, 48, energy=("fixed", 10 ** 19.5))
    p.x[:] = rng.uniform(0, 8 * MPC, (len(p), 3))
    d = 1 * MPC
    fw, rc = run_gpu([g], p, None, 1e-6, I.KPC, MPC, d, form=MIXED)
    assert rc == 0
    a = by_uid(fw.state())
    back = p.take(np.arange(len(p)))
    back.x[:] = np.stack([a["x"], a["y"], a["z"]], 1)
    back.u[:] = -np.stack([a["ux"], a["uy"], a["uz"]], 1)
    back.Z[:] = -p.Z
    bw, rc = run_gpu([g], back, None, 1e-6, I.KPC, MPC, d, form=MIXED)
    assert rc == 0
    b = by_uid(bw.state())
    xb = np.stack([b["x"], b["y"], b["z"]], 1)
    assert np.median(np.linalg.norm(xb - p.x, axis=1)) < 1e-4 * d
