"""Precision form (FP32 local-frame stages, double-float positions, FP64 error norm) against
the FP64 oracle. Per-particle agreement is checked where the chaos floor allows it (short
distances); over the full distance the arrival distributions are compared by two-sample KS
(p > 0.01), and nucleon bookkeeping must stay exact."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O
from paper_1410_5323_gb300 import inputs as I
from _parity import by_uid, run_gpu, run_oracle

pytestmark = pytest.mark.gpu
MIXED = 1
MIX = (("H", .4), ("He", .3), ("N", .2), ("Fe", .1))


def _angle_deg(a, b):
    ua = np.stack([a["ux"], a["uy"], a["uz"]], 1)
    ub = np.stack([b["ux"], b["uy"], b["uz"]], 1)
    c = np.cross(ua, ub)
    return np.degrees(np.arctan2(np.linalg.norm(c, axis=1), np.sum(ua * ub, 1)))


def _deflection_deg(d):
    u = np.stack([d["ux"], d["uy"], d["uz"]], 1)
    u0 = np.stack([d["u0x"], d["u0y"], d["u0z"]], 1)
    return np.degrees(np.arctan2(np.linalg.norm(np.cross(u, u0), axis=1), np.sum(u * u0, 1)))


@pytest.fixture(scope="module")
def c1():
    w = I.workload("fp64_64cube_1k_protons")
    g = I.kolmogorov_grid(w.grid_n, w.spacing_m, w.lmin_cells, w.lmax_cells, w.brms_t, w.grid_seed)
    return w, g.astype(np.float32), I.make_particles(w.n_particles, w.particle_seed, w.species, w.energy)


def test_mixed_gyration_closed_form():
    B0, E = 1e-13, 1e19
    rg = E / (299792458.0 * B0)
    g = np.zeros((4, 4, 4, 3), dtype=np.float32)
    g[..., 2] = B0
    p = I.Particles(np.zeros((1, 3)), np.array([[1.0, 0, 0]]), np.array([E]), np.array([1], np.int32),
                    np.array([1], np.int32), np.array([0], np.int64), np.array([0], np.int32))
    dmax = 2 * math.pi * rg
    sim, rc = run_gpu([g], p, None, 1e-6, I.KPC, 10 * I.MPC, dmax, spacing=I.MPC, form=MIXED)
    assert rc == 0
    s = sim.state()
    assert s["status"][0] == O.DONE and s["s"][0] == dmax
    # back at the start after one full turn, to the tolerance-controlled bound
    assert math.hypot(s["x"][0], s["y"][0]) <= 1e-6 * dmax * 10
    assert abs(s["uy"][0]) < 1e-4 and abs(s["ux"][0] - 1.0) < 1e-6


@pytest.mark.parametrize("dist_mpc", [2.0, 5.0])
def test_mixed_short_distance_matches_oracle(c1, dist_mpc):
    """Before chaos amplifies FP32 rounding, each particle follows the FP64 trajectory."""
    w, g, p = c1
    args = ([g], p, None, w.tol, w.hmin_m, w.hmax_m, dist_mpc * I.MPC)
    sim, rc = run_gpu(*args, form=MIXED)
    assert rc == 0
    st, _ = run_oracle(*args)
    a, b = by_uid(sim.state()), by_uid(st.snapshot())
    ang = _angle_deg(a, b)
    assert np.median(ang) < 1e-4 and np.quantile(ang, 0.95) < 0.1
    assert np.all(a["s"] == b["s"])
    dx = np.sqrt((a["x"] - b["x"]) ** 2 + (a["y"] - b["y"]) ** 2 + (a["z"] - b["z"]) ** 2)
    assert np.median(dx / (dist_mpc * I.MPC)) < 1e-5


def test_mixed_full_distance_distributions_match(c1):
    """Full 100 Mpc: deflection-angle distributions agree by two-sample KS."""
    w, g, p = c1
    args = ([g], p, None, w.tol, w.hmin_m, w.hmax_m, w.dmax_m)
    sim, rc = run_gpu(*args, form=MIXED)
    assert rc == 0
    st, _ = run_oracle(*args)
    da, db = _deflection_deg(sim.state()), _deflection_deg(st.snapshot())
    assert stats.ks_2samp(da, db).pvalue > 0.01
    assert np.all(sim.state()["status"] == O.DONE)


def test_mixed_nuclei_with_tables_statistics_and_bookkeeping():
    g = I.kolmogorov_grid(32, 0.25 * I.MPC, 2, 16, 1e-13, 5).astype(np.float32)
    p = I.make_particles(3000, 11, species=MIX, energy=("power", 1e18, 10 ** 20.5, 2.0))
    t = I.synthetic_tables()
    args = ([g], p, t, 1e-4, I.KPC, I.MPC, 60 * I.MPC)
    sim, rc = run_gpu(*args, seed=3, capacity=3000 * 56, form=MIXED)
    assert rc == 0
    st, _ = run_oracle(*args, seed=3, capacity=3000 * 56)
    a, b = sim.state(), st.snapshot()
    prim_a, prim_b = a["uid"] < 2 ** 32, b["uid"] < 2 ** 32
    # exact nucleon bookkeeping for every primary
    parent = np.where(prim_a, a["uid"], (a["uid"] - 2 ** 32) // 64)
    sumA = np.bincount(parent, weights=a["A"], minlength=3000)
    sumZ = np.bincount(parent, weights=a["Z"], minlength=3000)
    assert np.array_equal(sumA, p.A.astype(float)) and np.array_equal(sumZ, p.Z.astype(float))
    assert sim.counts()["secondaries"] == int((~prim_a).sum()) == int(a["n_int"][prim_a].sum())
    # arrival energies of primaries and interaction counts agree statistically
    assert stats.ks_2samp(np.log10(a["E"][prim_a]), np.log10(b["E"][prim_b])).pvalue > 0.01
    assert abs(a["n_int"][prim_a].mean() - b["n_int"][prim_b].mean()) < 0.1 * b["n_int"][prim_b].mean() + 0.05
    assert np.all(a["status"] == O.DONE)


def test_mixed_bf16_grid_statistics():
    g = I.kolmogorov_grid(32, 0.25 * I.MPC, 2, 16, 1.0, 6)
    bits = (g.astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)
    p = I.make_particles(2000, 12, species=(("H", .5), ("Fe", .5)), energy=("power", 1e18, 1e20, 2.0))
    args = ([bits], p, None, 1e-4, I.KPC, I.MPC, 40 * I.MPC)
    kw = dict(dtype=O.BF16, scale=0.5e-13)
    sim, rc = run_gpu(*args, form=MIXED, **kw)
    assert rc == 0
    st, _ = run_oracle(*args, **kw)
    assert stats.ks_2samp(_deflection_deg(sim.state()), _deflection_deg(st.snapshot())).pvalue > 0.01


def test_mixed_budgeted_calls_finish_every_particle(c1):
    w, g, p = c1
    sim, rc = run_gpu([g], p, None, w.tol, w.hmin_m, w.hmax_m, 30 * I.MPC, form=MIXED, max_steps=17,
                      calls=8)
    assert rc == 0
    s = sim.state()
    assert np.all(s["status"] == O.DONE) and np.all(s["s"] == 30 * I.MPC)
