"""Batching form: many field realisations in one persistent launch, the device-side graph
loop of budgeted slices, grid-major ordering; checked against the oracle (bit-exact in the
FP64 form, KS in the precision form) and for clean stops (queue full, slice limit)."""
import numpy as np
import pytest
from scipy import stats

import oracle as O
from paper_1410_5323_gb300 import inputs as I
from _parity import assert_bit_identical, by_uid, run_oracle

pytestmark = pytest.mark.gpu
MIX = (("H", .4), ("He", .3), ("N", .2), ("Fe", .1))


def _sim(grids, parts, tables=None, capacity=None, seed=1):
    import paper_1410_5323_gb300 as crp

    sim = crp.Simulation([crp.Field(g, 0.25 * I.MPC) for g in grids],
                         crp.Tables(tables) if tables is not None else None, seed=seed,
                         capacity=capacity or len(parts))
    sim.inject(parts)
    return sim


@pytest.fixture(scope="module")
def small_batch():
    w = I.workload("batched_64x128cube_12.8M_protons")
    grids, _ = I.batched_grids(w, n_grids=8, grid_n=32)
    parts = I.batched_particles(w, 64, n_grids=8)
    return w, grids, parts


def test_graph_loop_equals_single_call_and_repeated_calls(small_batch):
    w, grids, p = small_batch
    dmax = 15 * I.MPC
    a = _sim(grids, p)
    a.propagate(w.tol, w.hmin_m, w.hmax_m, dmax)
    a.sync(120.0)
    b = _sim(grids, p)
    b.propagate_loop(w.tol, w.hmin_m, w.hmax_m, dmax, max_steps=40)
    b.sync(120.0)
    c = _sim(grids, p)
    for _ in range(400):
        c.propagate(w.tol, w.hmin_m, w.hmax_m, dmax, max_steps=40)
        if c.counts()["n_active"] == 0:
            break
    c.sync(120.0)
    A, B, Cc = by_uid(a.state()), by_uid(b.state()), by_uid(c.state())
    for k in A:
        assert np.array_equal(A[k], B[k]) and np.array_equal(A[k], Cc[k]), k
    assert b.counts()["launches"] > 2 * 5       # several slices ran inside one graph launch


def test_graph_loop_matches_oracle_over_grids(small_batch):
    w, grids, p = small_batch
    dmax = 15 * I.MPC
    b = _sim(grids, p)
    b.propagate_loop(w.tol, w.hmin_m, w.hmax_m, dmax, max_steps=25, order=3)
    b.sync(120.0)
    st, _ = run_oracle(grids, p, None, w.tol, w.hmin_m, w.hmax_m, dmax)
    assert_bit_identical(b.state(), st.snapshot())


def test_graph_loop_reused_and_rebuilt(small_batch):
    w, grids, p = small_batch
    sim = _sim(grids, p)
    for dmax in (5 * I.MPC, 5 * I.MPC, 8 * I.MPC):       # same plan twice, then a new one
        sim.reset()
        sim.inject(p)
        sim.propagate_loop(w.tol, w.hmin_m, w.hmax_m, dmax, max_steps=30)
        sim.sync(120.0)
        assert sim.counts()["n_active"] == 0
        assert np.all(sim.read("s") == dmax)


def test_graph_loop_respects_slice_limit(small_batch):
    w, grids, p = small_batch
    sim = _sim(grids, p)
    sim.propagate_loop(w.tol, w.hmin_m, w.hmax_m, 50 * I.MPC, max_steps=3, max_slices=2)
    sim.sync(120.0)
    c = sim.counts()
    assert c["n_active"] > 0
    assert np.all(sim.read("n_steps") <= 6)


def test_graph_loop_stops_on_full_queue_then_resumes():
    import paper_1410_5323_gb300 as crp

    g = I.kolmogorov_grid(16, 0.25 * I.MPC, 2, 8, 1e-13, 2).astype(np.float32)
    p = I.make_particles(64, 5, species=(("Fe", 1.0),), energy=("fixed", 1e21))
    t = I.constant_rate_tables(pd_rate=1 / (5 * I.MPC))
    sim = _sim([g], p, t, capacity=70, seed=2)
    sim.propagate_loop(1e-4, I.KPC, I.MPC, 30 * I.MPC, max_steps=20)
    assert sim.sync(120.0, raise_on_error=False) == crp.api.ERR_QUEUE_FULL
    sim.reserve(64 * 56)
    sim.propagate_loop(1e-4, I.KPC, I.MPC, 30 * I.MPC, max_steps=20)
    assert sim.sync(120.0, raise_on_error=False) == 0
    st, _ = run_oracle([g], p, t, 1e-4, I.KPC, I.MPC, 30 * I.MPC, seed=2, capacity=64 * 56)
    assert_bit_identical(sim.state(), st.snapshot())


def test_orders_give_identical_results(small_batch):
    w, grids, p = small_batch
    ref = None
    for order in (1, 2, 3):
        sim = _sim(grids, p)
        sim.propagate(w.tol, w.hmin_m, w.hmax_m, 10 * I.MPC, order=order)
        sim.sync(120.0)
        s = by_uid(sim.state())
        if ref is None:
            ref = s
        for k in ref:
            assert np.array_equal(ref[k], s[k]), (order, k)


def test_full_size_batched_workload_sampled(oracle_lib):
    """64 realisations of 128^3 and 12.8M protons in one graph-loop launch of the precision
    form; 100 particles per realisation are rerun by the oracle and their arrival
    distributions compared by KS; every particle must finish."""
    import paper_1410_5323_gb300 as crp

    w = I.workload("batched_64x128cube_12.8M_protons")
    grids, _ = I.batched_grids(w)
    p = I.batched_particles(w, 200_000)
    sim = crp.Simulation([crp.Field(g, w.spacing_m) for g in grids], None, capacity=len(p))
    sim.inject(p)
    sim.propagate_loop(w.tol, w.hmin_m, w.hmax_m, w.dmax_m, max_steps=16000,
                       form=crp.FORM_MIXED, order=3)
    assert sim.sync(1200.0) == 0
    c = sim.counts()
    assert c["n_active"] == 0 and c["n_done"] == len(p)
    pick = (np.arange(64)[:, None] * 200_000 + np.arange(100)[None, :]).ravel()
    gs = {k: sim.read(k)[pick] for k in ("ux", "uy", "uz", "u0x", "u0y", "u0z", "s", "uid")}
    st, _ = run_oracle(grids, p.take(pick), None, w.tol, w.hmin_m, w.hmax_m, w.dmax_m)
    o = st.snapshot()

    def defl(d):
        u = np.stack([d["ux"], d["uy"], d["uz"]], 1)
        u0 = np.stack([d["u0x"], d["u0y"], d["u0z"]], 1)
        return np.degrees(np.arctan2(np.linalg.norm(np.cross(u, u0), axis=1), np.sum(u * u0, 1)))

    assert np.all(gs["s"] == w.dmax_m)
    assert stats.ks_2samp(defl(gs), defl(o)).pvalue > 0.01


def test_switching_orders_on_one_simulation(small_batch):
    """Consecutive calls with different work-list orders on the same simulation (the sort
    scratch is reused) give the same bits as a fresh simulation."""
    w, grids, p = small_batch
    ref = _sim(grids, p)
    ref.propagate(w.tol, w.hmin_m, w.hmax_m, 8 * I.MPC)
    ref.sync(120.0)
    R = by_uid(ref.state())
    sim = _sim(grids, p)
    for order in (2, 3, 2, 1, 3):
        sim.reset()
        sim.inject(p)
        sim.propagate(w.tol, w.hmin_m, w.hmax_m, 8 * I.MPC, order=order)
        assert sim.sync(120.0, raise_on_error=False) == 0
        S = by_uid(sim.state())
        for k in R:
            assert np.array_equal(R[k], S[k]), (order, k)
