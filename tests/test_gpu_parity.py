"""GPU FP64 form vs the FP64 CPU oracle through the C ABI: bit-identical particle state
(positions, directions, energies, species, optical depth, counters, secondaries)."""
import numpy as np
import pytest

import oracle as O
from paper_1410_5323_gb300 import inputs as I
from _parity import assert_bit_identical, by_uid, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

MIX = (("H", .4), ("He", .3), ("N", .2), ("Fe", .1))


@pytest.fixture(scope="module")
def c1():
    w = I.workload("fp64_64cube_1k_protons")
    g = I.kolmogorov_grid(w.grid_n, w.spacing_m, w.lmin_cells, w.lmax_cells, w.brms_t, w.grid_seed)
    return w, g.astype(np.float32), I.make_particles(w.n_particles, w.particle_seed, w.species, w.energy)


def test_first_200_steps_bit_identical(c1, oracle_lib):
    """The paper-scale 64^3 case: state after 200 accepted steps per particle."""
    w, g, p = c1
    args = ([g], p, None, w.tol, w.hmin_m, w.hmax_m, w.dmax_m)
    sim, rc = run_gpu(*args, max_steps=200)
    assert rc == 0
    st, orc = run_oracle(*args, max_steps=200)
    assert orc == 0
    assert_bit_identical(sim.state(), st.snapshot())


def test_full_distance_bit_identical(c1, oracle_lib):
    w, g, p = c1
    args = ([g], p, None, w.tol, w.hmin_m, w.hmax_m, w.dmax_m)
    sim, rc = run_gpu(*args)
    assert rc == 0
    st, orc = run_oracle(*args)
    gs = sim.state()
    assert np.all(gs["status"] == O.DONE) and np.all(gs["s"] == w.dmax_m)
    assert_bit_identical(gs, st.snapshot())


def test_interactions_and_secondaries_bit_identical(oracle_lib):
    g = I.kolmogorov_grid(32, 0.25 * I.MPC, 2, 16, 1e-13, 5).astype(np.float32)
    p = I.make_particles(1500, 11, species=MIX, energy=("power", 1e18, 10 ** 20.5, 2.0))
    t = I.synthetic_tables()
    args = ([g], p, t, 1e-4, I.KPC, I.MPC, 60 * I.MPC)
    sim, rc = run_gpu(*args, seed=3, capacity=1500 * 56)
    assert rc == 0
    st, orc = run_oracle(*args, seed=3, capacity=1500 * 56)
    assert orc == 0
    gs = sim.state()
    assert np.sum(gs["uid"] >= 2 ** 32) > 50          # secondaries were produced
    assert_bit_identical(gs, st.snapshot())


def test_high_interaction_rate_bookkeeping(oracle_lib):
    """Many splits per primary: integer state and queue contents (as a uid multiset)."""
    g = I.kolmogorov_grid(16, 0.25 * I.MPC, 2, 8, 1e-13, 6).astype(np.float32)
    p = I.make_particles(300, 12, species=(("Fe", 1.0),), energy=("fixed", 1e21))
    t = I.constant_rate_tables(loss_rate=1 / (300 * I.MPC), pd_rate=1 / (2 * I.MPC))
    args = ([g], p, t, 1e-4, I.KPC, I.MPC, 40 * I.MPC)
    sim, rc = run_gpu(*args, seed=9, capacity=300 * 56)
    assert rc == 0
    st, _ = run_oracle(*args, seed=9, capacity=300 * 56)
    gs = sim.state()
    assert_bit_identical(gs, st.snapshot())
    sec = gs["uid"] >= 2 ** 32
    assert sim.counts()["secondaries"] == int(sec.sum()) == int(gs["n_int"][~sec].sum())


@pytest.mark.parametrize("max_steps", [1, 37])
def test_budgeted_calls_resume_bit_identically(oracle_lib, max_steps):
    g = I.kolmogorov_grid(16, 0.25 * I.MPC, 2, 8, 1e-13, 2).astype(np.float32)
    p = I.make_particles(200, 4, species=MIX, energy=("power", 1e19, 1e21, 2.0))
    t = I.synthetic_tables()
    calls = 4 if max_steps == 37 else 3
    args = ([g], p, t, 1e-4, I.KPC, I.MPC, 10 * I.MPC)
    sim, rc = run_gpu(*args, capacity=200 * 56, max_steps=max_steps, calls=calls)
    assert rc == 0
    st, _ = run_oracle(*args, capacity=200 * 56, max_steps=max_steps, calls=calls)
    assert_bit_identical(sim.state(), st.snapshot())


def test_queue_full_then_reserve_resumes(oracle_lib):
    import paper_1410_5323_gb300 as crp

    g = I.kolmogorov_grid(16, 0.25 * I.MPC, 2, 8, 1e-13, 2).astype(np.float32)
    p = I.make_particles(64, 5, species=(("Fe", 1.0),), energy=("fixed", 1e21))
    t = I.constant_rate_tables(pd_rate=1 / (5 * I.MPC))
    f = crp.Field(g, 0.25 * I.MPC)
    sim = crp.Simulation([f], crp.Tables(t), seed=2, capacity=70)
    sim.inject(p)
    sim.propagate(1e-4, I.KPC, I.MPC, 30 * I.MPC)
    assert sim.sync(60.0, raise_on_error=False) == crp.api.ERR_QUEUE_FULL
    sim.reserve(64 * 56)
    sim.propagate(1e-4, I.KPC, I.MPC, 30 * I.MPC)
    assert sim.sync(60.0, raise_on_error=False) == 0
    st, _ = run_oracle([g], p, t, 1e-4, I.KPC, I.MPC, 30 * I.MPC, seed=2, capacity=64 * 56)
    assert_bit_identical(sim.state(), st.snapshot())


@pytest.mark.parametrize("n", [1, 31, 33, 129])
def test_ragged_batches(oracle_lib, n):
    g = I.kolmogorov_grid(16, 0.25 * I.MPC, 2, 8, 1e-13, 3).astype(np.float32)
    p = I.make_particles(n, 20 + n, species=MIX, energy=("power", 1e19, 1e21, 2.0))
    t = I.synthetic_tables()
    args = ([g], p, t, 1e-4, I.KPC, I.MPC, 15 * I.MPC)
    sim, rc = run_gpu(*args, capacity=n * 56)
    st, _ = run_oracle(*args, capacity=n * 56)
    assert_bit_identical(sim.state(), st.snapshot())


def test_non_power_of_two_grid_and_origin(oracle_lib):
    rng = np.random.default_rng(3)
    g = (rng.standard_normal((12, 10, 14, 3)) * 1e-13).astype(np.float32)
    p = I.make_particles(100, 8, energy=("power", 1e18, 1e20, 2.0))
    p.x[:] = [3.3e22, -1.7e22, 5.0e21]
    args = ([g], p, None, 1e-4, I.KPC, I.MPC, 30 * I.MPC)
    kw = dict(spacing=0.3 * I.MPC, origin=(-1e22, 2e21, 7e21))
    sim, _ = run_gpu(*args, **kw)
    st, _ = run_oracle(*args, **kw)
    assert_bit_identical(sim.state(), st.snapshot())


@pytest.mark.parametrize("dt", ["f64", "bf16", "f16"])
def test_grid_storage_types(oracle_lib, dt):
    g = I.kolmogorov_grid(16, 0.25 * I.MPC, 2, 8, 1.0, 4)      # unit rms, scaled below
    p = I.make_particles(64, 9, energy=("power", 1e18, 1e20, 2.0))
    if dt == "f64":
        grid, kw = g * 1e-13, {}
    elif dt == "bf16":
        bits = (g.astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)
        grid, kw = bits, dict(dtype=O.BF16, scale=1e-13)
    else:
        grid, kw = g.astype(np.float16).view(np.uint16), dict(dtype=O.F16, scale=1e-13)
    args = ([grid], p, None, 1e-4, I.KPC, I.MPC, 30 * I.MPC)
    sim, _ = run_gpu(*args, **kw)
    st, _ = run_oracle(*args, **kw)
    assert_bit_identical(sim.state(), st.snapshot())


@pytest.mark.parametrize("mixed_sizes", [False, True])
def test_several_grids_by_grid_id(oracle_lib, mixed_sizes):
    """All power-of-two grids take the kernels that wrap indices with a mask; one grid of
    other sizes among them switches the launch to the general wrap for all."""
    grids = [I.kolmogorov_grid(16, 0.25 * I.MPC, 2, 8, b, s).astype(np.float32)
             for s, b in ((1, 1e-13), (2, 5e-13), (3, 2e-14))]
    if mixed_sizes:
        grids[1] = (np.random.default_rng(11).standard_normal((12, 16, 10, 3)) * 3e-13).astype(np.float32)
    p = I.make_particles(300, 10, energy=("loguniform", 1e17, 1e20))
    p.grid_id[:] = np.arange(300) % 3
    args = (grids, p, None, 1e-4, I.KPC, I.MPC, 20 * I.MPC)
    sim, _ = run_gpu(*args)
    st, _ = run_oracle(*args)
    assert_bit_identical(sim.state(), st.snapshot())


def test_neutral_and_proton_secondary_species(oracle_lib):
    g = I.kolmogorov_grid(16, 0.25 * I.MPC, 2, 8, 1e-13, 5).astype(np.float32)
    p = I.make_particles(64, 13)
    p.Z[:32] = 0                                   # neutrons
    args = ([g], p, I.synthetic_tables(), 1e-4, I.KPC, I.MPC, 25 * I.MPC)
    sim, _ = run_gpu(*args)
    st, _ = run_oracle(*args)
    assert_bit_identical(sim.state(), st.snapshot())


def test_block_size_and_cadence_do_not_change_results(oracle_lib):
    g = I.kolmogorov_grid(16, 0.25 * I.MPC, 2, 8, 1e-13, 7).astype(np.float32)
    p = I.make_particles(500, 14, species=MIX, energy=("power", 1e19, 1e21, 2.0))
    t = I.synthetic_tables()
    args = ([g], p, t, 1e-4, I.KPC, I.MPC, 15 * I.MPC)
    ref = None
    for bs, cad in ((32, 1), (128, 4), (256, 16)):
        sim, _ = run_gpu(*args, capacity=500 * 56, block_size=bs, cadence=cad)
        s = by_uid(sim.state())
        if ref is None:
            ref = s
        else:
            for k in ref:
                assert np.array_equal(ref[k], s[k]), (bs, cad, k)


def test_nan_in_field_reports_status_not_hang(oracle_lib):
    import paper_1410_5323_gb300 as crp

    g = np.zeros((8, 8, 8, 3), dtype=np.float32)
    g[...] = [0, 0, 1e-13]
    g[3, 3, 3, 0] = np.nan
    p = I.make_particles(32, 15)
    f = crp.Field(g, 0.25 * I.MPC)
    sim = crp.Simulation([f], None, capacity=32)
    sim.inject(p)
    sim.propagate(1e-4, I.KPC, I.MPC, 50 * I.MPC)
    assert sim.sync(60.0, raise_on_error=False) == crp.api.ERR_NAN_STATE
    st = sim.state()
    assert np.any(st["status"] == crp.STATUS_NAN)
    assert np.all(np.isin(st["status"], [crp.STATUS_NAN, crp.STATUS_DONE]))


def test_observer_records_match_state(oracle_lib):
    import paper_1410_5323_gb300 as crp

    g = I.kolmogorov_grid(16, 0.25 * I.MPC, 2, 8, 1e-13, 8).astype(np.float32)
    p = I.make_particles(100, 16, species=MIX, energy=("power", 1e19, 1e21, 2.0))
    f = crp.Field(g, 0.25 * I.MPC)
    sim = crp.Simulation([f], crp.Tables(I.synthetic_tables()), capacity=100 * 56)
    sim.inject(p)
    sim.propagate(1e-4, I.KPC, I.MPC, 10 * I.MPC)
    sim.sync(60.0)
    obs = by_uid(sim.observe())
    st = by_uid(sim.state())
    assert len(obs["uid"]) == sim.counts()["n_done"] == len(st["uid"])
    for k in obs:
        assert np.array_equal(obs[k], st[k]), k
    # pinned host columns (written by the gather kernel directly), device columns and pageable
    # host columns (staged) give the same records; a window of the finished list too
    n = sim.counts()["n_done"]
    ref = sim.observe()
    for kind in ("pinned", "device"):
        out = (sim.observe_buffers(n + 7, pinned=True) if kind == "pinned"
               else sim.observe_buffers(n + 7, device="cuda"))
        got = sim.observe(out=out)
        for k in ref:
            v = got[k].cpu().numpy() if hasattr(got[k], "cpu") else got[k]
            assert np.array_equal(v, ref[k]), (kind, k)
    first, cnt = 3, max(n - 10, 1)
    out = sim.observe_buffers(cnt, pinned=True)
    got = sim.observe(first=first, capacity=cnt, out=out)
    for k in ref:
        assert np.array_equal(got[k].numpy(), ref[k][first:first + cnt]), ("window", k)


def test_device_columns_inject_like_host(oracle_lib):
    import torch

    import paper_1410_5323_gb300 as crp

    g = I.kolmogorov_grid(16, 0.25 * I.MPC, 2, 8, 1e-13, 9).astype(np.float32)
    p = I.make_particles(128, 17, species=MIX, energy=("power", 1e19, 1e21, 2.0))
    t = I.synthetic_tables()
    f = crp.Field(torch.from_numpy(g).cuda(), 0.25 * I.MPC)
    sim = crp.Simulation([f], crp.Tables(t), capacity=128 * 56)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    sim.inject(x=d(p.x), u=d(p.u), E=d(p.E), A=d(p.A), Z=d(p.Z), uid=d(p.uid))
    sim.propagate(1e-4, I.KPC, I.MPC, 12 * I.MPC)
    sim.sync(60.0)
    st, _ = run_oracle([g], p, t, 1e-4, I.KPC, I.MPC, 12 * I.MPC, capacity=128 * 56)
    assert_bit_identical(sim.state(), st.snapshot())


def test_invalid_arguments_rejected():
    import paper_1410_5323_gb300 as crp

    g = np.zeros((4, 4, 4, 3), dtype=np.float32)
    f = crp.Field(g, I.MPC)
    sim = crp.Simulation([f], crp.Tables(I.synthetic_tables()), capacity=4)
    bad = I.make_particles(2, 1)
    bad.A[0], bad.Z[0] = 60, 30                    # outside the tables
    with pytest.raises(crp.CrpError) as e:
        sim.inject(bad)
    assert e.value.code == crp.api.ERR_INVALID_ARG
    with pytest.raises(crp.CrpError):
        sim.inject(I.make_particles(5, 1))         # above capacity
    # every kind of invalid host particle is refused before the device is touched, wherever
    # it sits in the batch
    for field, value, where in (("A", 0, 1), ("Z", 2, 0), ("Z", -1, 1), ("uid", -1, 1),
                                ("uid", 1 << 32, 0), ("grid_id", 1, 1), ("grid_id", -1, 0)):
        bad = I.make_particles(2, 1)
        getattr(bad, field)[where] = value
        with pytest.raises(crp.CrpError) as e:
            sim.inject(bad)
        assert e.value.code == crp.api.ERR_INVALID_ARG, (field, value)
        assert sim.counts()["n_used"] == 0, (field, value)
    sim.inject(I.make_particles(2, 1))             # a valid batch still goes in
    assert sim.counts()["n_used"] == 2
    with pytest.raises(crp.CrpError):
        sim.propagate(-1.0, I.KPC, I.MPC, I.MPC)
    with pytest.raises(crp.CrpError):
        sim.propagate(1e-4, I.MPC, I.KPC, I.MPC)   # max step below min step


def test_invalid_particle_in_large_host_batch_rejected():
    """Batches of 2^21 and more are validated by several host threads; an invalid particle in
    any chunk (first, inner boundary, last) is still refused before the device is touched."""
    import paper_1410_5323_gb300 as crp

    n = (1 << 21) + 5
    g = np.zeros((4, 4, 4, 3), dtype=np.float32)
    sim = crp.Simulation([crp.Field(g, I.MPC)], None, capacity=n)
    p = I.make_particles(n, 3)
    for where in (0, n // 2, n - 1):
        A = p.A.copy()
        A[where] = 0
        q = I.Particles(p.x, p.u, p.E, A, p.Z, p.uid, p.grid_id)
        with pytest.raises(crp.CrpError) as e:
            sim.inject(q)
        assert e.value.code == crp.api.ERR_INVALID_ARG, where
        assert sim.counts()["n_used"] == 0, where
    sim.inject(p)
    assert sim.counts()["n_used"] == n


def test_full_size_workload_sampled_bit_identical(oracle_lib):
    """The whole 10^6-nuclei 256^3 batch in the launch configuration the benchmark times;
    256 primaries spread over the batch, with every secondary they produced, are checked bit
    for bit against the oracle run on those primaries alone (particles are independent)."""
    w = I.workload("fp64_256cube_1M_nuclei")
    g = I.kolmogorov_grid(w.grid_n, w.spacing_m, w.lmin_cells, w.lmax_cells, w.brms_t,
                          w.grid_seed).astype(np.float32)
    t = I.synthetic_tables()
    p = I.make_particles(w.n_particles, w.particle_seed, w.species, w.energy)
    cap = int(len(p) + np.sum(p.A.astype(np.int64) - 1))
    sim, rc = run_gpu([g], p, t, w.tol, w.hmin_m, w.hmax_m, w.dmax_m, seed=w.rng_seed, capacity=cap)
    assert rc == 0
    gs = sim.state()
    pick = np.sort(np.random.default_rng(0).choice(len(p), 256, replace=False))
    sub = p.take(pick)
    st, orc = run_oracle([g], sub, t, w.tol, w.hmin_m, w.hmax_m, w.dmax_m, seed=w.rng_seed,
                         capacity=int(256 * 56))
    assert orc == 0
    o = st.snapshot()
    root = np.where(gs["uid"] < 2 ** 32, gs["uid"], (gs["uid"] - 2 ** 32) // 64)
    keep = np.isin(root, pick)
    assert_bit_identical({k: v[keep] for k, v in gs.items()}, o)
    assert np.all(gs["status"] == O.DONE)
