"""Sec. 4 sources (Eq. 1 spectrum drawn on the device) and arrival maps (Fig. 4, HEALPix RING
pixels of -u): species, energies, directions, uids and pixel indices bit for bit against the
oracle; whole sampled-then-propagated batches bit for bit; large-sample statistics against
the quadrature CDFs of Eq. 1."""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import oracle as O
from paper_1410_5323_gb300 import inputs as I
from _parity import assert_bit_identical

pytestmark = pytest.mark.gpu
MPC = I.MPC
EQ1 = [(1, 1, 1.0), (4, 2, 0.5), (14, 7, 0.3), (56, 26, 0.1)]
RCUT = 10 ** 19.8


def _sim(n, seed=3, tables=None, grid=None, cap=None):
    import paper_1410_5323_gb300 as crp

    g = grid if grid is not None else I.kolmogorov_grid(16, 0.25 * MPC, 2, 8, 1e-13, 1).astype(np.float32)
    return crp.Simulation([crp.Field(g, 0.25 * MPC)], None if tables is None else crp.Tables(tables),
                          seed=seed, capacity=cap or n), g


def _particles_from(A, Z, E, u, x, uid0=0):
    n = len(A)
    return I.Particles(np.ascontiguousarray(x), np.ascontiguousarray(u), E.copy(), A.copy(), Z.copy(),
                       np.arange(n, dtype=np.int64) + uid0, np.zeros(n, np.int32))


def test_sampled_species_energies_directions_bit_identical():
    import paper_1410_5323_gb300 as crp

    n = 50_000
    x = np.random.default_rng(51).uniform(0, 4 * MPC, (n, 3))
    sim, _ = _sim(n, seed=77)
    spec = crp.Spectrum.of(EQ1, 1.8, RCUT, 1e18, 1e21)
    sim.sample_sources(spec, x)
    s = sim.state()
    A, Z, E, u, failed = O.source_sample(O.spectrum(EQ1, 1.8, RCUT, 1e18, 1e21), 77, 0, n)
    assert failed == 0
    assert np.array_equal(s["uid"], np.arange(n))
    assert np.array_equal(s["A"], A) and np.array_equal(s["Z"], Z)
    assert np.array_equal(s["E"], E)
    for c, k in (("ux", 0), ("uy", 1), ("uz", 2)):
        assert np.array_equal(s[c], u[:, k]) and np.array_equal(s["u0" + c[1]], u[:, k])
    assert np.array_equal(s["x"], x[:, 0])
    assert np.all(s["status"] == O.ACTIVE)
    # a second call continues the uids
    sim.reserve(n + 100)
    sim.sample_sources(spec, x[:100])
    s2 = sim.state()
    A2, _, E2, _, _ = O.source_sample(O.spectrum(EQ1, 1.8, RCUT, 1e18, 1e21), 77, n, 100)
    assert np.array_equal(s2["uid"][n:], np.arange(n, n + 100)) and np.array_equal(s2["E"][n:], E2)


def test_sampled_then_propagated_batch_bit_identical(oracle_lib):
    import paper_1410_5323_gb300 as crp
    import torch

    n = 1500
    t = I.synthetic_tables()
    x = np.random.default_rng(52).uniform(0, 4 * MPC, (n, 3))
    sim, g = _sim(n, seed=9, tables=t, cap=n * 56)
    spec = crp.Spectrum.of(EQ1, 1.8, RCUT, 1e18, 1e21)
    sim.sample_sources(spec, torch.from_numpy(x).cuda())          # device position columns
    sim.propagate(1e-4, I.KPC, MPC, 20 * MPC)
    assert sim.sync(timeout_s=300.0, raise_on_error=False) == 0
    A, Z, E, u, _ = O.source_sample(O.spectrum(EQ1, 1.8, RCUT, 1e18, 1e21), 9, 0, n)
    st = O.OracleState(n * 56)
    ot = O.OracleTables(t)
    O.inject(st, _particles_from(A, Z, E, u, x), 9, ot)
    rc, _ = O.propagate(st, [O.OracleField(g, 0.25 * MPC)], ot, 1e-4, I.KPC, MPC, 20 * MPC, seed=9)
    assert rc == 0
    assert_bit_identical(sim.state(), st.snapshot())


def test_large_sample_follows_eq1():
    import paper_1410_5323_gb300 as crp

    n = 1_000_000
    sim, _ = _sim(n, seed=5)
    sim.sample_sources(crp.Spectrum.of(EQ1, 1.8, RCUT, 1e18, 1e21), np.zeros((n, 3)))
    s = sim.state()
    f = lambda le, zr: math.exp(-0.8 * le - math.exp(le) / zr)
    w = np.array([x * a ** 0.8 * integrate.quad(f, math.log(1e18), math.log(1e21), args=(z * RCUT,),
                                                limit=200)[0] for a, z, x in EQ1])
    p = w / w.sum()
    counts = np.array([np.sum(s["A"] == a) for a, _, _ in EQ1])
    assert np.all(np.abs(counts - n * p) < 4.5 * np.sqrt(n * p * (1 - p))), (counts, n * p)
    for a, z, _ in EQ1:
        sel = s["E"][s["A"] == a][:3000]
        tot = integrate.quad(f, math.log(1e18), math.log(1e21), args=(z * RCUT,), limit=200)[0]
        cdf = lambda e: np.array([integrate.quad(f, math.log(1e18), math.log(v), args=(z * RCUT,),
                                                 limit=200)[0] / tot for v in np.atleast_1d(e)])
        assert stats.kstest(sel, cdf).pvalue > 0.01, a
    u = np.stack([s["ux"], s["uy"], s["uz"]], 1)
    assert np.all(np.abs(u.mean(0)) < 4.5 * math.sqrt(1 / 3 / n))


def test_unreachable_cutoff_is_reported_at_sync():
    import paper_1410_5323_gb300 as crp

    sim, _ = _sim(8)
    sim.sample_sources(crp.Spectrum.of([(1, 1, 1.0)], 1.8, 1e15, 1e19, 1e21), np.zeros((8, 3)))
    with pytest.raises(crp.CrpError):
        sim.sync(timeout_s=60.0)


def _hard_directions(nside, rng):
    """Pixel centres, points on the ring-zone borders and the cap/belt seams, nudged by a few
    ulp, plus random directions and degenerate ones."""
    out = [rng.standard_normal((20000, 3))]
    z = np.concatenate([np.full(400, 2 / 3), np.full(400, -2 / 3), np.nextafter(np.full(200, 2 / 3), 1),
                        np.nextafter(np.full(200, 2 / 3), 0), np.zeros(200)])
    phi = rng.integers(0, 8 * nside, len(z)) * (math.pi / (4 * nside))
    s = np.sqrt(1 - z * z)
    out.append(np.stack([s * np.cos(phi), s * np.sin(phi), z], 1))
    out.append(np.array([[0, 0, 1.0], [0, 0, -1.0], [1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0],
                         [1, 1, 0], [-1, -1e-300, 0], [0, 0, 0]]))
    return np.concatenate(out)


@pytest.mark.parametrize("nside", [1, 2, 8, 64, 1024, 8192])
def test_healpix_pixels_bit_identical(oracle_lib, nside):
    import paper_1410_5323_gb300 as crp
    import torch

    u = _hard_directions(nside, np.random.default_rng(nside))
    pg = crp.healpix_ring(nside, torch.from_numpy(u).cuda()).cpu().numpy()
    po = O.healpix_ring(nside, u)
    assert np.array_equal(pg, po)
    assert pg[-1] == -1 and pg.min() >= -1 and pg.max() < 12 * nside * nside


@pytest.mark.parametrize("nside", [8, 128])
def test_arrival_map_matches_oracle(oracle_lib, nside):
    """nside 8 bins through a shared-memory copy of the map, nside 128 straight to global."""
    import paper_1410_5323_gb300 as crp

    n = 4000
    x = np.random.default_rng(53).uniform(0, 4 * MPC, (n, 3))
    sim, g = _sim(n, seed=11)
    sim.sample_sources(crp.Spectrum.of(EQ1, 1.8, RCUT, 1e18, 1e21), x)
    sim.propagate(1e-4, I.KPC, MPC, 15 * MPC, max_steps=60)           # some stay active
    assert sim.sync(timeout_s=300.0, raise_on_error=False) == 0
    s = sim.state()
    m = sim.arrival_map(nside, 10 ** 18.7).cpu().numpy()
    st = O.OracleState(n)
    O.inject(st, I.Particles(np.stack([s["x"], s["y"], s["z"]], 1), np.stack([s["ux"], s["uy"], s["uz"]], 1),
                             s["E"], s["A"], s["Z"], s["uid"], s["grid_id"]), 11, None)
    st.status[:n] = s["status"]
    ref = O.arrival_map(st, nside, 10 ** 18.7)
    assert np.array_equal(m.astype(np.uint64), ref)
    keep = (s["status"] == O.DONE) & (s["E"] > 10 ** 18.7)
    assert 0 < m.sum() == keep.sum() < n


def test_full_size_sec4_workload_sampled_bit_identical_and_map(oracle_lib):
    """The whole Sec. 4 batch as the benchmark runs it (FP64 form): 10^6 primaries drawn from
    Eq. 1 on the device at density-weighted positions, the 440^3 x 256^3 modulated field in its
    reflective box, then the nside-64 arrival map above 10^18.7 eV. 96 primaries spread over
    the batch, with their secondaries, bit for bit against the oracle; the map against the
    oracle's pixels of every finished particle's final direction."""
    import paper_1410_5323_gb300 as crp

    w = I.workload("sec4_eq1_440cube_x_256cube_1M_nuclei")
    g = I.kolmogorov_grid(w.grid_n, w.spacing_m, w.lmin_cells, w.lmax_cells, w.brms_t,
                          w.grid_seed).astype(np.float32)
    rho = I.density_field(w.mod_n, w.mod_lmin_cells, w.mod_lmax_cells, w.mod_sigma_ln, w.mod_seed)
    m = I.modulation_from_density(rho)
    x = I.density_positions(w.n_particles, rho, w.mod_spacing_m, w.particle_seed)
    del rho
    t = I.synthetic_tables()
    f = crp.Field(g, w.spacing_m).modulate(m, w.mod_spacing_m)
    cap = w.n_particles * 56
    sim = crp.Simulation([f], crp.Tables(t), seed=w.rng_seed, capacity=cap)
    sim.set_boundary(I.workload_box(w))
    sim.sample_sources(crp.Spectrum.of(*w.spectrum), x)
    sim.propagate(w.tol, w.hmin_m, w.hmax_m, w.dmax_m)
    assert sim.sync(timeout_s=900.0, raise_on_error=False) == 0
    amap = sim.arrival_map(w.arrival_nside, w.arrival_emin_ev).cpu().numpy()
    gs = sim.state()
    assert np.all(gs["status"] == O.DONE)
    # sampled primaries: the oracle draws them itself from the same counters
    pick = np.sort(np.random.default_rng(0).choice(w.n_particles, 96, replace=False))
    sp = O.spectrum(*w.spectrum)
    rows = [O.source_sample(sp, w.rng_seed, int(k), 1) for k in pick]
    sub = I.Particles(x[pick].copy(), np.concatenate([r[3] for r in rows]), np.concatenate([r[2] for r in rows]),
                      np.concatenate([r[0] for r in rows]), np.concatenate([r[1] for r in rows]),
                      pick.astype(np.int64), np.zeros(len(pick), np.int32))
    st = O.OracleState(96 * 56)
    ot = O.OracleTables(t)
    O.inject(st, sub, w.rng_seed, ot)
    rc, _ = O.propagate(st, [O.OracleField(g, w.spacing_m, modulation=m, mod_spacing=w.mod_spacing_m)], ot,
                        w.tol, w.hmin_m, w.hmax_m, w.dmax_m, seed=w.rng_seed, box=I.workload_box(w))
    assert rc == 0
    root = np.where(gs["uid"] < 2 ** 32, gs["uid"], (gs["uid"] - 2 ** 32) // 64)
    keep = np.isin(root, pick)
    assert_bit_identical({k: v[keep] for k, v in gs.items()}, st.snapshot())
    # the map over the whole batch
    sel = gs["E"] > w.arrival_emin_ev
    u = -np.stack([gs["ux"][sel], gs["uy"][sel], gs["uz"][sel]], 1)
    ref = np.bincount(O.healpix_ring(w.arrival_nside, u), minlength=12 * w.arrival_nside ** 2)
    assert np.array_equal(amap, ref) and amap.sum() == sel.sum() > 0
