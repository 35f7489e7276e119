"""Modulated grids (paper Sec. 3.2, used so in Sec. 4): B(x) = M(x) b(x), a periodic vector
grid times a periodic scalar modulation grid on its own spacing and origin. The FP64 form is
compared bit for bit with the oracle on every particle column (secondaries included); the
precision form per particle over short distances and by two-sample KS over full distances."""
import numpy as np
import pytest
from scipy import stats

import oracle as O
from paper_1410_5323_gb300 import inputs as I
from _parity import assert_bit_identical, by_uid, run_gpu, run_oracle

pytestmark = pytest.mark.gpu
MIXED = 1
MIX = (("H", .4), ("He", .3), ("N", .2), ("Fe", .1))
VSP = 50.0 * I.KPC                       # vector grid spacing
MSP = 300.0 * I.KPC                      # modulation grid spacing
MORG = (-0.37 * I.MPC, 0.11 * I.MPC, 0.5 * I.MPC)
VORG = (0.013 * I.MPC, -0.02 * I.MPC, 0.0)


def _deflection_deg(d):
    u = np.stack([d["ux"], d["uy"], d["uz"]], 1)
    u0 = np.stack([d["u0x"], d["u0y"], d["u0z"]], 1)
    return np.degrees(np.arctan2(np.linalg.norm(np.cross(u, u0), axis=1), np.sum(u * u0, 1)))


def _angle_deg(a, b):
    ua = np.stack([a["ux"], a["uy"], a["uz"]], 1)
    ub = np.stack([b["ux"], b["uy"], b["uz"]], 1)
    c = np.cross(ua, ub)
    return np.degrees(np.arctan2(np.linalg.norm(c, axis=1), np.sum(ua * ub, 1)))


def _case(n_particles, mod_shape=(20, 18, 22), seed=3, vec_n=24):
    """Vector grid vec_n^3 (FP32, 50 kpc, Kolmogorov 100 kpc .. 600 kpc), modulation of
    mod_shape (300 kpc, log-normal density^(2/3)), nuclei placed like the density."""
    g = I.kolmogorov_grid(vec_n, VSP, 2.0, 12.0, 1e-13, seed).astype(np.float32)
    nm = max(mod_shape) + (max(mod_shape) % 2)
    rho = I.density_field(nm, 2.0, 8.0, 1.0, seed + 1)[:mod_shape[0], :mod_shape[1], :mod_shape[2]]
    m = I.modulation_from_density(np.ascontiguousarray(rho))
    p = I.make_particles(n_particles, seed + 2, species=MIX, energy=("power", 1e18, 10 ** 20.5, 2.0))
    p.x[:] = I.density_positions(n_particles, rho, MSP, seed, origin_m=MORG)
    return g, m, p


MODKW = dict(spacing=VSP, origin=VORG, mod_spacing=MSP, mod_origin=MORG)


def test_fp64_modulated_with_interactions_bit_identical(oracle_lib):
    g, m, p = _case(1500)
    t = I.synthetic_tables()
    args = ([g], p, t, 1e-4, I.KPC, I.MPC, 20 * I.MPC)
    kw = dict(seed=3, capacity=1500 * 56, mods=[m], **MODKW)
    sim, rc = run_gpu(*args, **kw)
    assert rc == 0
    st, orc = run_oracle(*args, **kw)
    assert orc == 0
    assert_bit_identical(sim.state(), st.snapshot())
    assert sim.counts()["secondaries"] > 0


@pytest.mark.parametrize("max_steps", [37, 200])
def test_fp64_modulated_budgeted_calls_bit_identical(oracle_lib, max_steps):
    g, m, p = _case(700, seed=5)
    args = ([g], p, None, 1e-4, I.KPC, I.MPC, 8 * I.MPC)
    kw = dict(max_steps=max_steps, calls=3, mods=[m], **MODKW)
    sim, rc = run_gpu(*args, **kw)
    assert rc == 0
    st, _ = run_oracle(*args, **kw)
    assert_bit_identical(sim.state(), st.snapshot())


def test_fp64_pow2_modulation_f64_vector_grid_bit_identical(oracle_lib):
    """Power-of-two modulation dims (mask wrap) and an FP64 vector grid (read directly)."""
    g, m, p = _case(900, mod_shape=(16, 16, 16), seed=7)
    g64 = g.astype(np.float64) * 1.0000001
    args = ([g64], p, None, 1e-4, I.KPC, I.MPC, 10 * I.MPC)
    kw = dict(mods=[m], **MODKW)
    sim, rc = run_gpu(*args, **kw)
    assert rc == 0
    st, _ = run_oracle(*args, **kw)
    assert_bit_identical(sim.state(), st.snapshot())


def test_fp64_two_modulated_fields_by_grid_id(oracle_lib):
    g1, m1, p = _case(1000, seed=9)
    g2, m2, _ = _case(10, seed=10)
    p.grid_id[:] = np.arange(len(p)) % 2
    args = ([g1, g2], p, None, 1e-4, I.KPC, I.MPC, 10 * I.MPC)
    kw = dict(mods=[m1, m2], **MODKW)
    sim, rc = run_gpu(*args, **kw)
    assert rc == 0
    st, _ = run_oracle(*args, **kw)
    assert_bit_identical(sim.state(), st.snapshot())


def test_mixed_modulated_short_distance_matches_oracle(oracle_lib):
    """Before chaos amplifies FP32 rounding, each particle follows the FP64 trajectory."""
    g, m, p = _case(1000, seed=11)
    p.A[:] = 1
    p.Z[:] = 1
    p.E[:] = 10 ** 19.5
    args = ([g], p, None, 1e-4, I.KPC, I.MPC, 1.0 * I.MPC)
    kw = dict(mods=[m], **MODKW)
    sim, rc = run_gpu(*args, form=MIXED, **kw)
    assert rc == 0
    st, _ = run_oracle(*args, **kw)
    a, b = by_uid(sim.state()), by_uid(st.snapshot())
    ang = _angle_deg(a, b)
    assert np.median(ang) < 1e-4 and np.quantile(ang, 0.95) < 0.1
    dx = np.sqrt((a["x"] - b["x"]) ** 2 + (a["y"] - b["y"]) ** 2 + (a["z"] - b["z"]) ** 2)
    assert np.median(dx / I.MPC) < 1e-5
    assert np.all(a["s"] == b["s"])


def test_mixed_modulated_nuclei_statistics_and_bookkeeping(oracle_lib):
    g, m, p = _case(3000, seed=13)
    t = I.synthetic_tables()
    args = ([g], p, t, 1e-4, I.KPC, I.MPC, 30 * I.MPC)
    kw = dict(seed=4, capacity=3000 * 56, mods=[m], **MODKW)
    sim, rc = run_gpu(*args, form=MIXED, **kw)
    assert rc == 0
    st, _ = run_oracle(*args, **kw)
    a, b = sim.state(), st.snapshot()
    prim_a, prim_b = a["uid"] < 2 ** 32, b["uid"] < 2 ** 32
    parent = np.where(prim_a, a["uid"], (a["uid"] - 2 ** 32) // 64)
    assert np.array_equal(np.bincount(parent, weights=a["A"], minlength=3000), p.A.astype(float))
    assert np.array_equal(np.bincount(parent, weights=a["Z"], minlength=3000), p.Z.astype(float))
    assert stats.ks_2samp(_deflection_deg(a)[prim_a], _deflection_deg(b)[prim_b]).pvalue > 0.01
    assert stats.ks_2samp(np.log10(a["E"][prim_a]), np.log10(b["E"][prim_b])).pvalue > 0.01
    assert np.all(a["status"] == O.DONE)


def test_mixed_modulated_bf16_vector_grid_statistics(oracle_lib):
    g, m, p = _case(2000, seed=15)
    bits = (g.view(np.uint32) >> 16).astype(np.uint16)
    args = ([bits], p, None, 1e-4, I.KPC, I.MPC, 20 * I.MPC)
    kw = dict(dtype=O.BF16, scale=1.0, mods=[m], **MODKW)
    sim, rc = run_gpu(*args, form=MIXED, **kw)
    assert rc == 0
    st, _ = run_oracle(*args, **kw)
    assert stats.ks_2samp(_deflection_deg(sim.state()), _deflection_deg(st.snapshot())).pvalue > 0.01


def test_modulation_rules_enforced():
    import paper_1410_5323_gb300 as crp
    from paper_1410_5323_gb300.adjoint import Adjoint

    g, m, _ = _case(10, seed=17)
    plain = crp.Field(g, VSP)
    mod = crp.Field(g, VSP).modulate(m, MSP, MORG)
    with pytest.raises(crp.CrpError):
        crp.Simulation([plain, mod], None, capacity=10)      # all modulated, or none
    with pytest.raises(crp.CrpError):
        mod.modulate(m, MSP)                                 # one modulation per field
    with pytest.raises(TypeError):
        plain.modulate(m.astype(np.float64), MSP)
    with pytest.raises(crp.CrpError):
        Adjoint(mod, 4, 10, 5)


def _full_size():
    w = I.workload("modulated_440cube_300kpc_x_256cube_50kpc_1M_nuclei")
    g = I.kolmogorov_grid(w.grid_n, w.spacing_m, w.lmin_cells, w.lmax_cells, w.brms_t,
                          w.grid_seed).astype(np.float32)
    rho = I.density_field(w.mod_n, w.mod_lmin_cells, w.mod_lmax_cells, w.mod_sigma_ln, w.mod_seed)
    m = I.modulation_from_density(rho)
    p = I.make_particles(w.n_particles, w.particle_seed, w.species, w.energy)
    p.x[:] = I.density_positions(w.n_particles, rho, w.mod_spacing_m, w.particle_seed)
    return w, g, m, p


def test_full_size_modulated_workload_sampled_bit_identical(oracle_lib):
    """The whole 10^6-nuclei batch through the 440^3 x 256^3 modulated field, reflective box of
    the modulation volume, in the launch configuration the benchmark times (FP64 form); 128
    primaries spread over the batch, with every secondary they produced, bit for bit against
    the oracle run on them alone."""
    w, g, m, p = _full_size()
    t = I.synthetic_tables()
    cap = int(len(p) + np.sum(p.A.astype(np.int64) - 1))
    kw = dict(spacing=w.spacing_m, mods=[m], mod_spacing=w.mod_spacing_m, box=I.workload_box(w))
    sim, rc = run_gpu([g], p, t, w.tol, w.hmin_m, w.hmax_m, w.dmax_m, seed=w.rng_seed, capacity=cap, **kw)
    assert rc == 0
    gs = sim.state()
    assert np.all(gs["status"] == O.DONE)
    pick = np.sort(np.random.default_rng(0).choice(len(p), 128, replace=False))
    st, orc = run_oracle([g], p.take(pick), t, w.tol, w.hmin_m, w.hmax_m, w.dmax_m, seed=w.rng_seed,
                         capacity=128 * 56, **kw)
    assert orc == 0
    root = np.where(gs["uid"] < 2 ** 32, gs["uid"], (gs["uid"] - 2 ** 32) // 64)
    keep = np.isin(root, pick)
    assert_bit_identical({k: v[keep] for k, v in gs.items()}, st.snapshot())
