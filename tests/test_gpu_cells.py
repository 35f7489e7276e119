"""Cell-major grid copies for the precision form: the 8 corners of every cell stored together
and read with 256-bit loads. They hold the node grid's values, so the precision form must
give bit-identical results with either layout: FP32 and BF16 grids, non-cubic and
non-power-of-two sizes (periodic wrap baked into the copy), interactions and secondaries,
several grids, modulated fields in a reflective box, budgeted calls and the graph loop."""
import numpy as np
import pytest

import oracle as O
from paper_1410_5323_gb300 import inputs as I
from _parity import assert_bit_identical, run_gpu

pytestmark = pytest.mark.gpu
MIXED = 1
MIX = (("H", .4), ("He", .3), ("N", .2), ("Fe", .1))


def _same(args, all_done=True, **kw):
    import paper_1410_5323_gb300 as crp

    states = []
    for layout in (crp.GRID_NODES, crp.GRID_CELLS, crp.GRID_AUTO):
        sim, rc = run_gpu(*args, form=MIXED, grid_layout=layout, **kw)
        assert rc == 0
        # small grids: AUTO finds room for the copies
        assert sim.grid_layout() == (crp.GRID_NODES if layout == crp.GRID_NODES else crp.GRID_CELLS)
        states.append(sim.state())
        del sim
    assert np.all(states[0]["status"] == O.DONE) or not all_done
    assert_bit_identical(states[1], states[0])
    assert_bit_identical(states[2], states[0])


def _grid(shape, seed, brms=1e-13):
    n = max(shape)
    g = I.kolmogorov_grid(n, 0.25 * I.MPC, 2, 8, brms, seed)
    return np.ascontiguousarray(g[:shape[0], :shape[1], :shape[2]])


def test_f32_non_cubic_grid_with_interactions():
    g = _grid((24, 20, 18), 21).astype(np.float32)
    p = I.make_particles(1500, 31, species=MIX, energy=("power", 1e18, 10 ** 20.5, 2.0))
    _same(([g], p, I.synthetic_tables(), 1e-4, I.KPC, I.MPC, 30 * I.MPC), seed=5, capacity=1500 * 56)


def test_bf16_grid_with_scale():
    g = _grid((16, 32, 24), 22, brms=1.0)
    bits = (g.astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)
    p = I.make_particles(1500, 32, species=(("H", .5), ("Fe", .5)), energy=("power", 1e18, 1e20, 2.0))
    _same(([bits], p, None, 1e-4, I.KPC, I.MPC, 25 * I.MPC), dtype=O.BF16, scale=0.5e-13)


def test_two_modulated_grids_in_a_reflective_box():
    g1 = _grid((20, 20, 20), 23).astype(np.float32)
    g2 = _grid((20, 20, 20), 24).astype(np.float32)
    rng = np.random.default_rng(25)
    mods = [np.exp(rng.normal(0.0, 0.5, (12, 10, 14))).astype(np.float32) for _ in range(2)]
    p = I.make_particles(1200, 33, species=MIX, energy=("power", 1e18, 1e20, 2.0))
    p.grid_id[:] = np.arange(1200) % 2
    box = ((0.0, 0.0, 0.0), (5 * I.MPC, 4.5 * I.MPC, 5.5 * I.MPC))
    p.x[:] = rng.uniform(0.2, 0.8, (1200, 3)) * np.array(box[1])
    _same(([g1, g2], p, None, 1e-4, I.KPC, I.MPC, 20 * I.MPC), mods=mods, mod_spacing=0.4 * I.MPC, box=box)


def test_budgeted_calls():
    g = _grid((16, 16, 16), 26).astype(np.float32)
    p = I.make_particles(800, 34, species=MIX, energy=("power", 1e18, 1e20, 2.0))
    _same(([g], p, I.synthetic_tables(), 1e-4, I.KPC, I.MPC, 15 * I.MPC), seed=2, capacity=800 * 56,
          max_steps=40, calls=5, all_done=False)


def test_graph_loop_and_allocation_failure():
    import paper_1410_5323_gb300 as crp
    from paper_1410_5323_gb300 import api

    g = _grid((16, 16, 16), 27).astype(np.float32)
    p = I.make_particles(600, 35, species=(("H", .5), ("He", .5)), energy=("power", 1e18, 1e20, 2.0))
    field = crp.Field(g, 0.25 * I.MPC)
    out = []
    for layout in (crp.GRID_NODES, crp.GRID_CELLS):
        sim = crp.Simulation([field], None, seed=3, capacity=600)
        sim.inject(p)
        if layout == crp.GRID_CELLS:
            crp.debug_fail_allocations(1)        # the cell copy's allocation fails
            with pytest.raises(crp.CrpError) as e:
                sim.propagate(1e-4, I.KPC, I.MPC, 10 * I.MPC, form=MIXED, grid_layout=layout)
            crp.debug_fail_allocations(0)
            assert e.value.code == api.ERR_OOM
        sim.propagate_loop(1e-4, I.KPC, I.MPC, 10 * I.MPC, max_steps=50, form=MIXED, grid_layout=layout)
        assert sim.sync(timeout_s=120.0) == 0
        out.append(sim.state())
    assert_bit_identical(out[1], out[0])
    with pytest.raises(crp.CrpError):
        sim.propagate(1e-4, I.KPC, I.MPC, 10 * I.MPC, form=MIXED, grid_layout=7)
