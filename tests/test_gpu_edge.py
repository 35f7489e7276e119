"""Degenerate inputs through the C ABI: an empty batch in the FP64 and precision forms, as
single calls and as the device-side graph loop, with an empty observer list and arrival map;
a batch of one afterwards; an adjoint of no particles (refused with INVALID_ARG)."""
import numpy as np
import pytest

from paper_1410_5323_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_empty_batch_every_form_then_one_particle():
    import paper_1410_5323_gb300 as crp

    g = I.kolmogorov_grid(16, 0.25 * I.MPC, 2, 8, 1e-13, 5).astype(np.float32)
    sim = crp.Simulation([crp.Field(g, 0.25 * I.MPC)], crp.Tables(I.synthetic_tables()), capacity=64)
    sim.inject(I.make_particles(0, 1))                     # n = 0: nothing to do
    for form in (crp.FORM_FP64, crp.FORM_MIXED):
        sim.propagate(1e-4, I.KPC, I.MPC, 10 * I.MPC, form=form)
        assert sim.sync(60.0) == 0
        sim.propagate_loop(1e-4, I.KPC, I.MPC, 10 * I.MPC, max_steps=100, form=form)
        assert sim.sync(60.0) == 0
    c = sim.counts()
    assert c["n_used"] == c["n_done"] == c["accepted"] == c["attempted"] == c["secondaries"] == 0
    rec = sim.observe()
    assert rec and all(len(v) == 0 for v in rec.values())
    assert int(sim.arrival_map(4, 1e18).sum()) == 0
    sim.inject(I.make_particles(1, 2))
    sim.propagate(1e-4, I.KPC, I.MPC, 10 * I.MPC)
    assert sim.sync(60.0) == 0
    c = sim.counts()
    assert c["n_used"] == c["n_done"] == 1 and c["accepted"] > 0
    assert len(sim.observe()["uid"]) == 1


def test_adjoint_of_no_particles_refused():
    import paper_1410_5323_gb300 as crp
    from paper_1410_5323_gb300.adjoint import Adjoint

    g = I.kolmogorov_grid(16, 0.25 * I.MPC, 2, 8, 1e-13, 6).astype(np.float32)
    f = crp.Field(g, 0.25 * I.MPC)
    for n, steps, k in ((0, 10, 4), (4, 0, 4), (4, 10, 0)):
        with pytest.raises(crp.CrpError) as e:
            Adjoint(f, n, steps, k)
        assert e.value.code == crp.api.ERR_INVALID_ARG, (n, steps, k)
