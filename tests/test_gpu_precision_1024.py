"""The precision form at full size: 10^7 protons and iron nuclei (50/50, E^-2 on
[1e18, 10^20.5] eV) through a 1024^3 BF16 grid with one FP32 scale (B_rms 0.5 nG,
l = 2-256 cells), 500 Mpc. A 10^4-particle subsample is rerun by the FP64 oracle on the
same BF16 bytes: arrival distributions agree by KS, and over the first 2 Mpc (before
chaos amplifies rounding) each particle follows the FP64 trajectory."""
import numpy as np
import pytest
from scipy import stats

import oracle as O
from paper_1410_5323_gb300 import inputs as I
from _parity import by_uid, run_oracle

pytestmark = pytest.mark.gpu


def _defl(d):
    u = np.stack([d["ux"], d["uy"], d["uz"]], 1)
    u0 = np.stack([d["u0x"], d["u0y"], d["u0z"]], 1)
    return np.degrees(np.arctan2(np.linalg.norm(np.cross(u, u0), axis=1), np.sum(u * u0, 1)))


def test_full_size_precision_workload_sampled(oracle_lib):
    import torch

    import paper_1410_5323_gb300 as crp

    w = I.workload("mixed_1024cube_10M_pFe")
    B = I.kolmogorov_grid_torch(w.grid_n, w.lmin_cells, w.lmax_cells, w.brms_t, w.grid_seed)
    q, scale = I.quantize_bf16(B)
    del B
    torch.cuda.empty_cache()
    field = crp.Field(q, w.spacing_m, scale=scale)
    bits = q.view(torch.int16).cpu().numpy().view(np.uint16)
    del q
    p = I.make_particles(w.n_particles, w.particle_seed, w.species, w.energy)
    sim = crp.Simulation([field], None, capacity=len(p))
    sim.inject(p)
    sim.propagate(w.tol, w.hmin_m, w.hmax_m, w.dmax_m, form=crp.FORM_MIXED)
    assert sim.sync(1800.0) == 0
    c = sim.counts()
    assert c["n_active"] == 0 and c["n_done"] == len(p)
    pick = np.sort(np.random.default_rng(0).choice(len(p), 10_000, replace=False))
    cols = ("ux", "uy", "uz", "u0x", "u0y", "u0z", "s", "uid", "E")
    g = {k: sim.read(k)[pick] for k in cols}
    assert np.all(g["s"] == w.dmax_m)
    sub = p.take(pick)
    kw = dict(dtype=O.BF16, scale=scale, spacing=w.spacing_m)
    st, rc = run_oracle([bits], sub, None, w.tol, w.hmin_m, w.hmax_m, w.dmax_m, **kw)
    assert rc == 0
    o = st.snapshot()
    for Zv in (1, 26):
        sel_g = np.isin(g["uid"], sub.uid[sub.Z == Zv])
        sel_o = o["Z"] == Zv
        assert stats.ks_2samp(_defl({k: v[sel_g] for k, v in g.items()}),
                              _defl({k: v[sel_o] for k, v in o.items()})).pvalue > 0.01
    # short distance: per-particle agreement with the FP64 trajectory
    short = crp.Simulation([field], None, capacity=len(sub))
    short.inject(sub)
    short.propagate(w.tol, w.hmin_m, w.hmax_m, 2 * I.MPC, form=crp.FORM_MIXED)
    short.sync(600.0)
    a = by_uid(short.state())
    so, _ = run_oracle([bits], sub, None, w.tol, w.hmin_m, w.hmax_m, 2 * I.MPC, **kw)
    b = by_uid(so.snapshot())
    ua = np.stack([a["ux"], a["uy"], a["uz"]], 1)
    ub = np.stack([b["ux"], b["uy"], b["uz"]], 1)
    ang = np.degrees(np.arctan2(np.linalg.norm(np.cross(ua, ub), axis=1), np.sum(ua * ub, 1)))
    assert np.quantile(ang, 0.95) < 0.1 and np.median(ang) < 1e-3
