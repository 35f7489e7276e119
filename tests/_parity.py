"""Run the same seeded case through the CUDA path (C ABI) and the CPU oracle and compare."""
import numpy as np

import oracle as O
from paper_1410_5323_gb300 import inputs as I

COLS = ["x", "y", "z", "ux", "uy", "uz", "E", "s", "hprop", "tau", "u0x", "u0y", "u0z", "A", "Z",
        "n_int", "status", "grid_id", "uid", "n_steps", "n_att"]


def by_uid(d):
    order = np.argsort(d["uid"], kind="stable")
    return {k: np.asarray(v)[order] for k, v in d.items()}


def run_gpu(grids, parts, tables, tol, hmin, hmax, dmax, seed=1, capacity=None, max_steps=0,
            spacing=0.25 * I.MPC, form=0, calls=1, dtype=None, scale=1.0, origin=(0.0, 0.0, 0.0),
            block_size=0, cadence=0, mods=None, mod_spacing=1.0, mod_origin=(0.0, 0.0, 0.0),
            box=None, grid_layout=0):
    """mods: None, or one modulation grid per vector grid (modulated fields)."""
    import paper_1410_5323_gb300 as crp

    fields = [crp.Field(g, spacing, origin, scale=scale, dtype=dtype) for g in grids]
    if mods is not None:
        for f, m in zip(fields, mods):
            f.modulate(m, mod_spacing, mod_origin)
    tabs = crp.Tables(tables) if tables is not None else None
    sim = crp.Simulation(fields, tabs, seed=seed, capacity=capacity or len(parts))
    if box is not None:
        sim.set_boundary(box)
    sim.inject(parts)
    for _ in range(calls):
        sim.propagate(tol, hmin, hmax, dmax, form=form, max_steps=max_steps, block_size=block_size,
                      cadence=cadence, grid_layout=grid_layout)
    rc = sim.sync(timeout_s=600.0, raise_on_error=False)
    return sim, rc


def run_oracle(grids, parts, tables, tol, hmin, hmax, dmax, seed=1, capacity=None, max_steps=0,
               spacing=0.25 * I.MPC, dtype=None, scale=1.0, origin=(0.0, 0.0, 0.0), calls=1,
               mods=None, mod_spacing=1.0, mod_origin=(0.0, 0.0, 0.0), box=None):
    mods = mods if mods is not None else [None] * len(grids)
    fields = [O.OracleField(g, spacing, origin, scale=scale, dtype=dtype, modulation=m,
                            mod_spacing=mod_spacing, mod_origin=mod_origin)
              for g, m in zip(grids, mods)]
    ot = O.OracleTables(tables) if tables is not None else None
    st = O.OracleState(capacity or len(parts))
    O.inject(st, parts, seed, ot)
    rc = 0
    for _ in range(calls):
        rc, _ = O.propagate(st, fields, ot, tol, hmin, hmax, dmax, seed=seed, max_steps=max_steps,
                            box=box)
    return st, rc


def assert_bit_identical(gpu_state: dict, ora_state: dict, cols=COLS):
    g, o = by_uid(gpu_state), by_uid(ora_state)
    assert len(g["uid"]) == len(o["uid"]), (len(g["uid"]), len(o["uid"]))
    bad = []
    for k in cols:
        a, b = g[k], o[k]
        if a.dtype.kind == "f":
            same = (a == b) | (np.isnan(a) & np.isnan(b))
        else:
            same = a == b
        if not np.all(same):
            i = int(np.argmin(same))
            bad.append(f"{k}: {int(np.sum(~same))} differ, first uid {g['uid'][i]}: gpu {a[i]!r} oracle {b[i]!r}")
    assert not bad, "\n".join(bad)
