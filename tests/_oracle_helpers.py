"""Small builders shared by the oracle pin tests (CPU only)."""
import numpy as np

import oracle as O
from paper_1410_5323_gb300 import inputs as I

C_LIGHT = 299792458.0


def uniform_grid(B, n=4, dtype=np.float64):
    g = np.zeros((n, n, n, 3), dtype=dtype)
    g[...] = B
    return g


def particles(u, E, A=1, Z=1, x=None, uid0=0):
    u = np.atleast_2d(np.asarray(u, dtype=np.float64))
    n = u.shape[0]
    x = np.zeros((n, 3)) if x is None else np.atleast_2d(np.asarray(x, dtype=np.float64))
    return I.Particles(x.copy(), u.copy(), np.broadcast_to(np.asarray(E, dtype=np.float64), (n,)).copy(),
                       np.broadcast_to(np.asarray(A, dtype=np.int32), (n,)).copy(),
                       np.broadcast_to(np.asarray(Z, dtype=np.int32), (n,)).copy(),
                       np.arange(n, dtype=np.int64) + uid0, np.zeros(n, dtype=np.int32))


def run(parts, grid, spacing, dmax, tol=1e-4, hmin=I.KPC, hmax=I.MPC, tables=None, seed=1,
        capacity=None, max_steps=0, n_threads=4, origin=(0.0, 0.0, 0.0)):
    f = O.OracleField(grid, spacing, origin)
    st = O.OracleState(capacity or len(parts))
    ot = O.OracleTables(tables) if tables is not None else None
    O.inject(st, parts, seed, ot)
    rc, stats = O.propagate(st, [f], ot, tol, hmin, hmax, dmax, seed=seed, max_steps=max_steps,
                            n_threads=n_threads)
    return st, rc, stats
