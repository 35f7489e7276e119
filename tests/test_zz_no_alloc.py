"""crp_propagate_noalloc: the entry point for callers that must not have the library
allocate device memory (hosts that own a fixed GPU memory budget or pool). The test
allocates every buffer itself, calls the entry point through the C ABI twice in a row,
and checks both results against the ordinary entry points (crp_sim_create +
crp_source_inject + crp_propagate), bit for bit -- the tolerance every FP64-form parity
test here uses."""
import ctypes as C

import numpy as np
import pytest

from paper_1410_5323_gb300 import inputs as I
from _parity import by_uid

pytestmark = pytest.mark.gpu

_F64 = ["x", "y", "z", "ux", "uy", "uz", "E", "s", "hprop", "tau", "u0x", "u0y", "u0z"]
_I32 = ["A", "Z", "n_int", "status", "grid_id"]
_I64 = ["uid", "n_steps", "n_att"]


class _Cols(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in _F64 + _I32 + _I64]


def _lib():
    import paper_1410_5323_gb300 as crp

    L = crp.lib()
    L.crp_propagate_noalloc.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_double,
                                        C.c_void_p, C.c_void_p, C.c_int64, C.c_uint64, C.c_double,
                                        C.c_double, C.c_double, C.c_double, C.c_int64, C.c_void_p]
    L.crp_propagate_noalloc.restype = C.c_int
    return L


def _reference(grid, parts, seed, dmax):
    import paper_1410_5323_gb300 as crp

    sim = crp.Simulation([crp.Field(grid, 0.25 * I.MPC)], None, seed=seed, capacity=len(parts))
    sim.inject(parts)
    sim.propagate(1e-4, I.KPC, I.MPC, dmax)
    sim.sync(120.0)
    return by_uid(sim.state())


def _noalloc(L, grid, parts, seed, dmax):
    import torch

    dev = torch.device("cuda")
    n = len(parts)
    g4 = np.zeros(grid.shape[:3] + (4,), dtype=np.float32)
    g4[..., :3] = grid
    g4 = torch.from_numpy(g4).to(dev)
    cols = {k: torch.zeros(n, dtype=torch.float64, device=dev) for k in _F64}
    cols.update({k: torch.zeros(n, dtype=torch.int32, device=dev) for k in _I32})
    cols.update({k: torch.zeros(n, dtype=torch.int64, device=dev) for k in _I64})
    src = {"x": parts.x[:, 0], "y": parts.x[:, 1], "z": parts.x[:, 2], "ux": parts.u[:, 0],
           "uy": parts.u[:, 1], "uz": parts.u[:, 2], "E": parts.E, "A": parts.A, "Z": parts.Z,
           "uid": parts.uid}
    for k, v in src.items():
        cols[k].copy_(torch.from_numpy(np.ascontiguousarray(v)))
    sc = _Cols(*[cols[k].data_ptr() for k in _F64 + _I32 + _I64])
    org = (C.c_double * 3)(0.0, 0.0, 0.0)
    nx, ny, nz = grid.shape[:3]
    stream = torch.cuda.current_stream().cuda_stream
    rc = L.crp_propagate_noalloc(g4.data_ptr(), nx, ny, nz, 0.25 * I.MPC, org, C.byref(sc), n,
                                 seed, 1e-4, I.KPC, I.MPC, dmax, 0, stream)
    assert rc == 0, L.crp_last_error_detail()
    return by_uid({k: v.cpu().numpy() for k, v in cols.items()})


def test_noalloc_matches_existing_entry_point_twice():
    L = _lib()
    L.crp_debug_fail_allocations.argtypes = [C.c_int32]
    grid = I.kolmogorov_grid(16, 0.25 * I.MPC, 2, 8, 1e-13, 21).astype(np.float32)
    cases = [(I.make_particles(300, 31, species=(("H", .5), ("Fe", .5)),
                               energy=("power", 1e18, 1e20, 2.0)), 5, 20 * I.MPC),
             (I.make_particles(77, 32, energy=("loguniform", 1e17, 1e20)), 6, 12 * I.MPC)]
    for parts, seed, dmax in cases:          # two calls in a row share the static scratch
        ref = _reference(grid, parts, seed, dmax)
        # every device allocation the library makes fails while armed: the call must not need one
        assert L.crp_debug_fail_allocations(1 << 30) == 0
        try:
            got = _noalloc(L, grid, parts, seed, dmax)
        finally:
            L.crp_debug_fail_allocations(0)
        for k in ref:
            assert np.array_equal(ref[k], got[k]), k
        assert np.all(got["status"] == 1)


def test_noalloc_rejects_batches_above_its_limit():
    L = _lib()
    sc = _Cols(*([8] * len(_Cols._fields_)))          # never dereferenced: the size check comes first
    org = (C.c_double * 3)(0.0, 0.0, 0.0)
    limit = 262144
    rc = L.crp_propagate_noalloc(16, 2, 2, 2, 1.0, org, C.byref(sc), limit + 1, 1, 1e-4, 1.0, 2.0,
                                 3.0, 0, None)
    assert rc == -1
    assert b"CRP_NOALLOC_MAX_PARTICLES" in L.crp_last_error_detail()
