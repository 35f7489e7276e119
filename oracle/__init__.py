"""ctypes binding of the plain FP64 CPU oracle (``crp_oracle.c``).

TEST INFRASTRUCTURE: imported only by the tests, the smoke check and the benchmark's
CPU-baseline leg. The product package never imports this module.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "crp_oracle.c")
LIB = os.path.join(HERE, "liborc.so")

ACTIVE, DONE, NAN, RANGE = 0, 1, 2, 3
OK, ERR_INVALID_ARG, ERR_QUEUE_FULL = 0, -1, -4
F64, F32, BF16, F16 = 0, 1, 2, 3

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
          "-pthread"]


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (no FMA contraction)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class Field(C.Structure):
    _fields_ = [("data", C.c_void_p), ("dtype", C.c_int32), ("nx", C.c_int32),
                ("ny", C.c_int32), ("nz", C.c_int32), ("pad_", C.c_int32),
                ("spacing", C.c_double), ("origin", C.c_double * 3), ("scale", C.c_double),
                ("mod_data", C.c_void_p), ("mod_dtype", C.c_int32), ("mod_nx", C.c_int32),
                ("mod_ny", C.c_int32), ("mod_nz", C.c_int32), ("mod_spacing", C.c_double),
                ("mod_origin", C.c_double * 3)]


class Tables(C.Structure):
    _fields_ = [("z_max", C.c_int32), ("n_max", C.c_int32), ("n_nodes", C.c_int32),
                ("pad_", C.c_int32), ("x0", C.c_double), ("inv_dx", C.c_double),
                ("log10_loss", C.c_void_p), ("log10_pd", C.c_void_p),
                ("has_loss", C.c_void_p), ("has_pd", C.c_void_p)]


class Params(C.Structure):
    _fields_ = [("tol", C.c_double), ("hmin", C.c_double), ("hmax", C.c_double),
                ("dmax", C.c_double), ("seed", C.c_uint64), ("max_steps", C.c_int64),
                ("n_threads", C.c_int32), ("boundary", C.c_int32),
                ("box_origin", C.c_double * 3), ("box_size", C.c_double * 3)]


BOUNDARY_NONE, BOUNDARY_REFLECT = 0, 1


_DBL = ["x", "y", "z", "ux", "uy", "uz", "E", "s", "hprop", "tau", "u0x", "u0y", "u0z"]
_I32 = ["A", "Z", "n_int", "status", "grid_id"]
_I64 = ["uid", "n_steps", "n_att"]


class _StateC(C.Structure):
    _fields_ = ([(n, C.c_void_p) for n in _DBL + _I32 + _I64]
                + [("capacity", C.c_int64), ("n", C.c_int64)])


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        d, p, i32, i64, u32, u64 = C.c_double, C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_uint64
        L.orc_philox4x32_10.argtypes = [p, p, p]
        L.orc_uniform.argtypes = [u64, u64, u32, u32]
        L.orc_uniform.restype = d
        L.orc_exp.argtypes = [d]
        L.orc_exp.restype = d
        L.orc_log.argtypes = [d]
        L.orc_log.restype = d
        L.orc_field_value.argtypes = [p, p, p]
        L.orc_grid_value.argtypes = [p, i64, i64, i64, i32]
        L.orc_grid_value.restype = d
        L.orc_modulation_value.argtypes = [p, p]
        L.orc_modulation_value.restype = d
        L.orc_deriv.argtypes = [p, d, p, p]
        L.orc_ck_attempt.argtypes = [p, d, p, p, d, p, p]
        L.orc_error_sums.argtypes = [p, p, p]
        L.orc_error_accept.argtypes = [d, d, d, d]
        L.orc_error_accept.restype = C.c_int
        L.orc_ctrl_log2.argtypes = [d]
        L.orc_ctrl_log2.restype = C.c_float
        L.orc_ctrl_log2r.argtypes = [d, d, d, d]
        L.orc_ctrl_log2r.restype = C.c_float
        L.orc_ctrl_factor.argtypes = [C.c_float, C.c_float, C.c_float, C.c_float]
        L.orc_ctrl_factor.restype = C.c_float
        L.orc_rates.argtypes = [p, i32, i32, d, p, p]
        L.orc_rates.restype = C.c_int
        L.orc_inject.argtypes = [p, i64, i64, u64, p]
        L.orc_inject.restype = C.c_int
        L.orc_propagate.argtypes = [p, p, i32, p, p, p]
        L.orc_propagate.restype = C.c_int
        _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class OracleField:
    """Keeps the grid array alive next to its C descriptor."""

    def __init__(self, grid: np.ndarray, spacing: float, origin=(0.0, 0.0, 0.0), scale: float = 1.0,
                 dtype: int | None = None, modulation: np.ndarray | None = None,
                 mod_spacing: float = 1.0, mod_origin=(0.0, 0.0, 0.0)):
        if dtype is None:
            dtype = {np.dtype(np.float64): F64, np.dtype(np.float32): F32}[grid.dtype]
        self.grid = np.ascontiguousarray(grid)
        nx, ny, nz = self.grid.shape[:3]
        if dtype in (BF16, F16):
            scale = float(np.float32(scale))      # half-precision grids carry an FP32 scale
        self.mod = None if modulation is None else np.ascontiguousarray(modulation)
        mdt = 0 if self.mod is None else {np.dtype(np.float64): F64, np.dtype(np.float32): F32}[self.mod.dtype]
        mshape = (0, 0, 0) if self.mod is None else self.mod.shape[:3]
        self.c = Field(_ptr(self.grid), dtype, nx, ny, nz, 0, float(spacing),
                       (C.c_double * 3)(*origin), float(scale),
                       None if self.mod is None else _ptr(self.mod), mdt, *mshape,
                       float(mod_spacing), (C.c_double * 3)(*mod_origin))


class OracleTables:
    def __init__(self, t):
        self.t = t
        self.ll = np.ascontiguousarray(t.log10_loss, dtype=np.float64)
        self.lp = np.ascontiguousarray(t.log10_pd, dtype=np.float64)
        self.hl = np.ascontiguousarray(t.has_loss, dtype=np.uint8)
        self.hp = np.ascontiguousarray(t.has_pd, dtype=np.uint8)
        self.c = Tables(t.z_max, t.n_max, t.n_nodes, 0, t.x0, t.inv_dx, _ptr(self.ll),
                        _ptr(self.lp), _ptr(self.hl), _ptr(self.hp))


class OracleState:
    """Structure-of-arrays particle state with `capacity` slots."""

    def __init__(self, capacity: int):
        self.capacity = int(capacity)
        for n in _DBL:
            setattr(self, n, np.zeros(self.capacity, dtype=np.float64))
        for n in _I32:
            setattr(self, n, np.zeros(self.capacity, dtype=np.int32))
        for n in _I64:
            setattr(self, n, np.zeros(self.capacity, dtype=np.int64))
        self.c = _StateC(*[_ptr(getattr(self, n)) for n in _DBL + _I32 + _I64], self.capacity, 0)

    @property
    def n(self) -> int:
        return int(self.c.n)

    def grow(self, capacity: int) -> None:
        """Copy into larger arrays (used to resume after a full secondary queue)."""
        old = self.n
        for n in _DBL + _I32 + _I64:
            a = getattr(self, n)
            b = np.zeros(capacity, dtype=a.dtype)
            b[:old] = a[:old]
            setattr(self, n, b)
        self.capacity = int(capacity)
        self.c = _StateC(*[_ptr(getattr(self, n)) for n in _DBL + _I32 + _I64], self.capacity, old)

    def load(self, p, first: int = 0) -> None:
        n = len(p)
        sl = slice(first, first + n)
        self.x[sl], self.y[sl], self.z[sl] = p.x[:, 0], p.x[:, 1], p.x[:, 2]
        self.ux[sl], self.uy[sl], self.uz[sl] = p.u[:, 0], p.u[:, 1], p.u[:, 2]
        self.E[sl] = p.E
        self.A[sl] = p.A
        self.Z[sl] = p.Z
        self.uid[sl] = p.uid
        self.grid_id[sl] = p.grid_id

    def snapshot(self) -> dict:
        n = self.n
        return {k: getattr(self, k)[:n].copy() for k in _DBL + _I32 + _I64}


def inject(state: OracleState, particles, seed: int, tables: OracleTables | None = None,
           first: int = 0) -> None:
    state.load(particles, first)
    rc = lib().orc_inject(C.byref(state.c), first, len(particles), seed,
                          C.byref(tables.c) if tables else None)
    if rc != OK:
        raise ValueError(f"orc_inject failed: {rc}")


def propagate(state: OracleState, fields, tables: OracleTables | None, tol: float, hmin: float,
              hmax: float, dmax: float, seed: int = 1, max_steps: int = 0, n_threads: int = 0,
              box=None):
    """Returns (rc, stats dict). box: None, or (origin[3], size[3]) of a reflective box."""
    if n_threads <= 0:
        n_threads = os.cpu_count() or 1
    arr = (Field * len(fields))(*[f.c for f in fields])
    org, size = box if box is not None else ((0.0, 0.0, 0.0), (0.0, 0.0, 0.0))
    prm = Params(tol, hmin, hmax, dmax, seed, max_steps, n_threads,
                 BOUNDARY_REFLECT if box is not None else BOUNDARY_NONE,
                 (C.c_double * 3)(*org), (C.c_double * 3)(*size))
    stats = np.zeros(4, dtype=np.int64)
    rc = lib().orc_propagate(C.byref(state.c), arr, len(fields),
                             C.byref(tables.c) if tables else None, C.byref(prm), _ptr(stats))
    return rc, dict(accepted=int(stats[0]), attempted=int(stats[1]), finished=int(stats[2]),
                    secondaries=int(stats[3]))


# ---- small helpers used by the pins -----------------------------------------------------
def field_value(field: OracleField, x) -> np.ndarray:
    xa = np.ascontiguousarray(x, dtype=np.float64)
    B = np.zeros(3)
    lib().orc_field_value(C.byref(field.c), _ptr(xa), _ptr(B))
    return B


def grid_values(field: OracleField) -> np.ndarray:
    """Every stored node value as the oracle widens it, shape (nx, ny, nz, 3)."""
    L = lib()
    nx, ny, nz = field.c.nx, field.c.ny, field.c.nz
    out = np.empty((nx, ny, nz, 3))
    for i in range(nx):
        for j in range(ny):
            for k in range(nz):
                for c in range(3):
                    out[i, j, k, c] = L.orc_grid_value(C.byref(field.c), i, j, k, c)
    return out


def modulation_value(field: OracleField, x) -> float:
    xa = np.ascontiguousarray(x, dtype=np.float64)
    return lib().orc_modulation_value(C.byref(field.c), _ptr(xa))


def deriv(field: OracleField, kappa: float, y) -> np.ndarray:
    ya = np.ascontiguousarray(y, dtype=np.float64)
    k = np.zeros(6)
    lib().orc_deriv(C.byref(field.c), kappa, _ptr(ya), _ptr(k))
    return k


def ck_attempt(field: OracleField, kappa: float, y, h: float):
    ya = np.ascontiguousarray(y, dtype=np.float64)
    k1 = deriv(field, kappa, ya)
    y5 = np.zeros(6)
    err = np.zeros(6)
    lib().orc_ck_attempt(C.byref(field.c), kappa, _ptr(ya), _ptr(k1), h, _ptr(y5), _ptr(err))
    return y5, err


def error_sums(err):
    """(|dx|^2, |du|^2) of an error vector (dx, du)."""
    e = np.ascontiguousarray(err, dtype=np.float64)
    out = np.zeros(2)
    lib().orc_error_sums(_ptr(e), _ptr(out), _ptr(out[1:]))
    return float(out[0]), float(out[1])


def error_accept(sx: float, su: float, h: float, tol: float) -> bool:
    return bool(lib().orc_error_accept(sx, su, h, tol))


def ctrl_log2(v: float) -> float:
    return float(lib().orc_ctrl_log2(v))


def ctrl_log2r(sx: float, su: float, h: float, tol: float) -> float:
    return float(lib().orc_ctrl_log2r(sx, su, h, tol))


def ctrl_factor(log2r: float, p: float, lo: float, hi: float) -> float:
    return float(lib().orc_ctrl_factor(log2r, p, lo, hi))


def rates(tables: OracleTables, A: int, Z: int, E: float):
    rl = C.c_double()
    rp = C.c_double()
    rc = lib().orc_rates(C.byref(tables.c), A, Z, E, C.byref(rl), C.byref(rp))
    return rc, rl.value, rp.value


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def uniform(seed: int, uid: int, k: int, tag: int) -> float:
    return lib().orc_uniform(seed, uid, k, tag)


def exp(x: float) -> float:
    return lib().orc_exp(x)


def log(x: float) -> float:
    return lib().orc_log(x)


# ---- frozen-step differentiation ------------------------------------------------------
def _sigs():
    L = lib()
    if not getattr(L, "_adj_sigs", False):
        p, d, i32 = C.c_void_p, C.c_double, C.c_int32
        L.orc_record_steps.argtypes = [p, d, p, d, d, d, i32, p, p]
        L.orc_record_steps.restype = C.c_int
        L.orc_frozen_forward.argtypes = [p, d, p, p, i32, p]
        L.orc_adjoint.argtypes = [p, d, p, p, i32, p, p, p, p]
        L._adj_sigs = True
    return L


def record_steps(field: OracleField, kappa: float, y0, tol: float, hmin: float, hmax: float,
                 n_steps: int):
    """Accepted step sizes of the propagation module alone; returns (h[n], y_T)."""
    y = np.ascontiguousarray(y0, dtype=np.float64)
    h = np.zeros(n_steps)
    yT = np.zeros(6)
    _sigs().orc_record_steps(C.byref(field.c), kappa, _ptr(y), tol, hmin, hmax, n_steps, _ptr(h), _ptr(yT))
    return h, yT


def frozen_forward(field: OracleField, kappa: float, y0, h) -> np.ndarray:
    y = np.ascontiguousarray(y0, dtype=np.float64)
    hh = np.ascontiguousarray(h, dtype=np.float64)
    yT = np.zeros(6)
    _sigs().orc_frozen_forward(C.byref(field.c), kappa, _ptr(y), _ptr(hh), len(hh), _ptr(yT))
    return yT


def adjoint(field: OracleField, kappa: float, y0, h, lamT, grid_bar: np.ndarray | None = None):
    """Reverse pass; returns (y0_bar, kappa_bar); grid_bar ([nx,ny,nz,3] float64) accumulates."""
    y = np.ascontiguousarray(y0, dtype=np.float64)
    hh = np.ascontiguousarray(h, dtype=np.float64)
    lam = np.ascontiguousarray(lamT, dtype=np.float64)
    yb = np.zeros(6)
    kb = C.c_double()
    gp = None if grid_bar is None else _ptr(grid_bar)
    _sigs().orc_adjoint(C.byref(field.c), kappa, _ptr(y), _ptr(hh), len(hh), _ptr(lam), gp, _ptr(yb),
                        C.byref(kb))
    return yb, kb.value


# ---- sources (Sec. 4, Eq. 1) and arrival binning -----------------------------------------
MAX_SPECIES = 8


class Spectrum(C.Structure):
    _fields_ = [("n_species", C.c_int32), ("A", C.c_int32 * MAX_SPECIES),
                ("Z", C.c_int32 * MAX_SPECIES), ("pad_", C.c_int32),
                ("x", C.c_double * MAX_SPECIES), ("alpha", C.c_double), ("rcut_v", C.c_double),
                ("e_min_ev", C.c_double), ("e_max_ev", C.c_double)]


def spectrum(species, alpha: float, rcut_v: float, e_min_ev: float, e_max_ev: float) -> Spectrum:
    """species: [(A, Z, x), ...]."""
    sp = Spectrum()
    sp.n_species = len(species)
    for i, (a, z, x) in enumerate(species):
        sp.A[i], sp.Z[i], sp.x[i] = int(a), int(z), float(x)
    sp.alpha, sp.rcut_v, sp.e_min_ev, sp.e_max_ev = float(alpha), float(rcut_v), float(e_min_ev), float(e_max_ev)
    return sp


def _src_sigs():
    L = lib()
    if not getattr(L, "_src_sigs", False):
        p, d, i32, i64, u64 = C.c_void_p, C.c_double, C.c_int32, C.c_int64, C.c_uint64
        L.orc_source_sample.argtypes = [p, u64, u64, i64, p, p, p, p, p, p]
        L.orc_source_sample.restype = i64
        L.orc_atan2.argtypes = [d, d]
        L.orc_atan2.restype = d
        L.orc_healpix_ring.argtypes = [i32, d, d, d]
        L.orc_healpix_ring.restype = i64
        L.orc_arrival_map.argtypes = [p, i32, d, p]
        L.orc_arrival_map.restype = C.c_int
        L._src_sigs = True
    return L


def source_sample(sp: Spectrum, seed: int, uid_base: int, n: int):
    """(A, Z, E, u [n, 3], n_failed) drawn from Eq. 1 with isotropic directions."""
    A = np.zeros(n, np.int32)
    Z = np.zeros(n, np.int32)
    E = np.zeros(n)
    u = np.zeros((3, n))
    failed = _src_sigs().orc_source_sample(C.byref(sp), seed, uid_base, n, _ptr(A), _ptr(Z), _ptr(E),
                                           _ptr(u[0]), _ptr(u[1]), _ptr(u[2]))
    if failed < 0:
        raise ValueError("invalid spectrum")
    return A, Z, E, np.ascontiguousarray(u.T), int(failed)


def atan2(y: float, x: float) -> float:
    return _src_sigs().orc_atan2(y, x)


def healpix_ring(nside: int, u) -> np.ndarray:
    """Pixel index of each direction row of u [n, 3] (plain loop over the rows)."""
    L = _src_sigs()
    u = np.atleast_2d(np.asarray(u, dtype=np.float64))
    return np.array([L.orc_healpix_ring(nside, float(a), float(b), float(c)) for a, b, c in u],
                    dtype=np.int64)


def arrival_map(state: OracleState, nside: int, e_min_ev: float) -> np.ndarray:
    m = np.zeros(12 * nside * nside, dtype=np.uint64)
    rc = _src_sigs().orc_arrival_map(C.byref(state.c), nside, e_min_ev, _ptr(m))
    if rc != OK:
        raise ValueError(f"orc_arrival_map failed: {rc}")
    return m


# ---- lenses (Sec. 3.3) ---------------------------------------------------------------------
def _lens_sigs():
    L = lib()
    if not getattr(L, "_lens_sigs", False):
        p, d, i32 = C.c_void_p, C.c_double, C.c_int32
        L.orc_lens_apply.argtypes = [i32, i32, p, p, p, p, i32, p]
        L.orc_lens_apply.restype = C.c_int
        L.orc_lens_bin.argtypes = [p, i32, i32, p, d, p]
        L.orc_lens_bin.restype = C.c_int
        L._lens_sigs = True
    return L


def lens_apply(n_pix: int, row_ptr, col, val, x) -> np.ndarray:
    """y [n_pix, n_maps] = sum_m M_m x[m]; row_ptr [n_mat, n_pix + 1] (global offsets into col
    and val), x [n_mat, n_pix, n_maps] float64."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    c = np.ascontiguousarray(col, dtype=np.int32)
    v = np.ascontiguousarray(val, dtype=np.float32)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    n_mat, _, n_maps = xx.shape
    y = np.zeros((n_pix, n_maps))
    rc = _lens_sigs().orc_lens_apply(n_pix, n_mat, _ptr(rp), _ptr(c) if c.size else None,
                                     _ptr(v) if v.size else None, _ptr(xx), n_maps, _ptr(y))
    if rc != OK:
        raise ValueError(f"orc_lens_apply failed: {rc}")
    return y


def lens_bin(state: OracleState, nside: int, edges, e_min_ev: float) -> np.ndarray:
    e = np.ascontiguousarray(edges, dtype=np.float64)
    x = np.zeros((len(e) - 1, 12 * nside * nside))
    rc = _lens_sigs().orc_lens_bin(C.byref(state.c), nside, len(e) - 1, _ptr(e), e_min_ev, _ptr(x))
    if rc != OK:
        raise ValueError(f"orc_lens_bin failed: {rc}")
    return x
