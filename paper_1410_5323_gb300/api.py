"""ctypes binding of libcrp.so: the same entry points as include/crp.h, with numpy or
torch buffers marshalled to plain pointers. No arithmetic of the method happens here."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcrp.so")

OK = 0
ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_QUEUE_FULL = -1, -2, -3, -4
ERR_TIMEOUT, ERR_NAN_STATE, ERR_TABLE_RANGE = -5, -6, -7
DTYPE_F64, DTYPE_F32, DTYPE_BF16, DTYPE_F16 = 0, 1, 2, 3
FORM_FP64, FORM_MIXED = 0, 1
# grid layout read by the precision form (crp.h CRP_GRID_*)
GRID_AUTO, GRID_NODES, GRID_CELLS = 0, 1, 2
ORDER_DEFAULT, ORDER_SLOT, ORDER_COST, ORDER_GRID = 0, 1, 2, 3
PICKUP_DEFAULT, PICKUP_OFF, PICKUP_ON = 0, 1, 2
STATUS_ACTIVE, STATUS_DONE, STATUS_NAN, STATUS_RANGE = 0, 1, 2, 3
BOUNDARY_NONE, BOUNDARY_REFLECT = 0, 1

# column name -> (id, numpy dtype)
COLUMNS = {
    "x": (0, np.float64), "y": (1, np.float64), "z": (2, np.float64),
    "ux": (3, np.float64), "uy": (4, np.float64), "uz": (5, np.float64),
    "E": (6, np.float64), "s": (7, np.float64), "hprop": (8, np.float64),
    "tau": (9, np.float64), "u0x": (10, np.float64), "u0y": (11, np.float64),
    "u0z": (12, np.float64), "A": (13, np.int32), "Z": (14, np.int32),
    "n_int": (15, np.int32), "status": (16, np.int32), "grid_id": (17, np.int32),
    "uid": (18, np.int64), "n_steps": (19, np.int64), "n_att": (20, np.int64),
}


class CrpError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        L = lib()
        super().__init__(f"{where}: {L.crp_error_string(code).decode()} ({code}): "
                         f"{L.crp_last_error_detail().decode()}")


class _Particles(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("x", "y", "z", "ux", "uy", "uz", "E", "A", "Z", "uid",
                                          "grid_id")] + [("is_device", C.c_int32), ("pad_", C.c_int32)]


MAX_SPECIES = 8


class Spectrum(C.Structure):
    """Source spectrum of paper Sec. 4, Eq. 1 (crp_spectrum)."""
    _fields_ = [("n_species", C.c_int32), ("A", C.c_int32 * MAX_SPECIES),
                ("Z", C.c_int32 * MAX_SPECIES), ("pad_", C.c_int32),
                ("x", C.c_double * MAX_SPECIES), ("alpha", C.c_double), ("rcut_v", C.c_double),
                ("e_min_ev", C.c_double), ("e_max_ev", C.c_double)]

    @classmethod
    def of(cls, species, alpha: float, rcut_v: float, e_min_ev: float, e_max_ev: float) -> "Spectrum":
        """species: [(A, Z, x), ...]."""
        sp = cls()
        sp.n_species = len(species)
        for i, (a, z, x) in enumerate(species):
            sp.A[i], sp.Z[i], sp.x[i] = int(a), int(z), float(x)
        sp.alpha, sp.rcut_v = float(alpha), float(rcut_v)
        sp.e_min_ev, sp.e_max_ev = float(e_min_ev), float(e_max_ev)
        return sp


def healpix_ring(nside: int, u, stream=None):
    """HEALPix RING pixel of each row of u ([n, 3] torch tensor on the GPU, float64)."""
    import torch

    u = u.contiguous()
    if not u.is_cuda or u.dtype != torch.float64:
        raise TypeError("u must be a float64 CUDA tensor")
    pix = torch.empty(u.shape[0], dtype=torch.int64, device=u.device)
    _check(lib().crp_healpix_ring(int(nside), u.data_ptr(), int(u.shape[0]), pix.data_ptr(),
                                  _stream_ptr(stream)), "crp_healpix_ring")
    return pix


def debug_fail_allocations(n: int) -> None:
    """Fault injection: the library's next n device allocations fail as out of memory."""
    _check(lib().crp_debug_fail_allocations(int(n)), "crp_debug_fail_allocations")


def kernel_runs() -> int:
    """How many of the library's kernels have run on the current device since it was loaded
    (synchronises the device)."""
    n = C.c_uint64()
    _check(lib().crp_kernel_runs(C.byref(n)), "crp_kernel_runs")
    return int(n.value)


def selftest_wait(limit: int, preset: int = -1, stream=None) -> int:
    """Runs the kernels' bounded wait on a flag preset to `preset`; returns the status code
    (ERR_TIMEOUT when the flag is never set, OK otherwise) without raising."""
    return int(lib().crp_selftest_wait(int(limit), int(preset), _stream_ptr(stream)))


class Lens:
    """Per-rigidity sparse lens matrices (paper Sec. 3.3), CSR over shared arrays:
    row_ptr [n_mat, n_pix + 1] int64 (offsets into col/val, matrices one after another),
    col int32, val float32; edges: n_mat + 1 rigidities (V) of the bins, or None."""

    def __init__(self, n_pix: int, row_ptr, col, val, edges=None):
        rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
        c = np.ascontiguousarray(col, dtype=np.int32)
        v = np.ascontiguousarray(val, dtype=np.float32)
        e = None if edges is None else np.ascontiguousarray(edges, dtype=np.float64)
        self.n_mat = int(rp.shape[0])
        self.n_pix = int(n_pix)
        self.nnz = int(c.size)
        h = C.c_void_p()
        _check(lib().crp_lens_create(self.n_pix, self.n_mat, rp.ctypes.data,
                                     c.ctypes.data if c.size else None, v.ctypes.data if v.size else None,
                                     None if e is None else e.ctypes.data, C.byref(h)), "crp_lens_create")
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.crp_lens_destroy(self._h)
            self._h = None

    def set_group(self, lanes_per_row: int) -> None:
        """Lanes per row for one map (4, 8, 16 or 32)."""
        _check(lib().crp_lens_set_group(self._h, int(lanes_per_row)), "crp_lens_set_group")

    def apply(self, x, out=None, stream=None):
        """x: float64 CUDA tensor [n_mat, n_pix] or [n_mat, n_pix, n_maps]; returns
        y = sum_m M_m x_m as [n_pix] or [n_pix, n_maps]."""
        import torch

        x = x.contiguous()
        if not x.is_cuda or x.dtype != torch.float64:
            raise TypeError("x must be a float64 CUDA tensor")
        n_maps = 1 if x.dim() == 2 else int(x.shape[2])
        if out is None:
            out = torch.empty((self.n_pix,) if x.dim() == 2 else (self.n_pix, n_maps),
                              dtype=torch.float64, device=x.device)
        _check(lib().crp_lens_apply(self._h, x.data_ptr(), out.data_ptr(), n_maps, _stream_ptr(stream)),
               "crp_lens_apply")
        return out

    def bin(self, sim: "Simulation", nside: int, e_min_ev: float, out=None, stream=None):
        """Rigidity-binned arrival maps of a simulation: [n_mat, 12 nside^2] float64, added to
        ``out`` (zeroed if created here)."""
        import torch

        if out is None:
            out = torch.zeros((self.n_mat, self.n_pix), dtype=torch.float64, device="cuda")
        _check(lib().crp_lens_bin(self._h, sim._h, int(nside), float(e_min_ev), out.data_ptr(),
                                  _stream_ptr(stream)), "crp_lens_bin")
        return out


class _Params(C.Structure):
    _fields_ = [("form", C.c_int32), ("block_size", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("cadence", C.c_int32), ("max_steps", C.c_int64), ("order", C.c_int32),
                ("pickup", C.c_int32), ("grid_layout", C.c_int32), ("pad_", C.c_int32)]


_OBS_I64 = ("uid",)
_OBS_I32 = ("A", "Z", "n_int", "status")
_OBS_F64 = ("E", "x", "y", "z", "ux", "uy", "uz", "u0x", "u0y", "u0z", "s")
_OBS_I64B = ("n_steps", "n_att")


class _Observer(C.Structure):
    _fields_ = ([(n, C.c_void_p) for n in _OBS_I64 + _OBS_I32 + _OBS_F64 + _OBS_I64B]
                + [("is_device", C.c_int32), ("pad_", C.c_int32)])


_lib = None


def lib() -> C.CDLL:
    """Load libcrp.so; raises if the CUDA library has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        L = C.CDLL(LIB_PATH)
        p, i32, i64, u64, d, f = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double, C.c_float
        sig = {
            "crp_field_create": ([p, i32, i32, i32, i32, i32, d, p, f, p], C.c_int),
            "crp_field_destroy": ([p], C.c_int),
            "crp_field_modulate": ([p, p, i32, i32, i32, i32, i32, d, p], C.c_int),
            "crp_tables_create": ([i32, i32, i32, d, d, p, p, p, p, p], C.c_int),
            "crp_tables_destroy": ([p], C.c_int),
            "crp_sim_create": ([p, i32, p, u64, i64, p], C.c_int),
            "crp_sim_reserve": ([p, i64], C.c_int),
            "crp_sim_destroy": ([p], C.c_int),
            "crp_sim_reset": ([p], C.c_int),
            "crp_sim_set_boundary": ([p, i32, p, p], C.c_int),
            "crp_source_sample": ([p, p, p, p, p, p, i32, i64, p], C.c_int),
            "crp_healpix_ring": ([i32, p, i64, p, p], C.c_int),
            "crp_arrival_map": ([p, i32, d, p, p], C.c_int),
            "crp_lens_create": ([i32, i32, p, p, p, p, p], C.c_int),
            "crp_debug_fail_allocations": ([i32], C.c_int),
            "crp_selftest_wait": ([i32, i32, p], C.c_int),
            "crp_kernel_runs": ([p], C.c_int),
            "crp_lens_destroy": ([p], C.c_int),
            "crp_lens_apply": ([p, p, p, i32, p], C.c_int),
            "crp_lens_bin": ([p, p, i32, d, p, p], C.c_int),
            "crp_source_inject": ([p, p, i64, p], C.c_int),
            "crp_propagate": ([p, p, d, d, d, d, p], C.c_int),
            "crp_propagate_loop": ([p, p, d, d, d, d, i32, p], C.c_int),
            "crp_sync": ([p, d], C.c_int),
            "crp_sim_counts": ([p, p], C.c_int),
            "crp_read_state": ([p, i32, p, i32, i64, i64], C.c_int),
            "crp_observe": ([p, p, i64, i64, p], C.c_int),
            "crp_error_string": ([i32], C.c_char_p),
            "crp_last_error_detail": ([], C.c_char_p),
            "crp_version": ([], C.c_char_p),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(rc: int, where: str) -> None:
    if rc != OK:
        raise CrpError(rc, where)


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _buf(x):
    """(pointer, is_device, keepalive) for a numpy array or torch tensor."""
    if x is None:
        return None, 0, None
    if _is_torch(x):
        x = x.contiguous()
        return x.data_ptr(), 1 if x.is_cuda else 0, x
    a = np.ascontiguousarray(x)
    return a.ctypes.data, 0, a


def _stream_ptr(stream) -> int | None:
    if stream is None:
        try:
            import torch

            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Field:
    """Periodic regular vector grid (paper Sec. 3.2). ``grid``: [nx, ny, nz, 3] numpy array
    or torch tensor (float64 / float32 / bfloat16 / float16; numpy uint16 with ``dtype``)."""

    def __init__(self, grid, spacing_m: float, origin_m=(0.0, 0.0, 0.0), scale: float = 1.0,
                 dtype: int | None = None):
        if dtype is None:
            name = str(grid.dtype)
            dtype = {"float64": DTYPE_F64, "torch.float64": DTYPE_F64, "float32": DTYPE_F32,
                     "torch.float32": DTYPE_F32, "torch.bfloat16": DTYPE_BF16,
                     "float16": DTYPE_F16, "torch.float16": DTYPE_F16}[name]
        nx, ny, nz = (int(v) for v in grid.shape[:3])
        ptr, dev, keep = _buf(grid)
        org = (C.c_double * 3)(*origin_m)
        h = C.c_void_p()
        _check(lib().crp_field_create(ptr, dtype, dev, nx, ny, nz, float(spacing_m), org,
                                      float(scale), C.byref(h)), "crp_field_create")
        del keep
        self._h = h
        self.shape = (nx, ny, nz)
        self.spacing = float(spacing_m)
        self.modulated = False

    def modulate(self, mod, spacing_m: float, origin_m=(0.0, 0.0, 0.0)) -> "Field":
        """Attach a scalar modulation grid (paper Sec. 3.2 modulated grids): the field
        becomes M(x) b(x). ``mod``: [nx, ny, nz] float32 numpy array or torch tensor."""
        name = str(mod.dtype)
        if name not in ("float32", "torch.float32"):
            raise TypeError("modulation grids are float32")
        nx, ny, nz = (int(v) for v in mod.shape[:3])
        ptr, dev, keep = _buf(mod)
        org = (C.c_double * 3)(*origin_m)
        _check(lib().crp_field_modulate(self._h, ptr, DTYPE_F32, dev, nx, ny, nz, float(spacing_m), org),
               "crp_field_modulate")
        del keep
        self.modulated = True
        return self

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.crp_field_destroy(self._h)
            self._h = None


class Tables:
    """Interaction tables (paper Sec. 2), from an ``inputs.TableArrays``."""

    def __init__(self, t):
        ll = np.ascontiguousarray(t.log10_loss, dtype=np.float64)
        lp = np.ascontiguousarray(t.log10_pd, dtype=np.float64)
        hl = np.ascontiguousarray(t.has_loss, dtype=np.uint8)
        hp = np.ascontiguousarray(t.has_pd, dtype=np.uint8)
        h = C.c_void_p()
        _check(lib().crp_tables_create(t.z_max, t.n_max, t.n_nodes, t.x0, t.inv_dx,
                                       ll.ctypes.data, lp.ctypes.data, hl.ctypes.data,
                                       hp.ctypes.data, C.byref(h)), "crp_tables_create")
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.crp_tables_destroy(self._h)
            self._h = None


class Simulation:
    def __init__(self, fields, tables: Tables | None = None, seed: int = 1,
                 capacity: int = 1 << 20):
        if isinstance(fields, Field):
            fields = [fields]
        self._fields = list(fields)      # handles must outlive the simulation
        self._tables = tables
        arr = (C.c_void_p * len(self._fields))(*[f._h.value for f in self._fields])
        h = C.c_void_p()
        _check(lib().crp_sim_create(arr, len(self._fields), tables._h if tables else None,
                                    int(seed), int(capacity), C.byref(h)), "crp_sim_create")
        self._h = h
        self.capacity = int(capacity)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.crp_sim_destroy(self._h)
            self._h = None

    def inject(self, p=None, *, x=None, u=None, E=None, A=None, Z=None, uid=None, grid_id=None,
               stream=None) -> None:
        """Append particles: an ``inputs.Particles`` (host) or columns (numpy or torch;
        x and u may be [n,3] arrays or 3-tuples of columns)."""
        if p is not None:
            x, u, E, A, Z, uid, grid_id = p.x, p.u, p.E, p.A, p.Z, p.uid, p.grid_id
        cols = []
        for v in (x, u):
            if isinstance(v, (tuple, list)):
                cols.extend(v)
            elif _is_torch(v):
                cols.extend([v[:, 0].contiguous(), v[:, 1].contiguous(), v[:, 2].contiguous()])
            else:
                v = np.asarray(v, dtype=np.float64)
                cols.extend([np.ascontiguousarray(v[:, 0]), np.ascontiguousarray(v[:, 1]),
                             np.ascontiguousarray(v[:, 2])])
        if not _is_torch(E):
            E = np.asarray(E, dtype=np.float64)
            A = np.asarray(A, dtype=np.int32)
            Z = np.asarray(Z, dtype=np.int32)
            uid = None if uid is None else np.asarray(uid, dtype=np.int64)
            grid_id = None if grid_id is None else np.asarray(grid_id, dtype=np.int32)
        bufs = [_buf(c) for c in cols + [E, A, Z, uid, grid_id]]
        devs = {b[1] for b in bufs if b[0] is not None}
        if len(devs) != 1:
            raise ValueError("particle columns must all be host or all be device buffers")
        n = int(E.shape[0])
        ps = _Particles(*[b[0] for b in bufs], devs.pop(), 0)
        _check(lib().crp_source_inject(self._h, C.byref(ps), n, _stream_ptr(stream)),
               "crp_source_inject")

    def sample_sources(self, spectrum: "Spectrum", x, grid_id=None, stream=None) -> None:
        """Append len(x) primaries at positions x ([n, 3] or a 3-tuple of columns, numpy or
        torch) with species, energy and direction drawn on the device from ``spectrum``."""
        if isinstance(x, (tuple, list)):
            cols = list(x)
        elif _is_torch(x):
            cols = [x[:, 0].contiguous(), x[:, 1].contiguous(), x[:, 2].contiguous()]
        else:
            x = np.asarray(x, dtype=np.float64)
            cols = [np.ascontiguousarray(x[:, c]) for c in range(3)]
        if grid_id is not None and not _is_torch(grid_id):
            grid_id = np.asarray(grid_id, dtype=np.int32)
        bufs = [_buf(c) for c in cols + [grid_id]]
        devs = {b[1] for b in bufs if b[0] is not None}
        if len(devs) != 1:
            raise ValueError("columns must all be host or all be device buffers")
        n = int(cols[0].shape[0])
        _check(lib().crp_source_sample(self._h, C.byref(spectrum), bufs[0][0], bufs[1][0], bufs[2][0],
                                       bufs[3][0], devs.pop(), n, _stream_ptr(stream)),
               "crp_source_sample")

    def arrival_map(self, nside: int, e_min_ev: float, out=None, stream=None):
        """Counts of finished particles above e_min_ev per HEALPix RING pixel of -u (paper
        Sec. 4, Fig. 4), accumulated into ``out`` (a zeroed uint64-sized int64 CUDA tensor of
        12 nside^2) or a new one."""
        import torch

        if out is None:
            out = torch.zeros(12 * nside * nside, dtype=torch.int64, device="cuda")
        _check(lib().crp_arrival_map(self._h, int(nside), float(e_min_ev), out.data_ptr(),
                                     _stream_ptr(stream)), "crp_arrival_map")
        return out

    def propagate(self, tolerance: float, min_step_m: float, max_step_m: float,
                  max_distance_m: float, form: int = FORM_FP64, max_steps: int = 0,
                  block_size: int = 0, blocks_per_sm: int = 0, cadence: int = 0,
                  order: int = 0, pickup: int = 0, grid_layout: int = GRID_AUTO, stream=None) -> None:
        prm = _Params(form, block_size, blocks_per_sm, cadence, max_steps, order, pickup, grid_layout)
        _check(lib().crp_propagate(self._h, C.byref(prm), tolerance, min_step_m, max_step_m,
                                   max_distance_m, _stream_ptr(stream)), "crp_propagate")

    def propagate_loop(self, tolerance: float, min_step_m: float, max_step_m: float,
                       max_distance_m: float, max_steps: int, max_slices: int = 1 << 20,
                       form: int = FORM_FP64, block_size: int = 0, blocks_per_sm: int = 0,
                       cadence: int = 0, order: int = 0, pickup: int = 0, grid_layout: int = GRID_AUTO,
                       stream=None) -> None:
        """Slices of max_steps accepted steps until done, as one device-side graph loop."""
        prm = _Params(form, block_size, blocks_per_sm, cadence, max_steps, order, pickup, grid_layout)
        _check(lib().crp_propagate_loop(self._h, C.byref(prm), tolerance, min_step_m, max_step_m,
                                        max_distance_m, int(max_slices), _stream_ptr(stream)),
               "crp_propagate_loop")

    def sync(self, timeout_s: float = 0.0, raise_on_error: bool = True) -> int:
        rc = lib().crp_sync(self._h, timeout_s)
        if raise_on_error:
            _check(rc, "crp_sync")
        return rc

    def reset(self) -> None:
        _check(lib().crp_sim_reset(self._h), "crp_sim_reset")

    def grid_layout(self) -> int:
        """GRID_CELLS once the precision form's cell-major copies are built, else GRID_NODES."""
        v = C.c_int32(0)
        _check(lib().crp_sim_grid_layout(self._h, C.byref(v)), "crp_sim_grid_layout")
        return int(v.value)

    def set_boundary(self, box=None) -> None:
        """Reflective box (paper Sec. 4): ``box`` = (origin[3], size[3]) in metres, or None
        for no boundary."""
        if box is None:
            _check(lib().crp_sim_set_boundary(self._h, BOUNDARY_NONE, None, None), "crp_sim_set_boundary")
            return
        org = (C.c_double * 3)(*[float(v) for v in box[0]])
        size = (C.c_double * 3)(*[float(v) for v in box[1]])
        _check(lib().crp_sim_set_boundary(self._h, BOUNDARY_REFLECT, org, size), "crp_sim_set_boundary")

    def reserve(self, capacity: int) -> None:
        _check(lib().crp_sim_reserve(self._h, int(capacity)), "crp_sim_reserve")
        self.capacity = max(self.capacity, int(capacity))

    def counts(self) -> dict:
        c = np.zeros(8, dtype=np.int64)
        _check(lib().crp_sim_counts(self._h, c.ctypes.data), "crp_sim_counts")
        keys = ("n_used", "n_active", "n_done", "accepted", "attempted", "secondaries",
                "launches", "status_bits")
        return {k: int(v) for k, v in zip(keys, c)}

    def read(self, name: str, first: int = 0, count: int | None = None, out=None):
        col, dt = COLUMNS[name]
        if count is None:
            count = self.counts()["n_used"] - first
        if out is None:
            out = np.empty(count, dtype=dt)
        ptr, dev, keep = _buf(out)
        _check(lib().crp_read_state(self._h, col, ptr, dev, first, count), "crp_read_state")
        return keep if dev else out

    def state(self) -> dict:
        n = self.counts()["n_used"]
        return {k: self.read(k, 0, n) for k in COLUMNS}

    @staticmethod
    def observe_bytes(n: int) -> int:
        """Bytes of n observer records (all columns)."""
        return int(n) * (8 * (len(_OBS_I64) + len(_OBS_F64) + len(_OBS_I64B)) + 4 * len(_OBS_I32))

    @staticmethod
    def observe_buffers(capacity: int, pinned: bool = False, device=None) -> dict:
        """Preallocated observer columns: numpy (default), pinned host or device torch tensors."""
        import torch

        dt = {**{n: torch.int64 for n in _OBS_I64 + _OBS_I64B},
              **{n: torch.int32 for n in _OBS_I32}, **{n: torch.float64 for n in _OBS_F64}}
        if device is not None:
            return {n: torch.empty(capacity, dtype=t, device=device) for n, t in dt.items()}
        return {n: torch.empty(capacity, dtype=t, pin_memory=pinned) for n, t in dt.items()}

    def observe(self, first: int = 0, capacity: int | None = None, out: dict | None = None) -> dict:
        """Records of finished particles (observer, paper Sec. 3.1), in finishing order.
        ``out``: preallocated columns (numpy or torch, all host or all device)."""
        if out is None:
            if capacity is None:
                capacity = self.counts()["n_done"] - first
            capacity = max(int(capacity), 0)
            out = {}
            for n in _OBS_I64 + _OBS_I64B:
                out[n] = np.empty(capacity, dtype=np.int64)
            for n in _OBS_I32:
                out[n] = np.empty(capacity, dtype=np.int32)
            for n in _OBS_F64:
                out[n] = np.empty(capacity, dtype=np.float64)
        names = _OBS_I64 + _OBS_I32 + _OBS_F64 + _OBS_I64B
        bufs = {n: _buf(out[n]) for n in names}
        if capacity is None:
            capacity = min(int(out[n].shape[0]) for n in names)
        devs = {b[1] for b in bufs.values()}
        if len(devs) != 1:
            raise ValueError("observer columns must all be host or all be device buffers")
        o = _Observer(*[bufs[n][0] for n in names], devs.pop(), 0)
        n_out = C.c_int64()
        _check(lib().crp_observe(self._h, C.byref(o), first, capacity, C.byref(n_out)), "crp_observe")
        return {k: v[:n_out.value] for k, v in out.items()}
