"""Differentiation through a frozen step sequence (binding of crp_adjoint_*), and a
torch.autograd.Function that gives dL/dB (every grid value) and dL/dp0 (initial momenta)
of any loss of the arrival directions. Argument marshalling only; the forward, the
reverse pass and the gradient scatter run in the library's CUDA kernels."""
from __future__ import annotations

import ctypes as C

import torch

from . import api
from .api import Field, _check, lib


def _sigs():
    L = lib()
    if not getattr(L, "_adj_sigs", False):
        p, i32, i64, d = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        sig = {
            "crp_adjoint_create": ([p, i64, i32, i32, p], C.c_int),
            "crp_adjoint_destroy": ([p], C.c_int),
            "crp_adjoint_forward": ([p, p, p, p, d, d, d, p, p, p], C.c_int),
            "crp_adjoint_replay": ([p, p, p, p, p, p, p], C.c_int),
            "crp_adjoint_backward": ([p, p, p, p, p, p], C.c_int),
            "crp_adjoint_read_steps": ([p, p, i32], C.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        L._adj_sigs = True
    return L


def _dev(t: torch.Tensor, dtype) -> torch.Tensor:
    return t.detach().to(device="cuda", dtype=dtype).contiguous()


class Adjoint:
    """Recorded forward + reverse pass for n particles through one field."""

    def __init__(self, field: Field, n: int, n_steps: int, checkpoint_every: int = 64):
        self.field = field
        self.n, self.n_steps, self.K = int(n), int(n_steps), int(checkpoint_every)
        h = C.c_void_p()
        _check(_sigs().crp_adjoint_create(field._h, self.n, self.n_steps, self.K, C.byref(h)),
               "crp_adjoint_create")
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None) and api._lib is not None:
            api._lib.crp_adjoint_destroy(self._h)
            self._h = None

    def forward(self, x0, p0, Z, tolerance: float, min_step_m: float, max_step_m: float):
        x0, p0 = _dev(x0, torch.float64), _dev(p0, torch.float64)
        Z = _dev(Z, torch.int32)
        xT = torch.empty_like(p0)
        uT = torch.empty_like(p0)
        stream = torch.cuda.current_stream().cuda_stream
        _check(_sigs().crp_adjoint_forward(self._h, x0.data_ptr(), p0.data_ptr(), Z.data_ptr(),
                                           tolerance, min_step_m, max_step_m, xT.data_ptr(),
                                           uT.data_ptr(), stream), "crp_adjoint_forward")
        return xT, uT

    def replay(self, field: Field | None = None, p0=None, cells: bool = False):
        """(x_T, u_T) of the frozen steps on another field and/or from other momenta; with
        cells=True also the per-particle hash of the visited cells."""
        xT = torch.empty((self.n, 3), dtype=torch.float64, device="cuda")
        uT = torch.empty_like(xT)
        hh = torch.empty(self.n, dtype=torch.int64, device="cuda") if cells else None
        pp = None if p0 is None else _dev(p0, torch.float64)
        stream = torch.cuda.current_stream().cuda_stream
        _check(_sigs().crp_adjoint_replay(self._h, field._h if field is not None else None,
                                          pp.data_ptr() if pp is not None else None,
                                          xT.data_ptr(), uT.data_ptr(),
                                          hh.data_ptr() if cells else None, stream),
               "crp_adjoint_replay")
        return (xT, uT, hh) if cells else (xT, uT)

    def backward(self, uT_bar, grid_shape):
        ub = _dev(uT_bar, torch.float64)
        grid_bar = torch.zeros(tuple(grid_shape[:3]) + (3,), dtype=torch.float64, device="cuda")
        p0_bar = torch.empty((self.n, 3), dtype=torch.float64, device="cuda")
        x0_bar = torch.empty_like(p0_bar)
        stream = torch.cuda.current_stream().cuda_stream
        _check(_sigs().crp_adjoint_backward(self._h, ub.data_ptr(), grid_bar.data_ptr(),
                                            p0_bar.data_ptr(), x0_bar.data_ptr(), stream),
               "crp_adjoint_backward")
        return grid_bar, p0_bar, x0_bar

    def steps(self) -> torch.Tensor:
        h = torch.empty((self.n_steps, self.n), dtype=torch.float64, device="cuda")
        _check(_sigs().crp_adjoint_read_steps(self._h, h.data_ptr(), 1), "crp_adjoint_read_steps")
        return h


class PropagateAdjoint(torch.autograd.Function):
    """u_T = Propagate(grid, p0): arrival directions after n_steps accepted Cash-Karp steps
    (frozen in the forward pass). Backward gives dL/dgrid and dL/dp0."""

    @staticmethod
    def forward(ctx, grid, p0, x0, Z, spacing_m, n_steps, checkpoint_every, tolerance,
                min_step_m, max_step_m):
        field = Field(grid.detach().contiguous(), spacing_m)
        adj = Adjoint(field, p0.shape[0], n_steps, checkpoint_every)
        _, uT = adj.forward(x0, p0, Z, tolerance, min_step_m, max_step_m)
        ctx.adj = adj
        ctx.grid_shape = tuple(grid.shape)
        ctx.grid_dtype = grid.dtype
        ctx.p0_dtype = p0.dtype
        return uT

    @staticmethod
    def backward(ctx, uT_bar):
        grid_bar, p0_bar, _ = ctx.adj.backward(uT_bar, ctx.grid_shape)
        return (grid_bar.to(ctx.grid_dtype), p0_bar.to(ctx.p0_dtype), None, None, None, None, None,
                None, None, None)


def direction_loss(uT: torch.Tensor, targets: torch.Tensor) -> torch.Tensor:
    """Summed squared misfit of the arrival directions u_T/|u_T| to target unit vectors."""
    u = uT / torch.linalg.norm(uT, dim=1, keepdim=True)
    return torch.sum((u - targets) ** 2)


def perturbed_targets(uT: torch.Tensor, angle_deg: float = 1.0, seed: int = 1) -> torch.Tensor:
    """Arrival directions rotated by a fixed angle about seeded random axes (Rodrigues)."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    u = (uT / torch.linalg.norm(uT, dim=1, keepdim=True)).detach().cpu().double()
    a = torch.randn(u.shape, generator=g, dtype=torch.float64)
    a = a - (a * u).sum(1, keepdim=True) * u
    a = a / torch.linalg.norm(a, dim=1, keepdim=True)
    th = torch.tensor(angle_deg * torch.pi / 180.0, dtype=torch.float64)
    t = u * torch.cos(th) + torch.cross(a, u, dim=1) * torch.sin(th)
    return t.to(uT.device)
