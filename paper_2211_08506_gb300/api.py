"""PyTorch-facing API over the C ABI: device tensors in, device tensors out.

PyTorch supplies device memory and streams only; every step of the voxelization runs in
the library's CUDA kernels.  ``Voxelize`` wraps forward (Sec. III-A, Eq. 1) and the
coordinate adjoint (Sec. IV-C) as a ``torch.autograd.Function``.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field
from typing import Sequence

import numpy as np
import torch

from . import binding as B

DTYPES = {"f32": (B.PG_F32, torch.float32), "f16": (B.PG_F16, torch.float16),
          "bf16": (B.PG_BF16, torch.bfloat16)}
TORCH_TO_PG = {torch.float32: B.PG_F32, torch.float16: B.PG_F16, torch.bfloat16: B.PG_BF16}
CUTOFFS = {"sphere": B.PG_CUTOFF_SPHERE, "none": B.PG_CUTOFF_NONE, "box": B.PG_CUTOFF_BOX}
PATHS = {"auto": B.PG_PATH_AUTO, "direct": B.PG_PATH_DIRECT, "separable": B.PG_PATH_SEPARABLE}
FORMS = {"point": B.PG_FORM_POINT, "integral": B.PG_FORM_INTEGRAL}


@dataclass
class Grid:
    """Grid shape, channels and Gaussian widths shared by a batch (see pg_grid)."""

    nx: int
    ny: int
    nz: int
    n_channels: int
    sigma: Sequence[float]
    cutoff: str = "sphere"
    cutoff_k: float = 3.0
    periodic: bool = False
    form: str = "point"          # "point" sample or voxel "integral" (erf form)
    _sigma_buf: object = field(default=None, repr=False, compare=False)

    @classmethod
    def from_workload(cls, wl) -> "Grid":
        return cls(wl.nx, wl.ny, wl.nz, wl.n_channels, [float(s) for s in wl.sigma],
                   wl.cutoff, float(wl.cutoff_k), bool(wl.periodic),
                   getattr(wl, "form", "point"))

    def to_c(self) -> B.pg_grid:
        sig = (ctypes.c_float * len(self.sigma))(*[float(s) for s in self.sigma])
        self._sigma_buf = sig
        return B.pg_grid(nx=int(self.nx), ny=int(self.ny), nz=int(self.nz),
                         n_channels=int(self.n_channels),
                         sigma=ctypes.cast(sig, ctypes.POINTER(ctypes.c_float)),
                         cutoff_k=float(self.cutoff_k), cutoff=CUTOFFS[self.cutoff],
                         periodic=1 if self.periodic else 0, voxel_form=FORMS[self.form])

    def out_shape(self, n_mol: int):
        return (n_mol, self.n_channels, self.nx, self.ny, self.nz)


def _ptr(t):
    return None if t is None or t.numel() == 0 else t.data_ptr()


class DeviceBatch:
    """CSR batch held in device tensors (float32 coords/origin/spacing, int32 ids/offsets),
    with optional per-atom weights (float32 [N]) and per-molecule cell matrices (float32
    [B, 3, 3], rows = the box edges along the grid's x, y, z axes)."""

    def __init__(self, coords, elem, mol_off, origin, spacing, weight=None, cell=None):
        self.coords = coords.reshape(-1, 3)
        self.elem = elem.reshape(-1)
        self.mol_off = mol_off.reshape(-1)
        self.origin = origin.reshape(-1, 3)
        self.spacing = spacing.reshape(-1, 3)
        self.weight = None if weight is None else weight.reshape(-1)
        self.cell = None if cell is None else cell.reshape(-1, 3, 3)
        checks = [("coords", self.coords, torch.float32), ("elem", self.elem, torch.int32),
                  ("mol_off", self.mol_off, torch.int32), ("origin", self.origin, torch.float32),
                  ("spacing", self.spacing, torch.float32)]
        if self.weight is not None:
            checks.append(("weight", self.weight, torch.float32))
        if self.cell is not None:
            checks.append(("cell", self.cell, torch.float32))
        for name, t, dt in checks:
            if t.dtype != dt:
                raise TypeError(f"{name} must be {dt}, got {t.dtype}")
            if not t.is_cuda:
                raise ValueError(f"{name} must be a CUDA tensor")
            if not t.is_contiguous():
                raise ValueError(f"{name} must be contiguous")

    @classmethod
    def from_numpy(cls, batch, device="cuda") -> "DeviceBatch":
        f = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(device=device, dtype=dt)
        w = getattr(batch, "weight", None)
        m = getattr(batch, "cell", None)
        return cls(f(batch.coords, torch.float32), f(batch.elem, torch.int32),
                   f(batch.mol_off, torch.int32), f(batch.origin, torch.float32),
                   f(batch.spacing, torch.float32),
                   None if w is None else f(w, torch.float32),
                   None if m is None else f(m, torch.float32))

    def with_weight(self, weight) -> "DeviceBatch":
        """The same batch with other per-atom weights (float32 [N], CUDA), tensors shared."""
        return DeviceBatch(self.coords, self.elem, self.mol_off, self.origin, self.spacing,
                           weight, self.cell)

    @property
    def n_mol(self) -> int:
        return int(self.mol_off.numel() - 1)

    @property
    def n_atoms(self) -> int:
        return int(self.coords.shape[0])

    def to_c(self, coords=None) -> B.pg_batch:
        c = self.coords if coords is None else coords
        return B.pg_batch(n_mol=self.n_mol, n_atoms=self.n_atoms, coords=_ptr(c),
                          elem=_ptr(self.elem), mol_off=_ptr(self.mol_off),
                          origin=_ptr(self.origin), spacing=_ptr(self.spacing),
                          weight=None if self.weight is None else _ptr(self.weight),
                          cell=None if self.cell is None else _ptr(self.cell))


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def voxelize(batch: DeviceBatch, grid: Grid, dtype: str = "f32", path: str = "auto",
             out: torch.Tensor | None = None, stream=None, coords=None) -> torch.Tensor:
    """pg_voxelize: dense grids [B, C, nx, ny, nz] in `dtype` (f32/f16/bf16)."""
    code, tdt = DTYPES[dtype]
    if out is None:
        out = torch.empty(grid.out_shape(batch.n_mol), dtype=tdt, device=batch.coords.device)
    B.check(B.pg_voxelize(batch.to_c(coords), grid.to_c(), code, _ptr(out), PATHS[path],
                          _stream(stream)))
    return out


def voxelize_tuned(batch: DeviceBatch, grid: Grid, tuning: dict, dtype: str = "f32",
                   out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """pg_voxelize_tuned with an explicit launch choice (dict of pg_tuning fields)."""
    code, tdt = DTYPES[dtype]
    if out is None:
        out = torch.empty(grid.out_shape(batch.n_mol), dtype=tdt, device=batch.coords.device)
    t = B.pg_tuning(**{k: int(v) for k, v in tuning.items()})
    B.check(B.pg_voxelize_tuned(batch.to_c(), grid.to_c(), code, _ptr(out), t, _stream(stream)))
    return out


def voxelize_backward(batch: DeviceBatch, grid: Grid, grad_out: torch.Tensor,
                      grad_coords: torch.Tensor | None = None, stream=None,
                      coords=None) -> torch.Tensor:
    """pg_voxelize_backward: dL/dx [N, 3] (float32) for upstream dL/dG = grad_out."""
    if grad_out.dtype not in TORCH_TO_PG:
        raise TypeError(f"unsupported grad dtype {grad_out.dtype}")
    grad_out = grad_out.contiguous()
    if grad_coords is None:
        grad_coords = torch.empty((batch.n_atoms, 3), dtype=torch.float32,
                                  device=batch.coords.device)
    B.check(B.pg_voxelize_backward(batch.to_c(coords), grid.to_c(), TORCH_TO_PG[grad_out.dtype],
                                   _ptr(grad_out), _ptr(grad_coords), _stream(stream)))
    return grad_coords


def voxelize_backward_weights(batch: DeviceBatch, grid: Grid, grad_out: torch.Tensor,
                              with_coords: bool = True, stream=None, coords=None):
    """pg_voxelize_backward_ex: (dL/dx [N, 3] or None, dL/dw [N]) for upstream dL/dG."""
    if grad_out.dtype not in TORCH_TO_PG:
        raise TypeError(f"unsupported grad dtype {grad_out.dtype}")
    grad_out = grad_out.contiguous()
    dev = batch.coords.device
    gc = torch.empty((batch.n_atoms, 3), dtype=torch.float32, device=dev) if with_coords else None
    gw = torch.empty(batch.n_atoms, dtype=torch.float32, device=dev)
    B.check(B.pg_voxelize_backward_ex(batch.to_c(coords), grid.to_c(),
                                      TORCH_TO_PG[grad_out.dtype], _ptr(grad_out),
                                      None if gc is None else _ptr(gc), _ptr(gw),
                                      _stream(stream)))
    return gc, gw


def refine(batch: DeviceBatch, grid: Grid, target: torch.Tensor, coords: torch.Tensor,
           iters: int, lr: float, eps: float = 0.0, work: torch.Tensor | None = None,
           stream=None):
    """pg_refine: grid reversal by gradient descent.  `coords` (float32 [N, 3], device) holds
    the start and is overwritten with the result.  Returns (loss [B], steps [B])."""
    target = target.contiguous()
    if target.dtype != torch.float32:
        raise TypeError("target must be float32")
    cb = batch.to_c(coords)
    cg = grid.to_c()
    n = B.pg_refine_work_floats(cb, cg)
    if work is None or work.numel() < n:
        work = torch.empty(max(n, 1), dtype=torch.float32, device=coords.device)
    loss = torch.empty(batch.n_mol, dtype=torch.float32, device=coords.device)
    steps = torch.empty(batch.n_mol, dtype=torch.int32, device=coords.device)
    B.check(B.pg_refine(cb, cg, _ptr(target), _ptr(coords), _ptr(work), _ptr(loss),
                        _ptr(steps), iters, lr, eps, _stream(stream)))
    return loss, steps


def sync_status(stream=None, raise_on_error: bool = True) -> int:
    """pg_sync_status: synchronize and return (and clear) the device error bits."""
    st, bits = B.pg_sync_status(_stream(stream))
    if raise_on_error and st != B.PG_OK:
        raise B.PGError(st, B.last_error())
    return bits


def autotune(batch: DeviceBatch, grid: Grid, dtype: str = "f32", path: str = "auto",
             out: torch.Tensor | None = None, stream=None) -> dict:
    """pg_autotune: time every candidate, record the fastest passing one for this bucket."""
    code, tdt = DTYPES[dtype]
    if out is None:
        out = torch.empty(grid.out_shape(batch.n_mol), dtype=tdt, device=batch.coords.device)
    st, t = B.pg_autotune(batch.to_c(), grid.to_c(), code, _ptr(out), PATHS[path],
                          _stream(stream))
    B.check(st)
    return t.as_dict()


def get_tuning(batch: DeviceBatch, grid: Grid, dtype: str = "f32", path: str = "auto") -> dict:
    st, t = B.pg_get_tuning(batch.to_c(), grid.to_c(), DTYPES[dtype][0], PATHS[path])
    B.check(st)
    return t.as_dict()


class Plan:
    """pg_plan_*: CUDA graph of (host-to-device copy of a batch + voxelization launch)."""

    def __init__(self, grid: Grid, dtype: str, max_mol: int, max_atoms: int, path: str = "auto"):
        self.grid = grid
        self.dtype = dtype
        self._cgrid = grid.to_c()
        st, h = B.pg_plan_create(self._cgrid, DTYPES[dtype][0], PATHS[path], int(max_mol),
                                 int(max_atoms))
        B.check(st)
        self._h = h

    def _host_batch(self, coords, elem, mol_off, origin, spacing, weight, cell):
        keep = []

        def host(a, dt):
            if isinstance(a, torch.Tensor):
                a = a.contiguous()
                keep.append(a)
                return a.data_ptr() if a.numel() else None
            arr = np.ascontiguousarray(a, dtype=dt)
            keep.append(arr)
            return arr.ctypes.data if arr.size else None

        n_atoms = int(len(elem))
        n_mol = int(len(mol_off) - 1)
        opt = lambda a: None if a is None else host(a, np.float32)
        hb = B.pg_batch(n_mol=n_mol, n_atoms=n_atoms, coords=host(coords, np.float32),
                        elem=host(elem, np.int32), mol_off=host(mol_off, np.int32),
                        origin=host(origin, np.float32), spacing=opt(spacing),
                        weight=opt(weight), cell=opt(cell))
        return hb, keep

    def run(self, coords, elem, mol_off, origin, spacing, out: torch.Tensor, stream=None,
            weight=None, cell=None):
        """Host arrays (numpy or CPU tensors, pinned or pageable) -> `out` on the device;
        `spacing` may be None when `cell` is given.  Synchronous: returns after the device
        error word has been read back."""
        hb, keep = self._host_batch(coords, elem, mol_off, origin, spacing, weight, cell)
        B.check(B.pg_plan_run(self._h, hb, _ptr(out), _stream(stream)))
        return out

    def launch(self, coords, elem, mol_off, origin, spacing, out: torch.Tensor, stream=None,
               weight=None, cell=None):
        """pg_plan_launch: as run(), but returns once the graph is enqueued; the host arrays
        must stay unchanged until wait()."""
        hb, keep = self._host_batch(coords, elem, mol_off, origin, spacing, weight, cell)
        self._keep = (hb, keep)
        B.check(B.pg_plan_launch(self._h, hb, _ptr(out), _stream(stream)))
        return out

    def wait(self, stream=None):
        """pg_plan_wait: synchronize the stream and check the outstanding launch's error word."""
        st = B.pg_plan_wait(self._h, _stream(stream))
        self._keep = None
        B.check(st)

    def close(self):
        if self._h:
            B.pg_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Voxelize(torch.autograd.Function):
    """G = voxelize(coords, weight); dL/dcoords (and dL/dweight for a weighted grid) through
    the hand-written adjoint kernel.  Only the inputs are saved."""

    @staticmethod
    def forward(ctx, coords, weight, batch: DeviceBatch, grid: Grid, dtype: str, path: str):
        coords = coords.contiguous()
        if weight is not None:
            batch = batch.with_weight(weight.contiguous())
        out = voxelize(batch, grid, dtype=dtype, path=path, coords=coords)
        ctx.save_for_backward(coords)
        ctx.batch = batch
        ctx.grid = grid
        ctx.weighted = weight is not None
        return out

    @staticmethod
    def backward(ctx, grad_out):
        (coords,) = ctx.saved_tensors
        if ctx.weighted and ctx.needs_input_grad[1]:
            g, gw = voxelize_backward_weights(ctx.batch, ctx.grid, grad_out,
                                              with_coords=ctx.needs_input_grad[0], coords=coords)
            return g, gw, None, None, None, None
        g = voxelize_backward(ctx.batch, ctx.grid, grad_out, coords=coords)
        return g, None, None, None, None, None


def voxelize_autograd(coords: torch.Tensor, batch: DeviceBatch, grid: Grid,
                      dtype: str = "f32", path: str = "auto",
                      weight: torch.Tensor | None = None) -> torch.Tensor:
    """Differentiable voxelization with respect to `coords` ([N, 3] float32, CUDA) and, when
    given, the per-atom `weight` ([N] float32, CUDA; it replaces the batch's own weights)."""
    return Voxelize.apply(coords, weight, batch, grid, dtype, path)
