"""FP64 CPU oracle for Gaussian-density voxelization (ParticleGrid, arXiv 2211.08506).

TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the benchmark's CPU
baseline are the only code allowed to import this package.  It shares no code with the
CUDA library (``paper_2211_08506_gb300``): the arithmetic lives in ``pg_oracle.c``
(plain C, FP64, optional OpenMP over molecules) and this module only builds, loads and
marshals it.

Functions (each mirrors one C entry point; see the C file for the equations):

* ``voxelize(wl_or_batch, ..., mode="bbox"|"brute")``    - Sec. III-A, Eq. 1, point sampled,
  or (``form="integral"``) integrated over each voxel with the per-axis erf factors
* ``voxelize_band(...)``                                 - same, split at the cutoff surface
* ``separable(...)``                                     - Sec. III-A / VI-A per-axis form
* ``gradient(...)``                                      - Sec. IV-C, dL/dx for L = <W, G>
* ``gradient_weight(...)``                               - dL/dw of a weighted grid
* ``fd_gradient_frozen(...)``                            - central differences, frozen support
* ``refine(...)``                                        - Sec. IV-A/IV-C grid reversal by descent
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libpg_oracle.so")

CUTOFFS = {"sphere": 0, "none": 1, "box": 2}
FORMS = {"point": 0, "integral": 1}
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile pg_oracle.c into a shared library (gcc, -O2, OpenMP, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and \
            os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(ctypes.Structure):
    _fields_ = [
        ("n_mol", ctypes.c_int32),
        ("mol_off", ctypes.c_void_p),
        ("coords", ctypes.c_void_p),
        ("elem", ctypes.c_void_p),
        ("origin", ctypes.c_void_p),
        ("spacing", ctypes.c_void_p),
        ("nx", ctypes.c_int32),
        ("ny", ctypes.c_int32),
        ("nz", ctypes.c_int32),
        ("n_channels", ctypes.c_int32),
        ("sigma", ctypes.c_void_p),
        ("cutoff_k", ctypes.c_double),
        ("cutoff", ctypes.c_int32),
        ("periodic", ctypes.c_int32),
        ("form", ctypes.c_int32),
        ("weight", ctypes.c_void_p),
        ("cell", ctypes.c_void_p),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(_Problem)
            dp = ctypes.c_void_p
            lib.pgo_voxelize.argtypes = [P, ctypes.c_int, dp, ctypes.c_int]
            lib.pgo_voxelize_band.argtypes = [P, ctypes.c_double, dp, dp, ctypes.c_int]
            lib.pgo_separable.argtypes = [P, dp, ctypes.c_int]
            lib.pgo_gradient.argtypes = [P, ctypes.c_int, dp, dp, ctypes.c_int]
            lib.pgo_gradient_weight.argtypes = [P, ctypes.c_int, dp, dp, ctypes.c_int]
            lib.pgo_fd_gradient_frozen.argtypes = [P, dp, ctypes.c_double, dp, ctypes.c_int]
            lib.pgo_refine.argtypes = [P, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                       dp, dp, dp, ctypes.c_int]
            lib.pgo_refine.restype = ctypes.c_int
            lib.pgo_inner.argtypes = [dp, dp, ctypes.c_long]
            lib.pgo_inner.restype = ctypes.c_double
            for f in (lib.pgo_voxelize, lib.pgo_voxelize_band, lib.pgo_separable,
                      lib.pgo_gradient, lib.pgo_gradient_weight, lib.pgo_fd_gradient_frozen):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


class Problem:
    """FP64 copy of a batch plus its grid description, kept alive for ctypes.

    ``weight`` (per atom) and ``cell`` (per molecule, 3x3 rows = box edges) default to the
    batch's own (``batch.weight`` / ``batch.cell`` when present); pass them to override."""

    def __init__(self, batch, nx, ny, nz, n_channels, sigma, cutoff="sphere", cutoff_k=3.0,
                 periodic=False, coords=None, form="point", weight=None, cell=None):
        self.mol_off = np.ascontiguousarray(batch.mol_off, np.int32)
        src = batch.coords if coords is None else coords
        self.coords = np.ascontiguousarray(np.asarray(src, np.float64).reshape(-1, 3))
        self.elem = np.ascontiguousarray(batch.elem, np.int32)
        self.origin = np.ascontiguousarray(np.asarray(batch.origin, np.float64).reshape(-1, 3))
        self.spacing = np.ascontiguousarray(np.asarray(batch.spacing, np.float64).reshape(-1, 3))
        self.sigma = np.ascontiguousarray(np.asarray(sigma, np.float64).reshape(-1))
        self.shape = (self.mol_off.shape[0] - 1, int(n_channels), int(nx), int(ny), int(nz))
        if self.sigma.shape[0] != n_channels:
            raise ValueError("sigma must have one entry per channel")
        w = weight if weight is not None else getattr(batch, "weight", None)
        m = cell if cell is not None else getattr(batch, "cell", None)
        self.weight = None if w is None else np.ascontiguousarray(
            np.asarray(w, np.float64).reshape(-1))
        self.cell = None if m is None else np.ascontiguousarray(
            np.asarray(m, np.float64).reshape(-1, 3, 3))
        if self.weight is not None and self.weight.shape[0] != self.coords.shape[0]:
            raise ValueError("weight must have one entry per atom")
        if self.cell is not None and self.cell.shape[0] != self.shape[0]:
            raise ValueError("cell must have one 3x3 matrix per molecule")
        self.c = _Problem(
            n_mol=self.shape[0],
            mol_off=self.mol_off.ctypes.data,
            coords=self.coords.ctypes.data,
            elem=self.elem.ctypes.data,
            origin=self.origin.ctypes.data,
            spacing=self.spacing.ctypes.data,
            nx=int(nx), ny=int(ny), nz=int(nz), n_channels=int(n_channels),
            sigma=self.sigma.ctypes.data,
            cutoff_k=float(cutoff_k),
            cutoff=CUTOFFS[cutoff],
            periodic=1 if periodic else 0,
            form=FORMS[form],
            weight=None if self.weight is None else self.weight.ctypes.data,
            cell=None if self.cell is None else self.cell.ctypes.data,
        )

    @classmethod
    def from_workload(cls, wl, batch=None, coords=None):
        return cls(batch if batch is not None else wl.batch, wl.nx, wl.ny, wl.nz,
                   wl.n_channels, wl.sigma, wl.cutoff, wl.cutoff_k, wl.periodic, coords,
                   getattr(wl, "form", "point"))


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def voxelize(prob: Problem, mode: str = "bbox", threads: int = 0) -> np.ndarray:
    out = np.empty(prob.shape, np.float64)
    _check(_load().pgo_voxelize(ctypes.byref(prob.c), 0 if mode == "brute" else 1,
                                out.ctypes.data, threads), "voxelize")
    return out


def voxelize_band(prob: Problem, eps: float = 1e-5, threads: int = 0):
    """(inside, band): contributions inside the cutoff by more than a relative margin eps,
    and every contribution (inside or just outside) within eps of the cutoff surface."""
    g_in = np.empty(prob.shape, np.float64)
    g_band = np.empty(prob.shape, np.float64)
    _check(_load().pgo_voxelize_band(ctypes.byref(prob.c), eps, g_in.ctypes.data,
                                     g_band.ctypes.data, threads), "voxelize_band")
    return g_in, g_band


def separable(prob: Problem, threads: int = 0) -> np.ndarray:
    out = np.empty(prob.shape, np.float64)
    _check(_load().pgo_separable(ctypes.byref(prob.c), out.ctypes.data, threads), "separable")
    return out


def gradient(prob: Problem, W: np.ndarray, mode: str = "bbox", threads: int = 0) -> np.ndarray:
    W = np.ascontiguousarray(W, np.float64).reshape(prob.shape)
    g = np.empty((prob.coords.shape[0], 3), np.float64)
    _check(_load().pgo_gradient(ctypes.byref(prob.c), 0 if mode == "brute" else 1,
                                W.ctypes.data, g.ctypes.data, threads), "gradient")
    return g


def gradient_weight(prob: Problem, W: np.ndarray, mode: str = "bbox",
                    threads: int = 0) -> np.ndarray:
    """dL/dw_a of L = <W, G> for a weighted grid: each atom's unweighted terms against W."""
    W = np.ascontiguousarray(W, np.float64).reshape(prob.shape)
    g = np.empty(prob.coords.shape[0], np.float64)
    _check(_load().pgo_gradient_weight(ctypes.byref(prob.c), 0 if mode == "brute" else 1,
                                       W.ctypes.data, g.ctypes.data, threads),
           "gradient_weight")
    return g


def fd_gradient_frozen(prob: Problem, W: np.ndarray, step: float = 1e-4,
                       threads: int = 0) -> np.ndarray:
    W = np.ascontiguousarray(W, np.float64).reshape(prob.shape)
    g = np.empty((prob.coords.shape[0], 3), np.float64)
    _check(_load().pgo_fd_gradient_frozen(ctypes.byref(prob.c), W.ctypes.data, float(step),
                                          g.ctypes.data, threads), "fd_gradient_frozen")
    return g


def refine(prob: Problem, target: np.ndarray, iters: int, lr: float, eps: float = 0.0,
           threads: int = 0):
    """Grid reversal by gradient descent (Sec. IV-A, IV-C) from the problem's coordinates
    towards `target` ([B][C][nx][ny][nz]).  Returns (coords [N][3], loss [B], steps [B])."""
    T = np.ascontiguousarray(target, np.float64).reshape(prob.shape)
    out = np.empty_like(prob.coords)
    loss = np.empty(prob.shape[0], np.float64)
    steps = np.empty(prob.shape[0], np.int32)
    _check(_load().pgo_refine(ctypes.byref(prob.c), T.ctypes.data, int(iters), float(lr),
                              float(eps), out.ctypes.data, loss.ctypes.data, steps.ctypes.data,
                              threads), "refine")
    return out, loss, steps


def loss(prob: Problem, W: np.ndarray, threads: int = 0) -> float:
    """L = <W, G(x)> with G from the support-box oracle."""
    G = voxelize(prob, "bbox", threads)
    W = np.ascontiguousarray(W, np.float64).reshape(prob.shape)
    return float(_load().pgo_inner(W.ctypes.data, G.ctypes.data, G.size))
