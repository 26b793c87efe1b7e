"""ctypes binding of the C ABI declared in include/pg.h.

Argument marshalling only: every function here forwards to the function of the same name
in libpg.so.  There is no CPU fallback; if the library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

PG_OK = 0
PG_ERR_INVALID_ARG = 1
PG_ERR_UNSUPPORTED = 2
PG_ERR_CUDA = 3
PG_ERR_DEVICE_VALIDATION = 4
PG_ERR_TIMEOUT = 5

PG_F32, PG_F16, PG_BF16 = 0, 1, 2
PG_CUTOFF_SPHERE, PG_CUTOFF_NONE, PG_CUTOFF_BOX = 0, 1, 2
PG_FORM_POINT, PG_FORM_INTEGRAL = 0, 1
PG_PATH_AUTO, PG_PATH_DIRECT, PG_PATH_SEPARABLE = 0, 1, 2
PG_MAX_CHANNELS = 64

PG_DEVERR_ELEMENT = 0x1
PG_DEVERR_OFFSETS = 0x2
PG_DEVERR_SPACING = 0x4
PG_DEVERR_PERIODIC = 0x8
PG_DEVERR_TIMEOUT = 0x10
PG_DEVERR_TMEM_HELD = 0x20

EXPORTED = (
    "pg_version", "pg_last_error", "pg_status_string", "pg_voxelize", "pg_voxelize_tuned",
    "pg_voxelize_backward", "pg_sync_status", "pg_autotune", "pg_get_tuning",
    "pg_tuning_save", "pg_tuning_load", "pg_plan_create", "pg_plan_run", "pg_plan_destroy",
    "pg_shutdown", "pg_voxelize_noalloc", "pg_refine", "pg_refine_work_floats",
    "pg_voxelize_backward_ex", "pg_plan_launch", "pg_plan_wait",
)


class pg_batch(ctypes.Structure):
    _fields_ = [
        ("n_mol", ctypes.c_int32),
        ("n_atoms", ctypes.c_int32),
        ("coords", ctypes.c_void_p),
        ("elem", ctypes.c_void_p),
        ("mol_off", ctypes.c_void_p),
        ("origin", ctypes.c_void_p),
        ("spacing", ctypes.c_void_p),
        ("weight", ctypes.c_void_p),
        ("cell", ctypes.c_void_p),
    ]


class pg_grid(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32),
        ("ny", ctypes.c_int32),
        ("nz", ctypes.c_int32),
        ("n_channels", ctypes.c_int32),
        ("sigma", ctypes.POINTER(ctypes.c_float)),
        ("cutoff_k", ctypes.c_float),
        ("cutoff", ctypes.c_int32),
        ("periodic", ctypes.c_int32),
        ("voxel_form", ctypes.c_int32),
    ]


class pg_tuning(ctypes.Structure):
    _fields_ = [
        ("path", ctypes.c_int32),
        ("block_threads", ctypes.c_int32),
        ("blocks_per_sm", ctypes.c_int32),
        ("store_hint", ctypes.c_int32),
        ("n_tile", ctypes.c_int32),
        ("gather_only", ctypes.c_int32),
        ("chunk_planes", ctypes.c_int32),
        ("separable_simple", ctypes.c_int32),
        ("chunk_order", ctypes.c_int32),
    ]

    def as_dict(self):
        return {"path": self.path, "block_threads": self.block_threads,
                "blocks_per_sm": self.blocks_per_sm, "store_hint": self.store_hint,
                "n_tile": self.n_tile, "gather_only": self.gather_only,
                "chunk_planes": self.chunk_planes, "separable_simple": self.separable_simple,
                "chunk_order": self.chunk_order}


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB_PATH


def load() -> ctypes.CDLL:
    """Load libpg.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB_PATH
        if not os.path.exists(path):
            raise RuntimeError(
                f"{path} is missing: build the CUDA library first "
                "(python -c 'import __graft_entry__ as g; g.build()'); there is no CPU path")
        lib = ctypes.CDLL(path)
        P = ctypes.POINTER
        vp = ctypes.c_void_p
        i32 = ctypes.c_int32
        lib.pg_version.restype = i32
        lib.pg_last_error.restype = ctypes.c_char_p
        lib.pg_status_string.restype = ctypes.c_char_p
        lib.pg_status_string.argtypes = [i32]
        lib.pg_voxelize.argtypes = [P(pg_batch), P(pg_grid), i32, vp, i32, vp]
        lib.pg_voxelize_tuned.argtypes = [P(pg_batch), P(pg_grid), i32, vp, P(pg_tuning), vp]
        lib.pg_voxelize_backward.argtypes = [P(pg_batch), P(pg_grid), i32, vp, vp, vp]
        lib.pg_voxelize_backward_ex.argtypes = [P(pg_batch), P(pg_grid), i32, vp, vp, vp, vp]
        lib.pg_sync_status.argtypes = [vp, P(ctypes.c_uint32)]
        lib.pg_autotune.argtypes = [P(pg_batch), P(pg_grid), i32, vp, i32, vp, P(pg_tuning)]
        lib.pg_get_tuning.argtypes = [P(pg_batch), P(pg_grid), i32, i32, P(pg_tuning)]
        lib.pg_tuning_save.argtypes = [ctypes.c_char_p]
        lib.pg_tuning_load.argtypes = [ctypes.c_char_p]
        lib.pg_plan_create.argtypes = [P(vp), P(pg_grid), i32, i32, i32, i32]
        lib.pg_plan_run.argtypes = [vp, P(pg_batch), vp, vp]
        lib.pg_plan_launch.argtypes = [vp, P(pg_batch), vp, vp]
        lib.pg_plan_wait.argtypes = [vp, vp]
        lib.pg_plan_destroy.argtypes = [vp]
        lib.pg_shutdown.restype = None
        lib.pg_voxelize_noalloc.argtypes = [P(pg_batch), P(pg_grid), i32, vp, vp,
                                            P(ctypes.c_uint32)]
        lib.pg_refine.argtypes = [P(pg_batch), P(pg_grid), vp, vp, vp, vp, vp, i32,
                                  ctypes.c_float, ctypes.c_float, vp]
        lib.pg_refine_work_floats.argtypes = [P(pg_batch), P(pg_grid)]
        lib.pg_refine_work_floats.restype = ctypes.c_size_t
        for name in ("pg_voxelize", "pg_voxelize_tuned", "pg_voxelize_backward",
                     "pg_sync_status", "pg_autotune", "pg_get_tuning", "pg_tuning_save",
                     "pg_tuning_load", "pg_plan_create", "pg_plan_run", "pg_plan_destroy",
                     "pg_voxelize_noalloc", "pg_refine", "pg_plan_launch", "pg_plan_wait"):
            getattr(lib, name).restype = i32
        _lib = lib
        return lib


class PGError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{status_name(status)}: {message}")
        self.status = status


def status_name(status: int) -> str:
    return load().pg_status_string(status).decode()


def last_error() -> str:
    return load().pg_last_error().decode()


def check(status: int) -> None:
    if status != PG_OK:
        raise PGError(status, last_error())


# Thin same-name wrappers (ctypes structs and raw addresses in, status out).

def pg_version() -> int:
    return load().pg_version()


def pg_voxelize(batch, grid, out_dtype, out, path, stream):
    return load().pg_voxelize(ctypes.byref(batch), ctypes.byref(grid), out_dtype, out, path,
                              stream)


def pg_voxelize_tuned(batch, grid, out_dtype, out, tuning, stream):
    return load().pg_voxelize_tuned(ctypes.byref(batch), ctypes.byref(grid), out_dtype, out,
                                    ctypes.byref(tuning), stream)


def pg_voxelize_backward(batch, grid, grad_dtype, grad_out, grad_coords, stream):
    return load().pg_voxelize_backward(ctypes.byref(batch), ctypes.byref(grid), grad_dtype,
                                       grad_out, grad_coords, stream)


def pg_voxelize_backward_ex(batch, grid, grad_dtype, grad_out, grad_coords, grad_weight,
                            stream):
    return load().pg_voxelize_backward_ex(ctypes.byref(batch), ctypes.byref(grid), grad_dtype,
                                          grad_out, grad_coords, grad_weight, stream)


def pg_refine(batch, grid, target, coords, work, loss, steps, iters, lr, eps, stream):
    return load().pg_refine(ctypes.byref(batch), ctypes.byref(grid), target, coords, work, loss,
                            steps, int(iters), float(lr), float(eps), stream)


def pg_refine_work_floats(batch, grid):
    return load().pg_refine_work_floats(ctypes.byref(batch), ctypes.byref(grid))


def pg_sync_status(stream):
    bits = ctypes.c_uint32(0)
    st = load().pg_sync_status(stream, ctypes.byref(bits))
    return st, bits.value


def pg_autotune(batch, grid, out_dtype, out, path, stream):
    t = pg_tuning()
    st = load().pg_autotune(ctypes.byref(batch), ctypes.byref(grid), out_dtype, out, path,
                            stream, ctypes.byref(t))
    return st, t


def pg_get_tuning(batch, grid, out_dtype, path):
    t = pg_tuning()
    st = load().pg_get_tuning(ctypes.byref(batch), ctypes.byref(grid), out_dtype, path,
                              ctypes.byref(t))
    return st, t


def pg_tuning_save(path: str):
    return load().pg_tuning_save(path.encode())


def pg_tuning_load(path: str):
    return load().pg_tuning_load(path.encode())


def pg_plan_create(grid, out_dtype, path, max_mol, max_atoms):
    h = ctypes.c_void_p()
    st = load().pg_plan_create(ctypes.byref(h), ctypes.byref(grid), out_dtype, path, max_mol,
                               max_atoms)
    return st, h


def pg_plan_run(plan, host_batch, out, stream):
    return load().pg_plan_run(plan, ctypes.byref(host_batch), out, stream)


def pg_plan_launch(plan, host_batch, out, stream):
    return load().pg_plan_launch(plan, ctypes.byref(host_batch), out, stream)


def pg_plan_wait(plan, stream):
    return load().pg_plan_wait(plan, stream)


def pg_plan_destroy(plan):
    return load().pg_plan_destroy(plan)


def pg_shutdown():
    load().pg_shutdown()


def pg_voxelize_noalloc(batch, grid, out_dtype, out, stream):
    """Allocation-free forward voxelization (synchronous); returns (status, error bits)."""
    bits = ctypes.c_uint32(0)
    st = load().pg_voxelize_noalloc(ctypes.byref(batch), ctypes.byref(grid), out_dtype, out,
                                    stream, ctypes.byref(bits))
    return st, bits.value
