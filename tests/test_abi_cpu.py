"""CPU-side checks of the C ABI: the library builds, loads, exports every function that
include/pg.h declares, and rejects bad arguments on the host before touching a GPU."""
import ctypes
import os
import re

import pytest

import paper_2211_08506_gb300 as pg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    pg.build()
    from paper_2211_08506_gb300 import binding
    return binding


def declared_functions():
    text = open(os.path.join(ROOT, "include", "pg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(pg_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pg_voxelize", "pg_voxelize_backward", "pg_autotune", "pg_last_error",
                     "pg_version"):
        assert required in names


def test_library_exports_every_declared_function(lib):
    so = ctypes.CDLL(lib.library_path())
    missing = [n for n in declared_functions() if not hasattr(so, n)]
    assert not missing, f"declared in pg.h but not exported: {missing}"
    assert set(declared_functions()) == set(lib.EXPORTED)


def test_version_and_status_strings(lib):
    assert lib.pg_version() == 2
    assert lib.status_name(lib.PG_ERR_UNSUPPORTED) == "PG_ERR_UNSUPPORTED"
    assert lib.status_name(99) == "PG_ERR_UNKNOWN"


def _grid(lib, **kw):
    sig = (ctypes.c_float * 5)(0.4, 0.6, 0.6, 0.6, 0.6)
    g = lib.pg_grid(nx=32, ny=32, nz=32, n_channels=5,
                    sigma=ctypes.cast(sig, ctypes.POINTER(ctypes.c_float)), cutoff_k=3.0,
                    cutoff=0, periodic=0)
    for k, v in kw.items():
        setattr(g, k, v)
    return g, sig


@pytest.mark.parametrize("field,value,needle", [
    ("nx", 0, "grid shape"),
    ("n_channels", 0, "n_channels"),
    ("n_channels", 65, "n_channels"),
    ("cutoff", 7, "cutoff mode"),
    ("cutoff_k", -1.0, "cutoff_k"),
    ("periodic", 2, "periodic"),
    ("voxel_form", 5, "voxel_form"),
])
def test_host_validation_rejects_bad_grid(lib, field, value, needle):
    g, keep = _grid(lib, **{field: value})
    b = lib.pg_batch(n_mol=0, n_atoms=0)
    st = lib.pg_voxelize(b, g, 0, None, 0, None)
    assert st == lib.PG_ERR_INVALID_ARG
    assert needle in lib.last_error()


def test_host_validation_rejects_bad_batch_and_sigma(lib):
    g, keep = _grid(lib)
    st = lib.pg_voxelize(lib.pg_batch(n_mol=-1, n_atoms=0), g, 0, None, 0, None)
    assert st == lib.PG_ERR_INVALID_ARG and "negative" in lib.last_error()
    st = lib.pg_voxelize(lib.pg_batch(n_mol=3, n_atoms=10), g, 0, None, 0, None)
    assert st == lib.PG_ERR_INVALID_ARG and "required" in lib.last_error()
    keep[2] = 0.0
    st = lib.pg_voxelize(lib.pg_batch(n_mol=0, n_atoms=0), g, 0, None, 0, None)
    assert st == lib.PG_ERR_INVALID_ARG and "sigma[2]" in lib.last_error()
    g2, k2 = _grid(lib)
    st = lib.pg_voxelize(lib.pg_batch(n_mol=0, n_atoms=0), g2, 0, None, 9, None)
    assert st == lib.PG_ERR_INVALID_ARG and "path" in lib.last_error()


def test_null_arguments_do_not_crash(lib):
    L = lib.load()
    assert L.pg_voxelize(None, None, 0, None, 0, None) == lib.PG_ERR_INVALID_ARG
    assert L.pg_voxelize_tuned(None, None, 0, None, None, None) == lib.PG_ERR_INVALID_ARG
    assert L.pg_voxelize_backward(None, None, 0, None, None, None) == lib.PG_ERR_INVALID_ARG
    assert L.pg_voxelize_backward_ex(None, None, 0, None, None, None, None) == \
        lib.PG_ERR_INVALID_ARG
    assert L.pg_plan_create(None, None, 0, 0, 0, 0) == lib.PG_ERR_INVALID_ARG
    assert L.pg_plan_run(None, None, None, None) == lib.PG_ERR_INVALID_ARG
    assert L.pg_tuning_save(None) == lib.PG_ERR_INVALID_ARG


def test_tuning_cache_file_round_trip(lib, tmp_path):
    f = tmp_path / "tune.txt"
    f.write_text("GPU|32x32x32|C5|dt0|cut0|per0|apm4|path0 1 256 2 1 128\n")
    assert lib.pg_tuning_load(str(f)) == 0
    out = tmp_path / "out.txt"
    assert lib.pg_tuning_save(str(out)) == 0
    assert "path0 1 256 2 1 128 0 8 0 0" in out.read_text()
    bad = tmp_path / "bad.txt"
    bad.write_text("key only\n")
    assert lib.pg_tuning_load(str(bad)) == lib.PG_ERR_INVALID_ARG


def test_refine_rejects_bad_arguments_on_the_host(lib):
    g, keep = _grid(lib)
    L = lib.load()
    b = lib.pg_batch(n_mol=1, n_atoms=1)
    bad = [
        (dict(iters=-1, lr=0.1, eps=0.0), "iters"),
        (dict(iters=3, lr=-1.0, eps=0.0), "lr"),
        (dict(iters=3, lr=float("inf"), eps=0.0), "lr"),
        (dict(iters=3, lr=0.1, eps=-1.0), "eps"),
    ]
    for kw, needle in bad:
        st = L.pg_refine(b, g, None, None, None, None, None, kw["iters"], kw["lr"], kw["eps"],
                         None)
        assert st == lib.PG_ERR_INVALID_ARG and needle in lib.last_error(), (kw, lib.last_error())
    assert L.pg_refine_work_floats(b, g) == 5 * 32 ** 3 + 3



def test_cells_and_weights_are_validated_on_the_host(lib):
    L = lib.load()
    fake = ctypes.c_void_p(16)  # never dereferenced: every case fails before any launch
    cell = dict(n_mol=1, n_atoms=1, coords=fake, elem=fake, mol_off=fake, origin=fake,
                cell=fake)
    g, keep = _grid(lib, voxel_form=1)
    st = L.pg_voxelize(lib.pg_batch(**cell), g, 0, fake, 0, None)
    assert st == lib.PG_ERR_UNSUPPORTED and "axis-aligned" in lib.last_error()
    g, keep = _grid(lib, periodic=1, cutoff=1)
    st = L.pg_voxelize(lib.pg_batch(**cell), g, 0, fake, 0, None)
    assert st == lib.PG_ERR_UNSUPPORTED and "cutoff" in lib.last_error()
    # Spacing may be absent only when a cell replaces it.
    nocell = dict(cell)
    nocell.pop("cell")
    g, keep = _grid(lib)
    st = L.pg_voxelize(lib.pg_batch(**nocell), g, 0, fake, 0, None)
    assert st == lib.PG_ERR_INVALID_ARG and "spacing" in lib.last_error()
    # The weight adjoint needs at least one output.
    st = L.pg_voxelize_backward_ex(lib.pg_batch(**cell), g, 0, fake, None, None, None)
    assert st == lib.PG_ERR_INVALID_ARG and "both" in lib.last_error()
