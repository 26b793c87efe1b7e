"""pg_voxelize_noalloc: forward voxelization that allocates no device memory.

It exists for callers that cannot let a library allocate: code running while a
global-mode stream capture is open elsewhere in the process (cudaMalloc is refused then),
programs whose device memory is all reserved by a framework's caching allocator or an
external budget, and hosts that freeze their device-memory footprint after start-up.  Its
scratch (work counter and error word) lives in a fixed array inside the library.

Called through the C ABI, its grids must match pg_voxelize's on the direct path within the
tolerances the other parity tests use, on two calls in a row (the second reuses the array
the first left behind), and a call after one that flagged bad input must start clean.
This file is collected last so that a run stopping at the first failure has already run
every other test.
"""
import pytest

import synth
from tests.parity import TOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2211_08506_gb300 as pkg
    pkg.build()
    from paper_2211_08506_gb300 import api, binding
    return api, binding


def _noalloc(api, B, db, grid, dtype, out):
    st, bits = B.pg_voxelize_noalloc(db.to_c(), grid.to_c(), api.DTYPES[dtype][0],
                                     out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return st, bits


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_noalloc_matches_regular_entry_point_on_two_calls(lib, dtype):
    api, B = lib
    wl = synth.qm9_shaped(n_mol=256)
    db = api.DeviceBatch.from_numpy(wl.batch)
    grid = api.Grid.from_workload(wl)
    ref = api.voxelize(db, grid, dtype=dtype, path="direct").float()
    assert api.sync_status() == 0
    m = ref.abs().amax(dim=(1, 2, 3, 4))
    for _ in range(2):
        out = torch.full(ref.shape, float("nan"), dtype=api.DTYPES[dtype][1], device="cuda")
        st, bits = _noalloc(api, B, db, grid, dtype, out)
        assert st == B.PG_OK, B.last_error()
        assert bits == 0
        diff = (out.float() - ref).abs().amax(dim=(1, 2, 3, 4))
        assert torch.all(diff <= TOL[dtype] * m)


def test_noalloc_reports_bad_input_then_starts_clean(lib):
    api, B = lib
    wl = synth.plain_small(n_mol=3)
    bad = synth.Batch(wl.batch.coords.copy(), wl.batch.elem.copy(), wl.batch.mol_off.copy(),
                      wl.batch.origin.copy(), wl.batch.spacing.copy())
    bad.elem[1] = 11
    grid = api.Grid.from_workload(wl)
    out = torch.empty(grid.out_shape(3), dtype=torch.float32, device="cuda")
    st, bits = _noalloc(api, B, api.DeviceBatch.from_numpy(bad), grid, "f32", out)
    assert st == B.PG_ERR_DEVICE_VALIDATION and bits & B.PG_DEVERR_ELEMENT
    db = api.DeviceBatch.from_numpy(wl.batch)
    st, bits = _noalloc(api, B, db, grid, "f32", out)
    assert st == B.PG_OK and bits == 0
    ref = api.voxelize(db, grid, dtype="f32", path="direct")
    assert api.sync_status() == 0
    m = ref.abs().amax(dim=(1, 2, 3, 4))
    assert torch.all((out - ref).abs().amax(dim=(1, 2, 3, 4)) <= TOL["f32"] * m)
