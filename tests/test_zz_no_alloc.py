"""pg_voxelize_noalloc: forward voxelization that allocates no device memory.

It exists for callers that cannot let a library allocate: code running while another thread
holds a global-mode stream capture open (cudaMalloc is refused then, and the attempt
invalidates that capture), programs whose device memory is all reserved by a framework's
caching allocator or an external budget, and hosts that freeze their device-memory
footprint after start-up.  Its scratch (work counter and error word) lives in a fixed array
inside the library.

Called through the C ABI, its grids must equal, bit for bit, those of pg_voxelize_tuned with
the direct path's default launch, on two calls in a row (the second reuses the array the
first left behind), and match the FP64 oracle on a sample; a call after one that flagged bad
input must start clean.  In a fresh process it must work as the very first call into the
library without creating the library's per-device state, and it must run while another
thread holds a global-mode capture open without disturbing that capture.
This file is collected last so that a run stopping at the first failure has already run
every other test.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import synth
from tests.parity import ABS_TOL, TOL, grid_check

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DEFAULT_DIRECT = {"path": 1}   # zeroed pg_tuning with path = PG_PATH_DIRECT


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2211_08506_gb300 as pkg
    pkg.build()
    from paper_2211_08506_gb300 import api, binding
    return api, binding


def _noalloc(api, B, db, grid, dtype, out, stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return B.pg_voxelize_noalloc(db.to_c(), grid.to_c(), api.DTYPES[dtype][0], out.data_ptr(),
                                 s.cuda_stream)


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_noalloc_matches_regular_entry_point_on_two_calls(lib, dtype):
    api, B = lib
    wl = synth.qm9_shaped(n_mol=256)
    db = api.DeviceBatch.from_numpy(wl.batch)
    grid = api.Grid.from_workload(wl)
    ref = api.voxelize_tuned(db, grid, DEFAULT_DIRECT, dtype=dtype)
    assert api.sync_status() == 0
    for _ in range(2):
        out = torch.full(ref.shape, float("nan"), dtype=api.DTYPES[dtype][1], device="cuda")
        st, bits = _noalloc(api, B, db, grid, dtype, out)
        assert st == B.PG_OK, B.last_error()
        assert bits == 0
        assert torch.equal(out, ref)
    idx = np.array([0, 37, 101, 255])
    grid_check(out[torch.as_tensor(idx, device="cuda")].float().cpu().numpy(),
               oracle.Problem.from_workload(wl, batch=wl.batch.subset(idx)), TOL[dtype],
               abs_tol=ABS_TOL[dtype])


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
    ref = api.voxelize_tuned(db, grid, DEFAULT_DIRECT, dtype="f32")
    assert api.sync_status() == 0
    assert torch.equal(out, ref)
    grid_check(out.cpu().numpy(), oracle.Problem.from_workload(wl), TOL["f32"],
               abs_tol=ABS_TOL["f32"])


def _child():
    """Runs in a fresh process: the library's first call is pg_voxelize_noalloc; then a
    second call while another thread holds a global-mode capture open; markers go to stderr
    so that they interleave in order with the library's allocation trace."""
    import threading

    sys.path.insert(0, ROOT)
    from paper_2211_08506_gb300 import api, binding as B

    def mark(text):
        print(text, file=sys.stderr, flush=True)

    wl = synth.qm9_shaped(n_mol=64)
    db = api.DeviceBatch.from_numpy(wl.batch)
    grid = api.Grid.from_workload(wl)
    outs = [torch.empty(grid.out_shape(64), dtype=torch.float32, device="cuda")
            for _ in range(2)]
    stream = torch.cuda.Stream()        # created with cudaStreamNonBlocking
    cb, cg = db.to_c(), grid.to_c()
    torch.cuda.synchronize()
    mark("CHILD first-call")
    st, bits = B.pg_voxelize_noalloc(cb, cg, B.PG_F32, outs[0].data_ptr(), stream.cuda_stream)
    mark(f"CHILD first-status {st} {bits}")

    x = torch.ones(4096, device="cuda")
    cap_stream = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    opened, release, errors = threading.Event(), threading.Event(), []

    def capture():
        try:
            with torch.cuda.graph(graph, stream=cap_stream, capture_error_mode="global"):
                x.mul_(2.0)
                opened.set()
                release.wait(60)
                x.add_(1.0)
        except Exception as e:  # reported by the parent
            errors.append(repr(e))
        finally:
            opened.set()

    t = threading.Thread(target=capture)
    t.start()
    opened.wait(60)
    mark("CHILD capture-open")
    st2, bits2 = B.pg_voxelize_noalloc(cb, cg, B.PG_F32, outs[1].data_ptr(), stream.cuda_stream)
    release.set()
    t.join(60)
    mark(f"CHILD capture-status {st2} {bits2} errors={len(errors)} {errors}")
    if st2 != B.PG_OK:
        mark(f"CHILD capture-message {B.last_error()}")
    if not errors:
        graph.replay()
        torch.cuda.synchronize()
    mark(f"CHILD replay {not errors and bool(torch.all(x == 3.0))}")
    mark("CHILD regular-call")
    ref = api.voxelize_tuned(db, grid, DEFAULT_DIRECT, dtype="f32")
    api.sync_status()
    mark(f"CHILD equal {torch.equal(outs[0], ref)} {torch.equal(outs[1], ref)}")


def test_noalloc_first_call_in_fresh_process_and_during_foreign_capture(lib):
    env = dict(os.environ, PG_DEBUG_LAUNCH="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--child"], cwd=ROOT,
                       env=env, capture_output=True, text=True, timeout=600)
    log = r.stderr
    assert r.returncode == 0, log[-4000:]
    lines = [l for l in log.splitlines() if l.startswith(("CHILD", "[pg] per-device"))]
    assert "CHILD first-status 0 0" in lines, log[-4000:]
    # The capture opened in another thread survives the call and replays correctly.
    assert "CHILD capture-status 0 0 errors=0 []" in lines, log[-4000:]
    assert "CHILD replay True" in lines, log[-4000:]
    assert "CHILD equal True True" in lines, log[-4000:]
    # No per-device state is allocated before the first regular call.
    first_alloc = next((i for i, l in enumerate(lines) if l.startswith("[pg] per-device")),
                       len(lines))
    assert lines.index("CHILD regular-call") < first_alloc, lines


if __name__ == "__main__" and "--child" in sys.argv:
    _child()
