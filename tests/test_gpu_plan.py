"""GPU checks of the end-to-end plan (pg_plan_*): a CUDA graph holding the host-to-device
copies of a CSR batch and the voxelization launch.  The graph is updated in place per run,
so the tests change batch size, input memory kind (pinned or pageable) and voxel form
between runs. Each result must equal the stream-ordered pg_voxelize bit for bit. Capacity
limits are rejected on the host, and device-detected errors come back as a status."""
import numpy as np
import pytest

import synth
from tests.parity import TOL, grid_check
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2211_08506_gb300 as pkg
    pkg.build()
    from paper_2211_08506_gb300 import api
    return api


def direct(pg, wl, batch, dtype):
    G = pg.voxelize(pg.DeviceBatch.from_numpy(batch), pg.Grid.from_workload(wl), dtype=dtype,
                    path="direct")
    assert pg.sync_status() == 0
    return G


def host_arrays(batch, pinned):
    arrs = [batch.coords.astype(np.float32).reshape(-1), batch.elem.astype(np.int32),
            batch.mol_off.astype(np.int32), batch.origin.astype(np.float32).reshape(-1),
            batch.spacing.astype(np.float32).reshape(-1)]
    if pinned:
        return [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in arrs]
    return arrs


@pytest.mark.parametrize("form", ["point", "integral"])
def test_plan_runs_equal_stream_launches_across_sizes(pg, form):
    wl = synth.qm9_shaped(n_mol=96)
    wl.form = form
    grid = pg.Grid.from_workload(wl)
    plan = pg.Plan(grid, "f32", max_mol=96, max_atoms=int(wl.batch.n_atoms), path="direct")
    try:
        for n, pinned in [(96, True), (17, False), (1, True), (64, False), (96, False)]:
            sub = wl.batch.subset(range(n))
            out = torch.empty(grid.out_shape(n), dtype=torch.float32, device="cuda")
            plan.run(*host_arrays(sub, pinned), out=out)
            ref = direct(pg, wl, sub, "f32")
            assert torch.equal(out, ref), (n, pinned)
        grid_check(out[:3].cpu().numpy(),
                   oracle.Problem.from_workload(wl, batch=wl.batch.subset(range(3))),
                   TOL["f32"])
    finally:
        plan.close()


def test_plan_rejects_batches_over_capacity(pg):
    wl = synth.qm9_shaped(n_mol=8)
    grid = pg.Grid.from_workload(wl)
    plan = pg.Plan(grid, "f16", max_mol=4, max_atoms=1000)
    try:
        out = torch.empty(grid.out_shape(8), dtype=torch.float16, device="cuda")
        with pytest.raises(Exception, match="capacity"):
            plan.run(*host_arrays(wl.batch, False), out=out)
        # The plan stays usable after a rejected call.
        sub = wl.batch.subset(range(4))
        out4 = torch.empty(grid.out_shape(4), dtype=torch.float16, device="cuda")
        plan.run(*host_arrays(sub, False), out=out4)
        assert torch.equal(out4, direct(pg, wl, sub, "f16"))
    finally:
        plan.close()


def test_plan_reports_device_detected_errors(pg):
    # An element id outside [0, C) is found on the device; the run returns an error status
    # (the plan reads the error word back) and the next valid run succeeds.
    wl = synth.qm9_shaped(n_mol=4)
    grid = pg.Grid.from_workload(wl)
    plan = pg.Plan(grid, "f32", max_mol=4, max_atoms=int(wl.batch.n_atoms), path="direct")
    try:
        bad = host_arrays(wl.batch, False)
        bad[1] = bad[1].copy()
        bad[1][2] = 9
        out = torch.empty(grid.out_shape(4), dtype=torch.float32, device="cuda")
        with pytest.raises(Exception):
            plan.run(*bad, out=out)
        plan.run(*host_arrays(wl.batch, False), out=out)
        assert torch.equal(out, direct(pg, wl, wl.batch, "f32"))
    finally:
        plan.close()



def test_plan_launch_then_adjoint_then_wait(pg):
    # pg_plan_launch enqueues the copies and the forward pass without synchronizing; the
    # adjoint and the gradient's copy to the host follow on the same stream; pg_plan_wait
    # waits for the plan's own work and reports its error word.  Results equal the
    # synchronous calls.
    wl = synth.differentiation(n_mol=24)
    grid = pg.Grid.from_workload(wl)
    db = pg.DeviceBatch.from_numpy(wl.batch)
    W = torch.as_tensor(synth.loss_weights(wl), device="cuda")
    stream = torch.cuda.Stream()
    plan = pg.Plan(grid, "f32", max_mol=24, max_atoms=int(wl.batch.n_atoms), path="direct")
    try:
        out = torch.empty(grid.out_shape(24), dtype=torch.float32, device="cuda")
        grad = torch.empty((wl.batch.n_atoms, 3), dtype=torch.float32, device="cuda")
        grad_host = torch.empty_like(grad, device="cpu").pin_memory()
        host = host_arrays(wl.batch, True)
        plan.wait(stream)  # nothing outstanding: a no-op
        for _ in range(2):
            plan.launch(*host, out=out, stream=stream)
            with pytest.raises(Exception, match="waited"):
                plan.launch(*host, out=out, stream=stream)
            pg.voxelize_backward(db, grid, W, grad_coords=grad, stream=stream)
            grad_host.copy_(grad, non_blocking=True)
            plan.wait(stream)      # the plan's own copies, kernel and error word
            stream.synchronize()   # the adjoint and the gradient copy that follow it
            assert torch.equal(out, direct(pg, wl, wl.batch, "f32"))
            ref = pg.voxelize_backward(db, grid, W)
            assert pg.sync_status() == 0
            assert torch.equal(grad_host, ref.cpu())
        # A device-detected error is reported by the wait.
        bad = host_arrays(wl.batch, False)
        bad[1] = bad[1].copy()
        bad[1][0] = 9
        plan.launch(*bad, out=out, stream=stream)
        with pytest.raises(Exception):
            plan.wait(stream)
    finally:
        plan.close()

_CACHE_CHILD = r"""
import json, sys
sys.path.insert(0, sys.argv[2])
import synth
from paper_2211_08506_gb300 import api
wl = synth.qm9_shaped(n_mol=64)
db = api.DeviceBatch.from_numpy(wl.batch)
grid = api.Grid.from_workload(wl)
if sys.argv[1] == "tune":
    print(json.dumps(api.autotune(db, grid, dtype="f32", path="direct")))
else:
    print(json.dumps(api.get_tuning(db, grid, dtype="f32", path="direct")))
"""


def test_two_plans_alternate(pg):
    # Double buffering: batch i is launched on one plan before batch i - 1's plan is waited
    # for; every output equals the stream-ordered call on its own batch.
    wl = synth.qm9_shaped(n_mol=72)
    grid = pg.Grid.from_workload(wl)
    plans = [pg.Plan(grid, "f16", max_mol=20, max_atoms=int(wl.batch.n_atoms), path="direct")
             for _ in range(2)]
    stream = torch.cuda.Stream()
    try:
        subs = [wl.batch.subset(range(k * 10, k * 10 + 10 + k % 3)) for k in range(6)]
        outs = [torch.empty(grid.out_shape(s.n_mol), dtype=torch.float16, device="cuda")
                for s in subs]
        hosts = [host_arrays(s, True) for s in subs]
        plans[0].launch(*hosts[0], out=outs[0], stream=stream)
        for i in range(1, len(subs)):
            plans[i % 2].launch(*hosts[i], out=outs[i], stream=stream)
            plans[(i - 1) % 2].wait(stream)
        plans[(len(subs) - 1) % 2].wait(stream)
        for s, o in zip(subs, outs):
            assert torch.equal(o, direct(pg, wl, s, "f16"))
    finally:
        for p in plans:
            p.close()


def test_tuning_cache_file_named_by_the_environment(pg, tmp_path):
    # PG_TUNING_CACHE: a tuning run writes the cache file; a fresh process merges it on first
    # use, so PG_PATH_DIRECT resolves to the stored launch without tuning again.
    import json
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    path = tmp_path / "tuning.txt"
    env = dict(os.environ, PG_TUNING_CACHE=str(path))

    def child(mode):
        r = subprocess.run([sys.executable, "-c", _CACHE_CHILD, mode, root], env=env,
                           capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-3000:]
        return json.loads(r.stdout.strip().splitlines()[-1])

    child("tune")
    lines = path.read_text().splitlines()
    key = next(l.split()[0] for l in lines if "|path1" in l.split()[0] and "|dt0|" in l)
    # A distinctive stored launch for that bucket, which the tuner itself would not pick.
    rest = [l for l in lines if l.split()[0] != key]
    path.write_text("\n".join(rest + [f"{key} 1 512 1 0 128 1 3 0 1"]) + "\n")
    got = child("get")
    assert (got["block_threads"], got["blocks_per_sm"], got["chunk_planes"],
            got["chunk_order"]) == (512, 1, 3, 1), got
