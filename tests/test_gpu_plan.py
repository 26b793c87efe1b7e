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
