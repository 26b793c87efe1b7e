"""GPU parity of general cells and weighted grids (Sec. III-A) against the FP64 oracle.

General cells run on their own kernel (fractional-coordinate staging, nearest image by
per-axis rounding under the reach condition).  Weights run through every forward path
(direct point and erf forms, separable one-stage and pipelined) and through the adjoint,
which also returns the weight gradient.  Plans, refinement, the tuner and the no-alloc
entry accept both; device-detected errors (singular cell, cutoff reaching half a cell)
come back as status bits."""
import numpy as np
import pytest

import oracle
import synth
from tests.parity import ABS_TOL, GRAD_TOL, SEPARABLE_TOL, TOL, grad_check, grid_check

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


def triclinic(n_cells=6, shape=(24, 20, 28)):
    wl = synth.crystal_triclinic(n_cells=n_cells)
    wl.nx, wl.ny, wl.nz = shape
    return wl


def run(pg, wl, dtype="f32", path="direct", batch=None):
    b = wl.batch if batch is None else batch
    G = pg.voxelize(pg.DeviceBatch.from_numpy(b), pg.Grid.from_workload(wl), dtype=dtype,
                    path=path)
    assert pg.sync_status() == 0
    return G


def check(G, wl, dtype, batch=None, tol=None):
    prob = oracle.Problem.from_workload(wl, batch=batch)
    return grid_check(G.float().cpu().numpy(), prob, tol or TOL[dtype], abs_tol=ABS_TOL[dtype])


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_triclinic_cells_match_oracle(pg, dtype):
    wl = triclinic()
    st = check(run(pg, wl, dtype), wl, dtype)
    assert st["max_abs_rel"] < TOL[dtype]


@pytest.mark.parametrize("cutoff,periodic", [("sphere", False), ("box", False),
                                             ("none", False), ("box", True)])
def test_cutoffs_and_open_cells(pg, cutoff, periodic):
    wl = triclinic(n_cells=4, shape=(20, 24, 16))
    wl.cutoff, wl.periodic = cutoff, periodic
    if cutoff == "box" and periodic:
        # The box reaches sqrt(3) r_c: keep the cutoff inside half of every cell width.
        wl.cutoff_k = 1.5
    check(run(pg, wl), wl, "f32")


def test_diagonal_cell_matches_the_axis_aligned_kernel(pg):
    wl = synth.crystal_shaped(n_cells=4, grid=24)
    wl.out_dtype = "f32"
    G0 = run(pg, wl)
    b = wl.batch
    b.cell = np.stack([np.diag(b.spacing[m].astype(np.float64) * 24) for m in range(b.n_mol)]
                      ).astype(np.float32)
    G1 = run(pg, wl)
    ref = float(G0.abs().max())
    assert float((G0 - G1).abs().max()) <= 2 * TOL["f32"] * ref


def test_more_channel_atoms_than_the_stage_holds(pg):
    # One channel with 300 atoms: the kernel reads the candidates from global memory.
    rng = np.random.default_rng(5)
    M, frac, _ = synth.triclinic_cell(rng, 300, edge_lo=13.0, edge_hi=15.0)
    wl = triclinic(n_cells=1)
    wl.batch = synth.Batch(coords=(frac @ M).astype(np.float32),
                           elem=np.zeros(300, np.int32), mol_off=np.array([0, 300], np.int32),
                           origin=np.zeros((1, 3), np.float32),
                           spacing=np.ones((1, 3), np.float32),
                           weight=rng.uniform(0.5, 1.5, 300).astype(np.float32),
                           cell=M[None].astype(np.float32))
    check(run(pg, wl), wl, "f32")


def weighted(wl, seed=3, lo=0.5, hi=1.5):
    wl.batch.weight = np.random.default_rng(seed).uniform(lo, hi, wl.batch.n_atoms).astype(
        np.float32)
    return wl


@pytest.mark.parametrize("form", ["point", "integral"])
def test_weighted_direct_path(pg, form):
    wl = weighted(synth.qm9_shaped(n_mol=24))
    wl.form = form
    check(run(pg, wl), wl, "f32")
    # Large molecules take the staged path (and, unweighted, scatter mode).
    wl = weighted(synth.crystal_shaped(n_cells=3, grid=24))
    wl.form = form
    check(run(pg, wl, "f16"), wl, "f16")


@pytest.mark.parametrize("simple", [0, 1])
@pytest.mark.parametrize("form", ["point", "integral"])
def test_weighted_separable_path(pg, simple, form):
    wl = weighted(synth.precision_form(n_mol=6))
    wl.form = form
    wl.cutoff = "box"
    G = pg.voxelize_tuned(pg.DeviceBatch.from_numpy(wl.batch), pg.Grid.from_workload(wl),
                          {"path": 2, "n_tile": 128, "separable_simple": simple}, dtype="f16")
    assert pg.sync_status() == 0
    check(G, wl, "f16", tol=SEPARABLE_TOL)


def test_weighted_packed_tiles(pg):
    wl = weighted(synth.pipeline_single_channel(n_mol=40))
    check(run(pg, wl, "bf16", path="separable"), wl, "bf16", tol=SEPARABLE_TOL)


@pytest.mark.parametrize("path", ["direct", "separable"])
def test_unit_weights_change_no_bit(pg, path):
    wl = synth.precision_form(n_mol=4)
    wl.cutoff = "box"
    G0 = run(pg, wl, "f16", path)
    wl.batch.weight = np.ones(wl.batch.n_atoms, np.float32)
    assert torch.equal(G0, run(pg, wl, "f16", path))


def test_signed_weights(pg):
    wl = weighted(synth.plain_small(n_mol=6), lo=-2.0, hi=2.0)
    wl.cutoff = "none"
    G = run(pg, wl).cpu().numpy().astype(np.float64)
    ref = oracle.voxelize(oracle.Problem.from_workload(wl))
    for b in range(wl.batch.n_mol):
        assert np.max(np.abs(G[b] - ref[b])) <= TOL["f32"] * np.abs(ref[b]).max()


def gradients(pg, wl, W):
    db = pg.DeviceBatch.from_numpy(wl.batch)
    gc, gw = pg.voxelize_backward_weights(db, pg.Grid.from_workload(wl),
                                          torch.as_tensor(W, device="cuda"))
    assert pg.sync_status() == 0
    return gc, gw


@pytest.mark.parametrize("kind", ["triclinic", "qm9", "integral"])
def test_coordinate_and_weight_gradients_match_oracle(pg, kind):
    if kind == "triclinic":
        wl = triclinic(n_cells=3, shape=(20, 20, 24))
    else:
        wl = weighted(synth.qm9_shaped(n_mol=16), lo=-1.0, hi=2.0)
        wl.form = "point" if kind == "qm9" else "integral"
    prob = oracle.Problem.from_workload(wl)
    W = np.random.default_rng(11).standard_normal(prob.shape).astype(np.float32)
    gc, gw = gradients(pg, wl, W)
    grad_check(gc.cpu().numpy(), oracle.gradient(prob, W.astype(np.float64)),
               wl.batch.mol_off)
    ref_w = oracle.gradient_weight(prob, W.astype(np.float64))
    for b in range(wl.batch.n_mol):
        s = wl.batch.atoms_of(b)
        m = np.abs(ref_w[s]).max()
        assert np.max(np.abs(gw.cpu().numpy()[s] - ref_w[s])) <= GRAD_TOL * m
    # Deterministic: the same bits on a second run.
    gc2, gw2 = gradients(pg, wl, W)
    assert torch.equal(gc, gc2) and torch.equal(gw, gw2)


def test_plan_runs_take_weights_and_cells(pg):
    wl = triclinic(n_cells=5)
    b = wl.batch
    grid = pg.Grid.from_workload(wl)
    plan = pg.Plan(grid, "f16", max_mol=8, max_atoms=int(b.n_atoms) + 64)
    try:
        for n in (5, 2, 5):
            sub = b.subset(range(n))
            out = torch.empty(grid.out_shape(n), dtype=torch.float16, device="cuda")
            plan.run(sub.coords, sub.elem, sub.mol_off, sub.origin, None, out=out,
                     weight=sub.weight, cell=sub.cell)
            assert torch.equal(out, run(pg, wl, "f16", batch=sub)), n
        # The same plan then takes an axis-aligned unweighted batch.
        q = synth.qm9_shaped(n_mol=8)
        for attr in ("nx", "ny", "nz", "n_channels", "sigma", "cutoff", "cutoff_k", "periodic",
                     "form"):
            setattr(q, attr, getattr(wl, attr))
        out = torch.empty(grid.out_shape(8), dtype=torch.float16, device="cuda")
        plan.run(q.batch.coords, q.batch.elem, q.batch.mol_off, q.batch.origin, q.batch.spacing,
                 out=out)
        assert torch.equal(out, run(pg, q, "f16"))
    finally:
        plan.close()


def test_no_alloc_entry_takes_cells(pg):
    from paper_2211_08506_gb300 import binding as B
    wl = triclinic(n_cells=3)
    db = pg.DeviceBatch.from_numpy(wl.batch)
    grid = pg.Grid.from_workload(wl)
    out = torch.empty(grid.out_shape(3), dtype=torch.float32, device="cuda")
    st, bits = B.pg_voxelize_noalloc(db.to_c(), grid.to_c(), pg.DTYPES["f32"][0],
                                     out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == 0 and bits == 0
    assert torch.equal(out, run(pg, wl))


def test_autotune_with_cells(pg):
    wl = triclinic(n_cells=8)
    db = pg.DeviceBatch.from_numpy(wl.batch)
    grid = pg.Grid.from_workload(wl)
    t = pg.autotune(db, grid, dtype="f16")
    assert t["path"] == 1
    assert torch.equal(pg.voxelize(db, grid, dtype="f16"), run(pg, wl, "f16"))


def test_refinement_in_triclinic_cells(pg):
    wl = triclinic(n_cells=3, shape=(24, 24, 24))
    wl.batch.weight = None
    truth = oracle.Problem.from_workload(wl)
    T = oracle.voxelize(truth).astype(np.float32)
    start = (wl.batch.coords + np.random.default_rng(4).normal(0, 0.05, wl.batch.coords.shape)
             ).astype(np.float32)
    db = pg.DeviceBatch.from_numpy(wl.batch)
    x = torch.as_tensor(start, device="cuda").clone()
    loss, steps = pg.refine(db, pg.Grid.from_workload(wl), torch.as_tensor(T, device="cuda"), x,
                            60, 0.01)
    assert pg.sync_status() == 0
    xr, Lr, sr = oracle.refine(oracle.Problem.from_workload(wl, coords=start.astype(np.float64)),
                               T.astype(np.float64), 60, 0.01)
    assert np.array_equal(steps.cpu().numpy(), sr)
    assert np.max(np.abs(x.cpu().numpy() - xr)) < 1e-3
    assert np.all(loss.cpu().numpy() <= Lr * 1.01 + 1e-3)


def test_device_errors_for_bad_cells(pg):
    wl = triclinic(n_cells=2)
    b = wl.batch
    grid = pg.Grid.from_workload(wl)
    singular = b.cell.copy()
    singular[1] = 0.0
    b.cell = singular
    G = pg.voxelize(pg.DeviceBatch.from_numpy(b), grid, dtype="f32")
    bits = pg.sync_status(raise_on_error=False)
    assert bits & 0x4
    assert float(G[1].abs().max()) == 0.0
    # A cell thinner than twice the cutoff along one axis is flagged.
    wl2 = triclinic(n_cells=2)
    wl2.cutoff_k = 8.0
    pg.voxelize(pg.DeviceBatch.from_numpy(wl2.batch), pg.Grid.from_workload(wl2), dtype="f32")
    assert pg.sync_status(raise_on_error=False) & 0x8
    assert pg.sync_status() == 0


def test_full_size_triclinic_batch_sampled(pg):
    wl = synth.crystal_triclinic()
    db = pg.DeviceBatch.from_numpy(wl.batch)
    grid = pg.Grid.from_workload(wl)
    G = pg.voxelize(db, grid, dtype="f16")
    assert pg.sync_status() == 0
    idx = [0, 211, wl.batch.n_mol - 1]
    sub = wl.batch.subset(idx)
    grid_check(G[idx].float().cpu().numpy(), oracle.Problem.from_workload(wl, batch=sub),
               TOL["f16"], abs_tol=ABS_TOL["f16"])


@pytest.mark.parametrize("kind", ["molecules", "triclinic"])
def test_autograd_through_learnable_weights(pg, kind):
    # L = <W, G(x, w)>: autograd returns dL/dx and dL/dw from the adjoint kernel, equal to the
    # oracle's gradient and weight gradient.
    if kind == "molecules":
        wl = weighted(synth.qm9_shaped(n_mol=8), lo=-1.0, hi=2.0)
    else:
        wl = triclinic(n_cells=2, shape=(20, 20, 24))
    db = pg.DeviceBatch.from_numpy(wl.batch)
    grid = pg.Grid.from_workload(wl)
    x = db.coords.clone().requires_grad_(True)
    w = torch.as_tensor(wl.batch.weight, device="cuda").clone().requires_grad_(True)
    prob = oracle.Problem.from_workload(wl)
    W = np.random.default_rng(21).standard_normal(prob.shape).astype(np.float32)
    G = pg.voxelize_autograd(x, db, grid, dtype="f32", path="direct", weight=w)
    (torch.as_tensor(W, device="cuda") * G).sum().backward()
    assert pg.sync_status() == 0
    grad_check(x.grad.cpu().numpy(), oracle.gradient(prob, W.astype(np.float64)),
               wl.batch.mol_off)
    ref_w = oracle.gradient_weight(prob, W.astype(np.float64))
    assert np.max(np.abs(w.grad.cpu().numpy() - ref_w)) <= GRAD_TOL * np.abs(ref_w).max()


def test_empty_cell_and_atoms_lattice_vectors_away(pg):
    # A cell with no atoms writes zeros; atoms moved by whole lattice vectors (several cells
    # away from the grid) give the same periodic grid.
    wl = triclinic(n_cells=3, shape=(20, 24, 16))
    b = wl.batch
    keep = [0, 2]
    atoms = np.concatenate([np.arange(b.mol_off[m], b.mol_off[m + 1]) for m in keep])
    off = np.array([0, b.mol_off[1] - b.mol_off[0], b.mol_off[1] - b.mol_off[0],
                    len(atoms)], np.int32)
    shift = np.zeros((len(atoms), 3), np.float64)
    n0 = int(off[1])
    shift[n0:] = np.array([2.0, -3.0, 1.0]) @ b.cell[2].astype(np.float64)
    wl.batch = synth.Batch(coords=(b.coords[atoms] + shift).astype(np.float32),
                           elem=b.elem[atoms], mol_off=off, origin=b.origin, spacing=b.spacing,
                           weight=b.weight[atoms], cell=b.cell)
    G = run(pg, wl)
    assert float(G[1].abs().max()) == 0.0
    check(G, wl, "f32")
    wl.batch.coords = (b.coords[atoms]).astype(np.float32)
    G0 = run(pg, wl)
    assert float((G - G0).abs().max()) <= 2 * TOL["f32"] * float(G0.abs().max())


@pytest.mark.parametrize("cutoff,periodic", [("sphere", True), ("box", True), ("sphere", False)])
@pytest.mark.parametrize("shape", [(17, 21, 40), (12, 19, 32)])
def test_two_row_passes_equal_row_groups_bitwise(pg, cutoff, periodic, shape):
    # FP32 with 16-byte stores walks each plane in two-row passes (nz = 40: 10 lanes per row,
    # 3 rows per lane group; nz = 32: 8 lanes, 4 rows).  An output that is not 16-byte
    # aligned takes scalar stores: nz = 40 then walks row groups of 32 voxels, nz = 32
    # two-row passes of one row per lane group.  All add the same terms in the same order:
    # identical bits, including the partial last pass of an odd row count, and they match the
    # oracle.
    wl = triclinic(n_cells=5, shape=shape)
    wl.cutoff, wl.periodic = cutoff, periodic
    db = pg.DeviceBatch.from_numpy(wl.batch)
    grid = pg.Grid.from_workload(wl)
    passes = pg.voxelize(db, grid, dtype="f32", path="direct")
    assert pg.sync_status() == 0
    buf = torch.zeros(passes.numel() + 1, dtype=torch.float32, device="cuda")
    groups = buf[1:].view(passes.shape)
    pg.voxelize(db, grid, dtype="f32", path="direct", out=groups)
    assert pg.sync_status() == 0
    assert torch.equal(passes, groups)
    check(passes[:3], wl, "f32", batch=wl.batch.subset(range(3)))
