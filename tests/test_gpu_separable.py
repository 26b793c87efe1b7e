"""GPU parity of the separable tcgen05 path (BF16 operands, FP32 tensor-memory
accumulation) against the FP64 oracle, through the C ABI.

The separable form is exact for the no-cutoff and box-cutoff indicators (Sec. III-A after
Eq. 5, Sec. VI-A); its only error is the BF16 rounding of the two operands (at most
2 x 2^-9 relative per term, every term positive) plus the store rounding, so the bar is
1e-2 of each grid's maximum.  Also checked: the oracle's own separable restatement,
agreement with the FP32 direct path, K chunking past 32 atoms, partial M and N tiles,
every tile width, determinism and the unsupported cases.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.parity import ABS_TOL, SEPARABLE_TOL, grid_check

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


def sep(pg, wl, dtype="f16", batch=None, n_tile=None, simple=0):
    batch = wl.batch if batch is None else batch
    db = pg.DeviceBatch.from_numpy(batch)
    grid = pg.Grid.from_workload(wl)
    if n_tile is None and not simple:
        G = pg.voxelize(db, grid, dtype=dtype, path="separable")
    else:
        G = pg.voxelize_tuned(db, grid, {"path": 2, "n_tile": n_tile or 128,
                                         "separable_simple": simple}, dtype=dtype)
    assert pg.sync_status() == 0
    return G.float().cpu().numpy()


def small(cutoff="none", periodic=False, n_mol=3, shape=(32, 32, 32)):
    wl = synth.plain_small(n_mol=n_mol)
    wl.cutoff, wl.periodic = cutoff, periodic
    wl.nx, wl.ny, wl.nz = shape
    wl.sigma = np.array([0.4, 0.5, 0.6, 0.55, 0.45], np.float32)
    if cutoff == "box" and periodic:
        wl.cutoff_k = 2.5
    return wl


def test_single_molecule_no_cutoff_f16(pg):
    wl = small(n_mol=1)
    stats = grid_check(sep(pg, wl), oracle.Problem.from_workload(wl), SEPARABLE_TOL,
                       abs_tol=ABS_TOL["f16"])
    assert stats["max_abs_rel"] < 5e-3


@pytest.mark.parametrize("dtype", ["f16", "bf16", "f32"])
@pytest.mark.parametrize("cutoff,periodic", [("none", False), ("box", False), ("none", True),
                                             ("box", True)])
def test_separable_matches_oracle(pg, dtype, cutoff, periodic):
    wl = small(cutoff, periodic, n_mol=4)
    prob = oracle.Problem.from_workload(wl)
    G = sep(pg, wl, dtype)
    grid_check(G, prob, SEPARABLE_TOL, abs_tol=ABS_TOL[dtype])
    # The oracle's separable restatement agrees with its direct form (pinned on the CPU);
    # the GPU result sits within the same bar of it.
    ref = oracle.separable(prob)
    for b in range(prob.shape[0]):
        m = np.abs(ref[b]).max()
        assert np.abs(G[b] - ref[b]).max() <= SEPARABLE_TOL * m + ABS_TOL[dtype]


@pytest.mark.parametrize("shape", [(20, 12, 20), (7, 16, 3), (33, 8, 8), (64, 16, 24)])
def test_partial_tiles(pg, shape):
    # M = C*nx not a multiple of 128 and N = ny*nz not a multiple of the tile width.
    wl = small("none", False, n_mol=3, shape=shape)
    grid_check(sep(pg, wl), oracle.Problem.from_workload(wl), SEPARABLE_TOL,
               abs_tol=ABS_TOL["f16"])


@pytest.mark.parametrize("simple", [0, 1])
@pytest.mark.parametrize("n_tile", [64, 128, 256])
def test_every_tile_width_and_variant(pg, n_tile, simple):
    wl = small("box", False, n_mol=3)
    grid_check(sep(pg, wl, n_tile=n_tile, simple=simple), oracle.Problem.from_workload(wl),
               SEPARABLE_TOL, abs_tol=ABS_TOL["f16"])


def test_pipelined_and_single_stage_agree_bitwise(pg):
    # Same BF16 operands, same accumulation order: identical bits from both kernels, also
    # with K chunks past 32 atoms and partial tiles.
    rng = np.random.default_rng(23)
    pos = [8.0 + rng.uniform(-4, 4, (n, 3)) for n in (3, 40, 29, 70)]
    el = [rng.integers(0, 5, n) for n in (3, 40, 29, 70)]
    nb = synth._pack(pos, el, np.zeros((4, 3)), np.full((4, 3), 0.5))
    for shape in ((32, 32, 32), (20, 12, 20)):
        wl = small("none", False, shape=shape)
        a = sep(pg, wl, batch=nb, n_tile=128, simple=0)
        b = sep(pg, wl, batch=nb, n_tile=128, simple=1)
        assert np.array_equal(a, b)


def test_more_than_32_atoms_accumulates_k_chunks(pg):
    rng = np.random.default_rng(21)
    pos = [8.0 + rng.uniform(-4, 4, (n, 3)) for n in (33, 70, 5, 100)]
    el = [rng.integers(0, 5, n) for n in (33, 70, 5, 100)]
    nb = synth._pack(pos, el, np.zeros((4, 3)), np.full((4, 3), 0.5))
    wl = small("none", False)
    grid_check(sep(pg, wl, batch=nb), oracle.Problem.from_workload(wl, batch=nb), SEPARABLE_TOL,
               abs_tol=ABS_TOL["f16"])


def test_empty_molecules_and_determinism(pg):
    wl = small("none", False, n_mol=3)
    b = wl.batch
    nb = synth._pack([b.coords[b.atoms_of(0)], np.zeros((0, 3)), b.coords[b.atoms_of(2)]],
                     [b.elem[b.atoms_of(0)], np.zeros(0), b.elem[b.atoms_of(2)]],
                     b.origin, b.spacing)
    G1 = sep(pg, wl, batch=nb)
    assert np.all(G1[1] == 0.0)
    grid_check(G1, oracle.Problem.from_workload(wl, batch=nb), SEPARABLE_TOL,
               abs_tol=ABS_TOL["f16"])
    assert np.array_equal(sep(pg, wl, batch=nb), G1)


def test_agrees_with_direct_fp32(pg):
    wl = small("none", False, n_mol=6)
    db = pg.DeviceBatch.from_numpy(wl.batch)
    grid = pg.Grid.from_workload(wl)
    d = pg.voxelize(db, grid, dtype="f32", path="direct").cpu().numpy()
    s = sep(pg, wl, "f32")
    for b in range(wl.batch.n_mol):
        assert np.abs(s[b] - d[b]).max() <= SEPARABLE_TOL * np.abs(d[b]).max()


def test_unsupported_cases_are_rejected(pg):
    wl = small("sphere", False, n_mol=2)
    with pytest.raises(Exception, match="UNSUPPORTED"):
        sep(pg, wl)
    wl = small("none", False, n_mol=2, shape=(8, 5, 3))  # N = 15, not a multiple of 16
    with pytest.raises(Exception, match="UNSUPPORTED"):
        sep(pg, wl)


def test_precision_form_full_batch_sampled(pg):
    wl = synth.precision_form()
    db = pg.DeviceBatch.from_numpy(wl.batch)
    grid = pg.Grid.from_workload(wl)
    G = pg.voxelize(db, grid, dtype="f16", path="separable")
    assert pg.sync_status() == 0
    idx = np.sort(np.random.default_rng(22).choice(wl.batch.n_mol, 6, replace=False))
    sub = G[torch.as_tensor(idx, device="cuda")].float().cpu().numpy()
    stats = grid_check(sub, oracle.Problem.from_workload(wl, batch=wl.batch.subset(idx)),
                       SEPARABLE_TOL, abs_tol=ABS_TOL["f16"])
    assert stats["max_abs_rel"] < SEPARABLE_TOL


@pytest.mark.parametrize("C,nx,ny,nz,n_mol,cutoff,periodic,form,dtype", [
    (1, 32, 32, 32, 9, "none", False, "point", "f16"),      # 4 molecules per tile, ragged end
    (2, 16, 24, 32, 7, "box", False, "point", "bf16"),      # 4 per tile
    (2, 32, 16, 16, 5, "box", True, "point", "f32"),        # 2 per tile, periodic
    (1, 32, 32, 32, 6, "box", False, "integral", "bf16"),   # erf tables per atom's molecule
    (4, 8, 16, 16, 33, "none", False, "integral", "f16"),   # 4 per tile, 9 tiles
])
def test_packed_tiles_match_oracle(pg, C, nx, ny, nz, n_mol, cutoff, periodic, form, dtype):
    # Molecules whose C * nx rows divide the 128-row tile share one tile: their atoms form
    # one K range, each atom carries its own molecule's grid geometry, and the rows go out as
    # global rows.  Every molecule gets its own spacing so a mix-up between molecules shows.
    wl = synth.plain_small(n_mol=n_mol)
    wl.n_channels = C
    wl.sigma = np.array([0.45, 0.55, 0.5, 0.6][:C], np.float32)
    wl.batch.elem = (wl.batch.elem % C).astype(np.int32)
    wl.cutoff, wl.periodic, wl.form = cutoff, periodic, form
    wl.nx, wl.ny, wl.nz = nx, ny, nz
    if periodic:
        wl.cutoff_k = 2.5
    h = 0.4 + 0.05 * np.arange(n_mol, dtype=np.float32)
    wl.batch.spacing = np.stack([h, h * 1.1, h * 0.9], axis=1).astype(np.float32)
    G = sep(pg, wl, dtype=dtype)
    grid_check(G, oracle.Problem.from_workload(wl), SEPARABLE_TOL, abs_tol=ABS_TOL[dtype])


def test_packed_tiles_with_uneven_atom_counts(pg):
    # Four molecules per tile; one tile holds far more atoms than the average, so its K
    # chunks exceed the resident table slots and take the rebuild-per-step fallback, while
    # the others keep their chunk tables resident.  Both must match the oracle.
    rng = np.random.default_rng(31)
    sizes = [3, 6, 4, 5, 150, 8, 2, 90, 7, 5, 4, 6]
    pos = [8.0 + rng.uniform(-3, 3, (n, 3)) for n in sizes]
    el = [np.zeros(n, np.int64) for n in sizes]
    nb = synth._pack(pos, el, np.zeros((len(sizes), 3)),
                     np.full((len(sizes), 3), 0.5))
    wl = small("none", False, n_mol=len(sizes), shape=(32, 32, 32))
    wl.n_channels = 1
    wl.sigma = np.array([0.5], np.float32)
    for form in ("point", "integral"):
        wl.form = form
        G = sep(pg, wl, batch=nb, dtype="f16")
        grid_check(G, oracle.Problem.from_workload(wl, batch=nb), SEPARABLE_TOL,
                   abs_tol=ABS_TOL["f16"])



@pytest.mark.parametrize("simple", [0, 1])
@pytest.mark.parametrize("packed", [False, True])
def test_bounded_waits_give_up_without_faulting_then_recover(pg, monkeypatch, simple, packed):
    # Failure detection without a GPU fault: PG_DEBUG_STALL_PRODUCERS=1 stops the operand
    # producers (the single-stage kernel: its MMA issue) before the first handoff and shortens
    # every wait to 2 ms.  No MMA is issued and no store starts; each CTA's bounded waits give
    # up, it confirms through the drain barrier that no MMA is outstanding, frees its tensor
    # memory and returns.  The host reads PG_ERR_TIMEOUT with the timeout bit (and not the bit
    # for kept tensor memory); the next normal call on the same device matches the oracle.
    from paper_2211_08506_gb300 import binding as B

    wl = small("box", n_mol=9, shape=(32, 32, 32) if not packed else (16, 16, 32))
    if packed:
        wl.n_channels, wl.sigma = 1, np.array([0.5], np.float32)
        wl.batch.elem[:] = 0
    db = pg.DeviceBatch.from_numpy(wl.batch)
    grid = pg.Grid.from_workload(wl)
    tuning = {"path": 2, "separable_simple": simple}
    out = torch.full(grid.out_shape(wl.batch.n_mol), 7.0, dtype=torch.float16, device="cuda")
    monkeypatch.setenv("PG_DEBUG_STALL_PRODUCERS", "1")
    pg.voxelize_tuned(db, grid, tuning, dtype="f16", out=out)
    st, bits = B.pg_sync_status(torch.cuda.current_stream().cuda_stream)
    assert st == B.PG_ERR_TIMEOUT, B.last_error()
    assert bits & B.PG_DEVERR_TIMEOUT and not bits & B.PG_DEVERR_TMEM_HELD
    if not simple:
        assert torch.all(out == 7.0)  # no store started
    monkeypatch.delenv("PG_DEBUG_STALL_PRODUCERS")
    pg.voxelize_tuned(db, grid, tuning, dtype="f16", out=out)
    assert pg.sync_status() == 0
    grid_check(out.float().cpu().numpy(), oracle.Problem.from_workload(wl), SEPARABLE_TOL,
               abs_tol=ABS_TOL["f16"])
