"""GPU parity of the forward voxelization against the FP64 oracle, through the C ABI.

Covers the direct kernel in every dtype, cutoff and boundary mode, ragged shapes (scalar
store path), empty molecules and batches, atoms outside the grid, the unstaged fallback
(more than 128 candidates per item), full-size sampled parity on the QM9-shaped and
crystal-shaped batches in the launch configuration the benchmark uses, bitwise
determinism across runs and launch shapes, canary bounds checks and device validation.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.parity import ABS_TOL, TOL, grid_check

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CUTOFF_CASES = [("sphere", False), ("box", False), ("none", False), ("sphere", True),
                ("box", True), ("none", True)]


@pytest.fixture(scope="module")
def pg():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2211_08506_gb300 as pkg
    pkg.build()
    from paper_2211_08506_gb300 import api
    return api


def run(pg, wl, dtype=None, path="direct", batch=None, grid=None, tuning=None):
    batch = wl.batch if batch is None else batch
    db = pg.DeviceBatch.from_numpy(batch)
    grid = pg.Grid.from_workload(wl) if grid is None else grid
    if tuning is not None:
        G = pg.voxelize_tuned(db, grid, tuning, dtype=dtype or wl.out_dtype)
    else:
        G = pg.voxelize(db, grid, dtype=dtype or wl.out_dtype, path=path)
    assert pg.sync_status() == 0
    return G.float().cpu().numpy()


def test_plain_small_f32_matches_oracle(pg):
    wl = synth.plain_small()
    G = run(pg, wl)
    stats = grid_check(G, oracle.Problem.from_workload(wl), TOL["f32"],
               abs_tol=ABS_TOL["f32"])
    assert stats["max_abs_rel"] < 1e-5


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("cutoff,periodic", CUTOFF_CASES)
def test_dtypes_cutoffs_and_boundaries(pg, dtype, cutoff, periodic):
    wl = synth.plain_small(n_mol=6)
    wl.cutoff, wl.periodic = cutoff, periodic
    wl.sigma = np.array([0.4, 0.5, 0.6, 0.55, 0.45], np.float32)
    if periodic:
        wl.cutoff_k = 2.5  # r_c = 1.5 A < L/2 = 8 A
    G = run(pg, wl, dtype=dtype)
    grid_check(G, oracle.Problem.from_workload(wl), TOL[dtype],
               abs_tol=ABS_TOL[dtype])


@pytest.mark.parametrize("shape,dtype", [((17, 19, 23), "f32"), ((9, 5, 31), "f16"),
                                          ((20, 24, 36), "f32"), ((12, 10, 40), "bf16"),
                                          ((3, 3, 8), "f16"), ((1, 1, 1), "f32"),
                                          ((40, 7, 4), "f32"), ((16, 16, 64), "f16")])
def test_ragged_and_odd_shapes(pg, shape, dtype):
    wl = synth.plain_small(n_mol=5)
    wl.nx, wl.ny, wl.nz = shape
    b = wl.batch
    b.spacing = np.tile(np.array([0.55, 0.45, 0.6], np.float32), (b.n_mol, 1))
    G = run(pg, wl, dtype=dtype)
    grid_check(G, oracle.Problem.from_workload(wl), TOL[dtype],
               abs_tol=ABS_TOL[dtype])


def test_empty_molecules_atoms_outside_and_empty_batch(pg):
    wl = synth.plain_small(n_mol=4)
    b = wl.batch
    # Molecule 1 empty, molecule 3 shifted mostly outside its box.
    coords = [b.coords[b.atoms_of(0)], np.zeros((0, 3), np.float32), b.coords[b.atoms_of(2)],
              b.coords[b.atoms_of(3)] + np.float32(7.0)]
    elems = [b.elem[b.atoms_of(0)], np.zeros(0, np.int32), b.elem[b.atoms_of(2)],
             b.elem[b.atoms_of(3)]]
    nb = synth._pack(coords, elems, b.origin, b.spacing)
    G = run(pg, wl, batch=nb)
    grid_check(G, oracle.Problem.from_workload(wl, batch=nb), TOL["f32"],
               abs_tol=ABS_TOL["f32"])
    assert np.all(G[1] == 0.0)
    # No molecules at all, and molecules without atoms.
    empty = synth._pack([], [], np.zeros((0, 3)), np.zeros((0, 3)))
    assert run(pg, wl, batch=empty).shape == (0, 5, 32, 32, 32)
    hollow = synth._pack([np.zeros((0, 3))] * 3, [np.zeros(0)] * 3, b.origin[:3], b.spacing[:3])
    assert np.all(run(pg, wl, batch=hollow) == 0.0)


def test_dense_items_take_unstaged_fallback_bitwise(pg):
    # 400 atoms of one channel inside a 3 A cube: far more than 128 candidates per plane.
    rng = np.random.default_rng(11)
    pos = 8.0 + rng.uniform(-1.5, 1.5, (400, 3))
    el = np.where(rng.uniform(size=400) < 0.9, 1, 0)
    nb = synth._pack([pos, pos[:20]], [el, el[:20]], np.zeros((2, 3)), np.full((2, 3), 0.5))
    wl = synth.plain_small(n_mol=1)
    for dtype in ("f32", "f16"):
        G = run(pg, wl, batch=nb, dtype=dtype)
        grid_check(G, oracle.Problem.from_workload(wl, batch=nb), TOL[dtype],
               abs_tol=ABS_TOL[dtype])


def test_deterministic_across_runs_and_launch_shapes(pg):
    wl = synth.qm9_shaped(n_mol=64)
    ref = run(pg, wl)
    assert np.array_equal(run(pg, wl), ref)
    for threads in (128, 256, 512):
        for bps in (1, 2, 0):
            for hint in (0, 1):
                t = {"path": 1, "block_threads": threads, "blocks_per_sm": bps,
                     "store_hint": hint}
                G = run(pg, wl, tuning=t)
                assert np.array_equal(G.view(np.uint32), ref.view(np.uint32)), t
    for cp in (1, 3, 8, 64):
        G = run(pg, wl, tuning={"path": 1, "chunk_planes": cp})
        assert np.array_equal(G.view(np.uint32), ref.view(np.uint32)), cp


def test_outputs_stay_in_bounds(pg):
    wl = synth.plain_small(n_mol=3)
    for dtype, (nx, ny, nz) in (("f32", (32, 32, 32)), ("f16", (7, 9, 11)), ("bf16", (8, 8, 24))):
        wl.nx, wl.ny, wl.nz = nx, ny, nz
        grid = pg.Grid.from_workload(wl)
        tdt = pg.DTYPES[dtype][1]
        n = wl.batch.n_mol * 5 * nx * ny * nz
        pad = 4096
        buf = torch.full((n + 2 * pad,), 7.0, dtype=tdt, device="cuda")
        out = buf[pad:pad + n].view(wl.batch.n_mol, 5, nx, ny, nz)
        db = pg.DeviceBatch.from_numpy(wl.batch)
        pg.voxelize(db, grid, dtype=dtype, path="direct", out=out)
        pg.sync_status()
        assert torch.all(buf[:pad] == 7.0) and torch.all(buf[pad + n:] == 7.0)
        grid_check(out.float().cpu().numpy(), oracle.Problem.from_workload(wl), TOL[dtype],
               abs_tol=ABS_TOL[dtype])


def test_misaligned_output_uses_scalar_stores(pg):
    wl = synth.plain_small(n_mol=2)
    grid = pg.Grid.from_workload(wl)
    n = 2 * 5 * 32 ** 3
    buf = torch.zeros(n + 1, dtype=torch.float32, device="cuda")
    out = buf[1:].view(2, 5, 32, 32, 32)  # 4-byte but not 16-byte aligned
    pg.voxelize(pg.DeviceBatch.from_numpy(wl.batch), grid, dtype="f32", path="direct", out=out)
    pg.sync_status()
    grid_check(out.cpu().numpy(), oracle.Problem.from_workload(wl), TOL["f32"],
               abs_tol=ABS_TOL["f32"])


def test_device_validation_flags_without_faulting(pg):
    wl = synth.plain_small(n_mol=3)
    b = wl.batch
    bad = synth.Batch(b.coords.copy(), b.elem.copy(), b.mol_off.copy(), b.origin.copy(),
                      b.spacing.copy())
    bad.elem[2] = 9  # channel outside [0, 5)
    db = pg.DeviceBatch.from_numpy(bad)
    G = pg.voxelize(db, pg.Grid.from_workload(wl), path="direct")
    bits = pg.sync_status(raise_on_error=False)
    assert bits & 0x1
    assert pg.sync_status() == 0  # cleared
    # The bad atom is skipped; the rest matches the oracle without it.
    keep = np.ones(b.n_atoms, bool)
    keep[2] = False
    ok = synth.Batch(b.coords[keep], b.elem[keep], b.mol_off.copy(), b.origin, b.spacing)
    ok.mol_off[1:] -= 1
    grid_check(G.cpu().numpy(), oracle.Problem.from_workload(wl, batch=ok), TOL["f32"],
               abs_tol=ABS_TOL["f32"])
    # Offsets past n_atoms and non-positive spacing: flagged, zeros written, no fault.
    bad2 = synth.Batch(b.coords.copy(), b.elem.copy(), b.mol_off.copy(), b.origin.copy(),
                       b.spacing.copy())
    bad2.mol_off[2] = b.n_atoms + 50
    bad2.spacing[0, 1] = -0.5
    G2 = pg.voxelize(pg.DeviceBatch.from_numpy(bad2), pg.Grid.from_workload(wl), path="direct")
    bits = pg.sync_status(raise_on_error=False)
    assert bits & 0x2 and bits & 0x4
    assert torch.all(G2[0] == 0) and torch.all(G2[1] == 0)
    with pytest.raises(Exception):
        pg.voxelize(pg.DeviceBatch.from_numpy(bad2), pg.Grid.from_workload(wl), path="direct")
        pg.sync_status()


def test_separable_rejects_sphere_cutoff(pg):
    wl = synth.plain_small(n_mol=2)
    with pytest.raises(Exception, match="UNSUPPORTED"):
        pg.voxelize(pg.DeviceBatch.from_numpy(wl.batch), pg.Grid.from_workload(wl),
                    path="separable")


def _sampled(pg, wl, dtype, n_sample, seed, path="auto", tune=True):
    db = pg.DeviceBatch.from_numpy(wl.batch)
    grid = pg.Grid.from_workload(wl)
    if tune:
        pg.autotune(db, grid, dtype=dtype, path=path)
    G = pg.voxelize(db, grid, dtype=dtype, path=path)
    assert pg.sync_status() == 0
    idx = np.sort(np.random.default_rng(seed).choice(wl.batch.n_mol, n_sample, replace=False))
    sub = G[torch.as_tensor(idx, device="cuda")].float().cpu().numpy()
    return grid_check(sub, oracle.Problem.from_workload(wl, batch=wl.batch.subset(idx)),
                      TOL[dtype], abs_tol=ABS_TOL[dtype])


def test_qm9_shaped_full_batch_sampled_parity(pg):
    wl = synth.qm9_shaped()
    stats = _sampled(pg, wl, "f32", 24, 12)
    assert stats["max_abs_rel"] < 1e-5


def test_qm9_shaped_full_batch_f16_sampled_parity(pg):
    wl = synth.qm9_shaped()
    _sampled(pg, wl, "f16", 16, 13, path="direct")


def test_crystal_shaped_sampled_parity(pg):
    wl = synth.crystal_shaped(n_cells=96)
    _sampled(pg, wl, "f16", 12, 14)


def test_register_and_staged_paths_agree_bitwise(pg):
    # The same molecule voxelized through the <=32-atom register path and, padded with far
    # atoms to 40 atoms, through the staged path: identical bits on every voxel.
    wl = synth.qm9_shaped(n_mol=32)
    b = wl.batch
    coords, elems = [], []
    for i in range(b.n_mol):
        s = b.atoms_of(i)
        far = np.full((40 - (s.stop - s.start), 3), 1.0e4, np.float32)
        coords.append(np.concatenate([b.coords[s], far]))
        elems.append(np.concatenate([b.elem[s], np.full(far.shape[0], 2, np.int32)]))
    padded = synth._pack(coords, elems, b.origin, b.spacing)
    for dtype in ("f32", "f16"):
        G1 = run(pg, wl, dtype=dtype)
        G2 = run(pg, wl, dtype=dtype, batch=padded, tuning={"path": 1, "gather_only": 1})
        assert np.array_equal(G1, G2)
        # With lane-list mode allowed, each lane of a staged plane adds only the candidates
        # that reach its own voxels: the same terms in the same order, identical bits.
        G3 = run(pg, wl, dtype=dtype, batch=padded, tuning={"path": 1})
        assert np.array_equal(G3, G1)


@pytest.mark.parametrize("cutoff,periodic,shape", [
    ("sphere", False, (48, 48, 48)), ("box", False, (48, 48, 48)), ("box", True, (48, 48, 48)),
    ("sphere", True, (40, 44, 45)), ("box", False, (37, 52, 30))])
def test_lane_list_mode_every_cutoff_boundary_and_ragged_plane(pg, cutoff, periodic, shape):
    # Lane-list mode against the gather mode on dense cells, for both cutoffs, open and
    # periodic boundaries, and ragged planes that take the scalar store path (one column per
    # lane).  The two modes add the same terms in the same order: identical bits, and both
    # match the oracle.
    wl = synth.crystal_shaped(n_cells=10)
    wl.cutoff, wl.periodic = cutoff, periodic
    wl.nx, wl.ny, wl.nz = shape
    prob = oracle.Problem.from_workload(wl, batch=wl.batch.subset(range(4)))
    for dtype in ("f32", "bf16"):
        auto = run(pg, wl, dtype=dtype, tuning={"path": 1, "block_threads": 256})
        gather = run(pg, wl, dtype=dtype,
                     tuning={"path": 1, "block_threads": 256, "gather_only": 1})
        assert np.array_equal(auto.view(np.uint32), gather.view(np.uint32))
        for G in (auto, gather):
            grid_check(G[:4], prob, TOL[dtype], abs_tol=ABS_TOL[dtype])


def test_lane_list_and_gather_modes_on_dense_cells(pg):
    # Dense periodic cells: staged planes take lane-list mode unless gather_only is set.
    # Both modes are bitwise equal to each other across launch shapes and match the oracle.
    wl = synth.crystal_shaped(n_cells=24)
    for dtype in ("f32", "f16"):
        auto = run(pg, wl, dtype=dtype, tuning={"path": 1, "block_threads": 256})
        gather = run(pg, wl, dtype=dtype,
                     tuning={"path": 1, "block_threads": 256, "gather_only": 1})
        assert np.array_equal(auto, gather)
        one = run(pg, wl, dtype=dtype,
                  tuning={"path": 1, "block_threads": 512, "chunk_planes": 1})
        assert np.array_equal(auto, one)
        g512 = run(pg, wl, dtype=dtype, tuning={"path": 1, "block_threads": 512,
                                                "chunk_planes": 2, "gather_only": 1})
        assert np.array_equal(gather, g512)
    grid_check(auto[:6], oracle.Problem.from_workload(wl, batch=wl.batch.subset(range(6))),
               TOL["f16"], abs_tol=ABS_TOL["f16"])


@pytest.mark.parametrize("kind", ["qm9", "crystal", "triclinic"])
def test_chunk_orders_give_identical_bits(pg, kind):
    # Molecule-major and channel-major chunk orders visit each voxel's atoms in the same
    # order, so the grids are bitwise equal (direct and general-cell kernels).
    wl = {"qm9": lambda: synth.qm9_shaped(n_mol=32),
          "crystal": lambda: synth.crystal_shaped(n_cells=6, grid=24),
          "triclinic": lambda: synth.crystal_triclinic(n_cells=6)}[kind]()
    db = pg.DeviceBatch.from_numpy(wl.batch)
    grid = pg.Grid.from_workload(wl)
    outs = []
    for order in (0, 1):
        outs.append(pg.voxelize_tuned(db, grid, {"path": 1, "block_threads": 256,
                                                 "chunk_planes": 4, "chunk_order": order},
                                      dtype="f16"))
    assert pg.sync_status() == 0
    assert torch.equal(outs[0], outs[1])


@pytest.mark.parametrize("periodic", [False, True])
def test_lane_list_mode_wide_discs(pg, periodic):
    # Wide discs on a fine grid (r_c = 1.5 A on 0.05 A voxels: about 60 voxels across, wider
    # than a pass) and dense planes of up to about 30 candidates; atoms near the faces so that
    # periodic images wrap.  Bitwise equal to the gather, and equal to the oracle.
    rng = np.random.default_rng(41)
    n = 64
    h = 0.05
    mols = []
    for _ in range(3):
        pos = rng.uniform(0.0, n * h, (40, 3))
        pos[:4] = [[0.02, 0.03, 3.1], [3.15, 0.1, 0.05], [1.6, 1.6, 1.6], [1.62, 1.58, 1.61]]
        mols.append(pos)
    el = [np.where(rng.uniform(size=40) < 0.7, 0, 1) for _ in range(3)]
    nb = synth._pack(mols, el, np.zeros((3, 3)), np.full((3, 3), h))
    wl = synth.plain_small(n_mol=1)
    wl.nx = wl.ny = wl.nz = n
    wl.periodic = periodic
    wl.cutoff_k = 3.0 if not periodic else 2.0    # r_c = 1.0 A < L / 2 = 1.6 A when periodic
    for dtype in ("f32", "f16"):
        auto = run(pg, wl, dtype=dtype, batch=nb, tuning={"path": 1, "block_threads": 128})
        gather = run(pg, wl, dtype=dtype, batch=nb, tuning={"path": 1, "gather_only": 1})
        assert np.array_equal(auto, gather)
        grid_check(auto, oracle.Problem.from_workload(wl, batch=nb), TOL[dtype],
                   abs_tol=ABS_TOL[dtype])
