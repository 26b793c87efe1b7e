"""GPU parity of the voxel-integrated (erf) form of Sec. III-A through the C ABI, against
the FP64 oracle: the direct kernel in every dtype, cutoff and boundary mode (ragged and
vector store paths), the separable tcgen05 path, the adjoint, the conservation law after
Eq. 5 on the GPU's own output, and sampled parity on the full precision-form batch in the
launch configuration the benchmark uses."""
import numpy as np
import pytest

import oracle
import synth
from tests.parity import ABS_TOL, GRAD_TOL, SEPARABLE_TOL, TOL, grad_check, grid_check

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [("sphere", False), ("box", False), ("none", False), ("sphere", True), ("box", True),
         ("none", True)]


@pytest.fixture(scope="module")
def pg():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2211_08506_gb300 as pkg
    pkg.build()
    from paper_2211_08506_gb300 import api
    return api


def integral(wl):
    wl.form = "integral"
    return wl


def run(pg, wl, dtype="f32", path="direct", batch=None):
    batch = wl.batch if batch is None else batch
    G = pg.voxelize(pg.DeviceBatch.from_numpy(batch), pg.Grid.from_workload(wl), dtype=dtype,
                    path=path)
    assert pg.sync_status() == 0
    return G.float().cpu().numpy()


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("cutoff,periodic", CASES)
def test_direct_matches_oracle(pg, dtype, cutoff, periodic):
    wl = integral(synth.plain_small(n_mol=6))
    wl.cutoff, wl.periodic = cutoff, periodic
    wl.sigma = np.array([0.4, 0.5, 0.6, 0.55, 0.45], np.float32)
    if periodic:
        wl.cutoff_k = 2.5
    stats = grid_check(run(pg, wl, dtype), oracle.Problem.from_workload(wl), TOL[dtype],
                       abs_tol=ABS_TOL[dtype])
    if dtype == "f32":
        assert stats["max_abs_rel"] < 1e-5


def test_ragged_grid_scalar_store_path(pg):
    wl = integral(synth.plain_small(n_mol=4))
    wl.nx, wl.ny, wl.nz = 21, 19, 23
    for dtype in ("f32", "f16"):
        grid_check(run(pg, wl, dtype), oracle.Problem.from_workload(wl), TOL[dtype],
                   abs_tol=ABS_TOL[dtype])


def test_large_molecules_staged_path(pg):
    # Crystal cells (tens to hundreds of atoms) take the staged gather path.
    wl = integral(synth.crystal_shaped(n_cells=4))
    grid_check(run(pg, wl, "f32"), oracle.Problem.from_workload(wl), TOL["f32"],
               abs_tol=ABS_TOL["f32"])


def test_conservation_on_the_gpu_output(pg):
    # No cutoff and atoms far from the edges: each molecule's grid sums to its atom count
    # and each channel to its element count (the law after Eq. 5), in FP32 accumulation.
    wl = integral(synth.plain_small(n_mol=8))
    wl.cutoff = "none"
    wl.nx = wl.ny = wl.nz = 48
    wl.batch.origin = wl.batch.origin - 4.0   # 24 A box around the 16 A molecules
    G = run(pg, wl, "f32").astype(np.float64)
    b = wl.batch
    for m in range(b.n_mol):
        counts = np.bincount(b.elem[b.atoms_of(m)], minlength=wl.n_channels)
        assert G[m].reshape(wl.n_channels, -1).sum(axis=1) == pytest.approx(counts, abs=2e-4)


@pytest.mark.parametrize("cutoff,periodic", [("none", False), ("box", False), ("box", True)])
def test_separable_matches_oracle(pg, cutoff, periodic):
    wl = integral(synth.plain_small(n_mol=3))
    wl.cutoff, wl.periodic = cutoff, periodic
    if periodic:
        wl.cutoff_k = 2.5
    grid_check(run(pg, wl, "f16", "separable"), oracle.Problem.from_workload(wl),
               SEPARABLE_TOL, abs_tol=ABS_TOL["f16"])


@pytest.mark.parametrize("cutoff,periodic", CASES)
def test_adjoint_matches_oracle(pg, cutoff, periodic):
    wl = integral(synth.differentiation(n_mol=8))
    wl.cutoff, wl.periodic = cutoff, periodic
    if periodic:
        wl.cutoff_k = 2.5
    W = synth.loss_weights(wl)
    db = pg.DeviceBatch.from_numpy(wl.batch)
    g = pg.voxelize_backward(db, pg.Grid.from_workload(wl), torch.as_tensor(W, device="cuda"))
    assert pg.sync_status() == 0
    prob = oracle.Problem.from_workload(wl)
    grad_check(g.cpu().numpy(), oracle.gradient(prob, W), wl.batch.mol_off)
    grad_check(g.cpu().numpy(), oracle.fd_gradient_frozen(prob, W, 1e-4), wl.batch.mol_off,
               rel_tol=GRAD_TOL + 1e-6)


def test_full_precision_form_batch_sampled(pg):
    # The 4096-molecule erf-form batch on the tuned path (separable, FP16), as the benchmark
    # runs it; sampled molecules against the oracle.
    wl = synth.precision_form_integral()
    db = pg.DeviceBatch.from_numpy(wl.batch)
    grid = pg.Grid.from_workload(wl)
    out = torch.empty(grid.out_shape(wl.batch.n_mol), dtype=torch.float16, device="cuda")
    pg.autotune(db, grid, dtype="f16", path="auto", out=out)
    G = pg.voxelize(db, grid, dtype="f16", path="auto", out=out)
    assert pg.sync_status() == 0
    pick = [0, 1, 2047, 4095]
    sub = wl.batch.subset(pick)
    grid_check(G[pick].float().cpu().numpy(), oracle.Problem.from_workload(wl, batch=sub),
               SEPARABLE_TOL, abs_tol=ABS_TOL["f16"])


def test_factor_tables_bitwise_across_launch_shapes(pg):
    # With a separable cutoff, molecules of at most 32 atoms use per-chunk factor tables.  The
    # table entries are the values the kernel would compute per voxel, so every chunk size,
    # chunk order and block size gives identical bits, matching the oracle.
    wl = synth.precision_form_integral(n_mol=12)
    db = pg.DeviceBatch.from_numpy(wl.batch)
    grid = pg.Grid.from_workload(wl)
    ref = None
    for threads in (128, 256, 512):
        for cp in (1, 3, 8, 64):
            for order in (0, 1):
                G = pg.voxelize_tuned(db, grid, {"path": 1, "block_threads": threads,
                                                 "chunk_planes": cp, "chunk_order": order},
                                      dtype="f32")
                assert pg.sync_status() == 0
                if ref is None:
                    ref = G.clone()
                assert torch.equal(G, ref), (threads, cp, order)
    # Without the tables (every factor computed where it is used): the same bits.
    G = pg.voxelize_tuned(db, grid, {"path": 1, "gather_only": 1}, dtype="f32")
    assert pg.sync_status() == 0
    assert torch.equal(G, ref)
    pick = [0, 5, 11]
    grid_check(ref[pick].cpu().numpy(),
               oracle.Problem.from_workload(wl, batch=wl.batch.subset(pick)), TOL["f32"],
               abs_tol=ABS_TOL["f32"])


@pytest.mark.parametrize("cutoff,periodic", [("box", False), ("none", False), ("box", True)])
def test_factor_tables_with_large_molecules_interleaved(pg, cutoff, periodic):
    # Small molecules interleaved with 40-atom ones (staged path, which overwrites the small
    # molecules' cached table), one-plane chunks so that warps switch between the two often.
    wl = integral(synth.plain_small(n_mol=6))
    wl.cutoff, wl.periodic = cutoff, periodic
    wl.cutoff_k = 2.5
    b = wl.batch
    coords, elems = [], []
    rng = np.random.default_rng(5)
    for i in range(b.n_mol):
        s = b.atoms_of(i)
        c, e = b.coords[s], b.elem[s]
        if i % 2:
            extra = c[rng.integers(0, len(c), 40 - len(c))] + rng.normal(0, 0.7, (40 - len(c), 3))
            c = np.concatenate([c, extra]).astype(np.float32)
            e = np.concatenate([e, rng.integers(0, 5, 40 - len(e))]).astype(np.int32)
        coords.append(c)
        elems.append(e)
    nb = synth._pack(coords, elems, b.origin, b.spacing)
    db = pg.DeviceBatch.from_numpy(nb)
    grid = pg.Grid.from_workload(wl)
    # Tables for the small molecules (register path) and for the 40-atom ones (staged path),
    # against every factor computed where it is used: identical bits.
    outs = [pg.voxelize_tuned(db, grid, {"path": 1, "chunk_planes": cp, "gather_only": go},
                              dtype=dt)
            for dt in ("f32", "bf16") for cp in (1, 8) for go in (0, 1)]
    assert pg.sync_status() == 0
    for k in (1, 2, 3):
        assert torch.equal(outs[0], outs[k]), k
    for k in (5, 6, 7):
        assert torch.equal(outs[4], outs[k]), k
    grid_check(outs[0].cpu().numpy(), oracle.Problem.from_workload(wl, batch=nb), TOL["f32"],
               abs_tol=ABS_TOL["f32"])
