"""The multi-rank path on CPU: two gloo ranks each voxelize their own contiguous shard of one
batch (no collective on the data path); the union of their grids must equal the
single-process result, shard by shard.  The collectives here only gather checksums for the
check itself."""
import os
import socket

import numpy as np
import pytest

import synth
from paper_2211_08506_gb300 import shard

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_partition_covers_once_and_balances():
    wl = synth.qm9_shaped(n_mol=1000)
    per_mol = wl.voxels_per_grid * 4
    for world in (1, 2, 3, 8):
        parts = shard.partition(wl.batch.mol_off, world, per_mol)
        assert parts[0][0] == 0 and parts[-1][1] == 1000
        assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
        cost = shard.molecule_costs(wl.batch.mol_off, per_mol)
        loads = [cost[a:b].sum() for a, b in parts]
        assert max(loads) - min(loads) <= 2 * cost.max()


def test_partition_handles_more_parts_than_molecules():
    off = np.array([0, 3, 5], np.int32)
    parts = shard.partition(off, 4, 100.0)
    assert len(parts) == 4 and parts[-1][1] == 2
    assert sum(b - a for a, b in parts) == 2


def _worker(rank, world, port, q):
    import oracle

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = synth.qm9_shaped(n_mol=24)
        sub, (start, stop) = shard.shard(wl.batch, rank, world, wl.voxels_per_grid * 4)
        G = oracle.voxelize(oracle.Problem.from_workload(wl, batch=sub), "bbox", 1)
        sums = [float(G[i].sum()) for i in range(G.shape[0])]
        gathered = [None] * world
        dist.all_gather_object(gathered, (start, stop, sums))
        if rank == 0:
            q.put(gathered)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_single_process_grids():
    import multiprocessing as mp

    import oracle

    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    wl = synth.qm9_shaped(n_mol=24)
    G = oracle.voxelize(oracle.Problem.from_workload(wl), "bbox", 1)
    covered = []
    for start, stop, sums in gathered:
        covered += list(range(start, stop))
        for i, s in zip(range(start, stop), sums):
            assert s == float(G[i].sum())
    assert covered == list(range(24))


def _union_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # As the benchmark's ranks do: every rank builds the same global batch (world times the
        # per-rank size, one seed) and keeps its contiguous range.
        whole = synth.qm9_shaped(n_mol=40 * world)
        sub, (start, stop) = shard.shard(whole.batch, rank, world, whole.voxels_per_grid * 4)
        parts = [None] * world
        dist.all_gather_object(parts, (start, stop, sub.coords, sub.elem, sub.mol_off,
                                       sub.origin, sub.spacing))
        if rank == 0:
            q.put(parts)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_rank_shares_reassemble_the_global_batch(world):
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_union_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    parts = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    whole = synth.qm9_shaped(n_mol=40 * world).batch
    assert parts[0][0] == 0 and parts[-1][1] == whole.n_mol
    assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
    # Concatenated per-molecule inputs equal the global batch's, molecule by molecule.
    coords = np.concatenate([p[2] for p in parts])
    elem = np.concatenate([p[3] for p in parts])
    assert np.array_equal(coords, whole.coords) and np.array_equal(elem, whole.elem)
    assert np.array_equal(np.concatenate([p[5] for p in parts]), whole.origin)
    assert np.array_equal(np.concatenate([p[6] for p in parts]), whole.spacing)
    counts = np.concatenate([np.diff(p[4]) for p in parts])
    assert np.array_equal(counts, np.diff(whole.mol_off))
    # Every share is within one molecule's cost of an equal split.
    cost = shard.molecule_costs(whole.mol_off, synth.qm9_shaped(n_mol=1).voxels_per_grid * 4)
    loads = [cost[a:b].sum() for a, b, *_ in parts]
    assert max(loads) - min(loads) <= 2 * cost.max()
