"""Split one batch of independent molecules across data-parallel ranks.

Molecules are independent units of the voxelization (each grid depends only on its own
atoms), so a batch shards into contiguous molecule ranges with no exchange between ranks:
each rank voxelizes its range on its own GPU.  Ranges are balanced by the estimated cost of
a molecule - its output bytes (the dominant, write-bound part) plus a per-atom term.
"""
from __future__ import annotations

import numpy as np


def molecule_costs(mol_off, out_bytes_per_mol: float, bytes_per_atom: float = 2048.0):
    """Estimated cost of each molecule in byte-equivalents."""
    mol_off = np.asarray(mol_off, dtype=np.int64)
    atoms = np.diff(mol_off)
    return out_bytes_per_mol + bytes_per_atom * atoms


def partition(mol_off, n_parts: int, out_bytes_per_mol: float, bytes_per_atom: float = 2048.0):
    """Contiguous ranges [(start, stop), ...] of molecules, one per part, whose costs are as
    equal as the molecule granularity allows (each boundary is placed at the prefix-cost
    quantile k * total / n_parts)."""
    if n_parts < 1:
        raise ValueError("n_parts must be >= 1")
    cost = molecule_costs(mol_off, out_bytes_per_mol, bytes_per_atom)
    n = cost.shape[0]
    prefix = np.concatenate([[0.0], np.cumsum(cost)])
    total = prefix[-1]
    bounds = [0]
    for k in range(1, n_parts):
        target = total * k / n_parts
        j = int(np.searchsorted(prefix, target, side="left"))
        # pick the closer of the two prefix points around the target
        if j > 0 and (j > n or abs(prefix[j - 1] - target) <= abs(prefix[j] - target)):
            j -= 1
        bounds.append(min(max(j, bounds[-1]), n))
    bounds.append(n)
    return [(bounds[i], bounds[i + 1]) for i in range(n_parts)]


def shard(batch, rank: int, world: int, out_bytes_per_mol: float, bytes_per_atom: float = 2048.0):
    """This rank's contiguous sub-batch of `batch` (a ``synth.Batch``-like object with
    coords/elem/mol_off/origin/spacing arrays); returns (sub_batch, (start, stop))."""
    start, stop = partition(batch.mol_off, world, out_bytes_per_mol, bytes_per_atom)[rank]
    return batch.subset(range(start, stop)), (start, stop)
