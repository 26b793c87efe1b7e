"""CPU checks of the seeded input recipes that the general-cell and pipeline workloads rely on:
the triclinic generator's guarantees (face-to-face widths, minimum separation under the
nearest image, weights, coordinates inside the cell, determinism) and the pipeline
workload's adaptive boxes (every atom's support inside its grid, one channel, sizes)."""
import numpy as np

import synth


def test_triclinic_cells_keep_their_guarantees():
    wl = synth.crystal_triclinic(n_cells=8)
    b = wl.batch
    assert b.cell.shape == (8, 3, 3) and b.weight.shape == (b.n_atoms,)
    assert np.all((b.weight >= 0.5) & (b.weight <= 1.5))
    shifts = np.stack(np.meshgrid(*[np.arange(-1, 2)] * 3, indexing="ij"), -1).reshape(-1, 3)
    for m in range(b.n_mol):
        M = b.cell[m].astype(np.float64)
        Mi = np.linalg.inv(M)
        # Every face-to-face width is at least 3.2 A, so the 1.5 A cutoff stays within half
        # a cell along each fractional axis.
        assert np.min(1.0 / np.linalg.norm(Mi, axis=0)) >= 3.2 - 1e-4
        x = b.coords[b.atoms_of(m)].astype(np.float64)
        frac = (x - b.origin[m]) @ Mi
        assert np.all(frac > -1e-5) and np.all(frac < 1 + 1e-5)
        # Minimum separation 1.2 A over all neighbouring images (float32 rounding aside).
        d = frac[:, None, :] - frac[None, :, :]
        d -= np.round(d)
        img = (d[:, :, None, :] + shifts[None, None]) @ M
        r = np.sqrt((img ** 2).sum(axis=3)).min(axis=2)
        np.fill_diagonal(r, np.inf)
        assert r.min() >= 1.2 - 1e-4
    again = synth.crystal_triclinic(n_cells=8)
    assert np.array_equal(again.batch.coords, b.coords)
    assert np.array_equal(again.batch.cell, b.cell)


def test_triclinic_subsets_carry_cells_and_weights():
    b = synth.crystal_triclinic(n_cells=5).batch
    sub = b.subset([3, 1])
    assert np.array_equal(sub.cell, b.cell[[3, 1]])
    assert np.array_equal(sub.weight, np.concatenate([b.weight[b.atoms_of(3)],
                                                      b.weight[b.atoms_of(1)]]))


def test_pipeline_boxes_hold_every_support():
    wl = synth.pipeline_single_channel(n_mol=64)
    b = wl.batch
    assert wl.n_channels == 1 and np.all(b.elem == 0)
    sizes = np.diff(b.mol_off)
    assert sizes.min() >= 4 and sizes.max() <= 51
    reach = wl.cutoff_k * float(wl.sigma[0])
    for m in range(b.n_mol):
        x = b.coords[b.atoms_of(m)]
        lo = b.origin[m]
        hi = lo + wl.nx * b.spacing[m]
        assert np.all(x - reach >= lo - 1e-4) and np.all(x + reach <= hi + 1e-4)
