"""Pins for the oracle's general cells and weighted grids (Sec. III-A).

General cells: the grid's axes run along the rows a, b, c of a 3x3 matrix M, and periodic
cells take the nearest image over the lattice translations.  What pins it:
- a diagonal M reproduces the axis-aligned box of spacing L/n (periodic or not);
- rotating the cell, origin and atoms together leaves the grid unchanged, which fails if M
  is used transposed anywhere;
- adding a lattice vector to an atom changes nothing;
- moving an atom by one voxel along a lattice vector rolls the grid by one index, including
  across the cell faces;
- a numpy search over a wide block of images agrees in a strongly skewed cell, where
  rounding the fractional displacement alone picks the wrong image for some voxels;
- the mass closed form holds in a skewed box, and the gradient of <v_x, G> is its
  closed form (2 pi sigma^2)^{3/2} / V_voxel along x.

Weights: unit weights change no bit; the grid is linear in the weights; the voxel-integrated
form conserves the weight sum; the weight gradient reproduces L by Euler's identity and
its finite difference; the coordinate gradient scales with the weight.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from synth import Batch

SKEW = np.array([[16.0, 0.0, 0.0], [5.0, 15.0, 0.0], [-3.0, 4.0, 14.0]])


def rotation(seed):
    q = np.random.default_rng(seed).standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def cell_batch(frac, elem, mol_off, cells, origins, weight=None):
    """Batch whose atoms are given in fractional coordinates of their molecule's cell."""
    coords = np.concatenate([
        frac[mol_off[b]:mol_off[b + 1]] @ cells[b] + origins[b]
        for b in range(len(cells))]) if len(frac) else np.zeros((0, 3))
    return Batch(coords=coords, elem=np.asarray(elem, np.int32),
                 mol_off=np.asarray(mol_off, np.int32), origin=np.asarray(origins, np.float64),
                 spacing=np.ones((len(cells), 3)), weight=weight,
                 cell=np.asarray(cells, np.float64))


def random_cells(seed, n_mol=3, atoms=6, C=2):
    rng = np.random.default_rng(seed)
    cells = np.stack([SKEW * rng.uniform(0.8, 1.1) for _ in range(n_mol)])
    origins = rng.uniform(-2.0, 2.0, (n_mol, 3))
    mol_off = np.arange(n_mol + 1) * atoms
    frac = rng.uniform(0.0, 1.0, (n_mol * atoms, 3))
    elem = rng.integers(0, C, n_mol * atoms)
    return frac, elem, mol_off, cells, origins


def problem(batch, n=(12, 10, 14), C=2, cutoff="sphere", periodic=True, sigma=(0.5, 0.7),
            **kw):
    return oracle.Problem(batch, *n, C, list(sigma)[:C], cutoff, 3.0, periodic, **kw)


@pytest.mark.parametrize("cutoff", ["sphere", "box", "none"])
@pytest.mark.parametrize("periodic", [False, True])
def test_diagonal_cell_equals_the_axis_aligned_box(oracle_lib, cutoff, periodic):
    wl = synth.plain_small(n_mol=3)
    b = wl.batch
    n = np.array([wl.nx, wl.ny, wl.nz])
    cells = np.stack([np.diag(n * b.spacing[m].astype(np.float64)) for m in range(b.n_mol)])
    boxed = oracle.Problem(b, wl.nx, wl.ny, wl.nz, wl.n_channels, wl.sigma, cutoff, 3.0,
                           periodic)
    celled = oracle.Problem(b, wl.nx, wl.ny, wl.nz, wl.n_channels, wl.sigma, cutoff, 3.0,
                            periodic, cell=cells)
    G0, G1 = oracle.voxelize(boxed), oracle.voxelize(celled)
    assert G0.max() > 0.5
    assert np.max(np.abs(G0 - G1)) < 1e-12


@pytest.mark.parametrize("cutoff", ["sphere", "none"])
@pytest.mark.parametrize("periodic", [False, True])
def test_rotating_cell_and_atoms_leaves_the_grid_unchanged(oracle_lib, cutoff, periodic):
    frac, elem, off, cells, origins = random_cells(1)
    G = oracle.voxelize(problem(cell_batch(frac, elem, off, cells, origins), cutoff=cutoff,
                                periodic=periodic))
    R = rotation(5)
    Gr = oracle.voxelize(problem(cell_batch(frac, elem, off, cells @ R, origins @ R),
                                 cutoff=cutoff, periodic=periodic))
    assert G.max() > 0.5
    assert np.max(np.abs(G - Gr)) < 1e-12


@pytest.mark.parametrize("cutoff", ["sphere", "box"])
def test_lattice_translations_change_nothing(oracle_lib, cutoff):
    frac, elem, off, cells, origins = random_cells(2)
    G = oracle.voxelize(problem(cell_batch(frac, elem, off, cells, origins), cutoff=cutoff))
    shift = np.random.default_rng(3).integers(-2, 3, frac.shape).astype(np.float64)
    Gt = oracle.voxelize(problem(cell_batch(frac + shift, elem, off, cells, origins),
                                 cutoff=cutoff))
    assert np.max(np.abs(G - Gt)) < 1e-11


@pytest.mark.parametrize("cutoff", ["sphere", "box"])
def test_one_voxel_lattice_shift_rolls_the_grid(oracle_lib, cutoff):
    n = (12, 10, 14)
    frac, elem, off, cells, origins = random_cells(4, n_mol=2, atoms=4)
    # Atoms at voxel centres' fractional offsets, moved across the faces by the shift.
    G = oracle.voxelize(problem(cell_batch(frac, elem, off, cells, origins), n=n,
                                cutoff=cutoff))
    s = np.array([5, -3, 9])
    Gs = oracle.voxelize(problem(cell_batch(frac + s / np.array(n), elem, off, cells, origins),
                                 n=n, cutoff=cutoff))
    assert np.max(np.abs(np.roll(G, tuple(s), axis=(2, 3, 4)) - Gs)) < 1e-11


def test_nearest_image_matches_a_wide_search_in_a_skewed_cell(oracle_lib):
    # A strongly sheared cell: the image nearest a voxel is often not the one found by
    # rounding the fractional displacement.
    M = np.array([[6.0, 0.0, 0.0], [5.2, 2.4, 0.0], [4.7, 1.9, 2.2]])
    n = (5, 4, 6)
    rng = np.random.default_rng(11)
    frac = rng.uniform(0, 1, (5, 3))
    b = cell_batch(frac, np.zeros(5, np.int32), [0, 5], M[None], np.zeros((1, 3)))
    sigma = 0.8
    G = oracle.voxelize(oracle.Problem(b, *n, 1, [sigma], "none", 3.0, True))
    x = frac @ M
    t = np.stack(np.meshgrid(*[np.arange(-4, 5)] * 3, indexing="ij"), -1).reshape(-1, 3)
    ref = np.zeros(n)
    rounded_differs = 0
    for i in range(n[0]):
        for j in range(n[1]):
            for k in range(n[2]):
                v = (np.array([i, j, k]) + 0.5) / np.array(n) @ M
                for a in range(5):
                    d = v - x[a] - t @ M
                    r2 = np.einsum("ij,ij->i", d, d)
                    best = r2.min()
                    ref[i, j, k] += math.exp(-best / (2 * sigma * sigma))
                    e = (v - x[a]) @ np.linalg.inv(M)
                    d0 = v - x[a] - np.rint(e) @ M
                    rounded_differs += (d0 @ d0) > best * (1 + 1e-9)
    assert rounded_differs > 10
    assert np.max(np.abs(G[0, 0] - ref)) < 1e-12


@pytest.mark.parametrize("cutoff", ["sphere", "box", "none"])
@pytest.mark.parametrize("periodic", [False, True])
def test_support_box_equals_brute_force_in_cells(oracle_lib, cutoff, periodic):
    frac, elem, off, cells, origins = random_cells(6)
    p = problem(cell_batch(frac, elem, off, cells, origins), cutoff=cutoff, periodic=periodic)
    assert np.array_equal(oracle.voxelize(p, "bbox"), oracle.voxelize(p, "brute"))


def single_atom_in(M, frac, n, cutoff, periodic, sigma=0.5, w=None):
    b = cell_batch(np.array([frac], np.float64), [0], [0, 1], M[None], np.zeros((1, 3)),
                   None if w is None else np.array([w], np.float64))
    return oracle.Problem(b, *n, 1, [sigma], cutoff, 3.0, periodic)


def test_mass_in_a_skewed_box(oracle_lib):
    n = (40, 40, 40)
    vvox = abs(np.linalg.det(SKEW)) / np.prod(n)
    mass = (2 * math.pi * 0.25) ** 1.5
    G = oracle.voxelize(single_atom_in(SKEW, [0.5, 0.5, 0.5], n, "none", False, w=1.5))
    assert abs(G.sum() * vvox / mass - 1.5) < 1e-12
    # Hard cutoffs converge to their own fractions of the mass, up to the sampling of the
    # cutoff surface (about 1e-3 at 40 voxels per edge), centred or wrapped across faces.
    sphere = math.erf(3 / math.sqrt(2)) - math.sqrt(2 / math.pi) * 3 * math.exp(-4.5)
    box = math.erf(3 / math.sqrt(2)) ** 3
    for frac in ([0.5, 0.5, 0.5], [0.02, 0.97, 0.01]):
        for cutoff, f in (("sphere", sphere), ("box", box)):
            G = oracle.voxelize(single_atom_in(SKEW, frac, n, cutoff, True))
            assert abs(G.sum() * vvox / mass / f - 1) < 2e-3, (frac, cutoff)


def test_gradient_of_x_weighting_in_a_skewed_box(oracle_lib):
    # L = sum_v v_x G(v): dL/dx_a = w (2 pi sigma^2)^{3/2} / V_voxel along x, zero along y, z.
    n = (40, 40, 40)
    w = 0.75
    p = single_atom_in(SKEW, [0.5, 0.45, 0.55], n, "none", False, w=w)
    u = (np.indices(n).reshape(3, -1).T + 0.5) / np.array(n)
    W = (u @ SKEW)[:, 0].reshape((1, 1) + n)
    g = oracle.gradient(p, W)
    expect = w * (2 * math.pi * 0.25) ** 1.5 / (abs(np.linalg.det(SKEW)) / np.prod(n))
    assert np.allclose(g[0], [expect, 0.0, 0.0], rtol=0, atol=1e-9 * expect)


@pytest.mark.parametrize("cutoff", ["sphere", "box"])
def test_cell_gradient_matches_frozen_finite_differences(oracle_lib, cutoff):
    frac, elem, off, cells, origins = random_cells(7, n_mol=2, atoms=5)
    w = np.random.default_rng(8).uniform(-1.5, 1.5, len(frac))
    p = problem(cell_batch(frac, elem, off, cells, origins, w), cutoff=cutoff)
    W = np.random.default_rng(9).standard_normal(p.shape)
    g = oracle.gradient(p, W)
    fd = oracle.fd_gradient_frozen(p, W, 1e-4)
    assert np.max(np.abs(g - fd)) <= 1e-6 * np.max(np.abs(g))
    # Brute force visits the voxels in another order (wrapped support vs grid order).
    assert np.max(np.abs(g - oracle.gradient(p, W, "brute"))) <= 1e-13 * np.max(np.abs(g))


def weighted_workload(seed=12):
    wl = synth.plain_small(n_mol=3)
    w = np.random.default_rng(seed).uniform(-1.0, 2.0, wl.batch.n_atoms)
    return wl, w


def test_unit_weights_change_no_bit(oracle_lib):
    wl = synth.plain_small(n_mol=3)
    p0 = oracle.Problem.from_workload(wl)
    p1 = oracle.Problem(wl.batch, wl.nx, wl.ny, wl.nz, wl.n_channels, wl.sigma, wl.cutoff,
                        wl.cutoff_k, wl.periodic, weight=np.ones(wl.batch.n_atoms))
    assert np.array_equal(oracle.voxelize(p0), oracle.voxelize(p1))


@pytest.mark.parametrize("form", ["point", "integral"])
def test_the_grid_is_linear_in_the_weights(oracle_lib, form):
    wl, w = weighted_workload()
    wl.form = form
    b = wl.batch
    G = oracle.voxelize(oracle.Problem(b, wl.nx, wl.ny, wl.nz, wl.n_channels, wl.sigma,
                                       wl.cutoff, wl.cutoff_k, wl.periodic, form=form,
                                       weight=w))
    ref = np.zeros_like(G)
    for m in range(b.n_mol):
        for a in range(b.mol_off[m], b.mol_off[m + 1]):
            one = Batch(coords=b.coords[a:a + 1], elem=b.elem[a:a + 1],
                        mol_off=np.array([0, 1], np.int32), origin=b.origin[m:m + 1],
                        spacing=b.spacing[m:m + 1])
            Ga = oracle.voxelize(oracle.Problem(one, wl.nx, wl.ny, wl.nz, wl.n_channels,
                                                wl.sigma, wl.cutoff, wl.cutoff_k, wl.periodic,
                                                form=form))
            ref[m] += w[a] * Ga[0]
    assert np.max(np.abs(G - ref)) < 1e-12


def test_the_integral_form_conserves_the_weight_sum(oracle_lib):
    wl, w = weighted_workload()
    wl.cutoff = "none"
    p = oracle.Problem(wl.batch, wl.nx, wl.ny, wl.nz, wl.n_channels, wl.sigma, "none", 3.0,
                       False, form="integral", weight=w)
    G = oracle.voxelize(p)
    for m in range(wl.batch.n_mol):
        s = wl.batch.atoms_of(m)
        assert abs(G[m].sum() - w[s].sum()) < 1e-6 * np.abs(w[s]).sum()


@pytest.mark.parametrize("cell", [False, True])
def test_weight_gradient_reproduces_the_loss(oracle_lib, cell):
    if cell:
        frac, elem, off, cells, origins = random_cells(13)
        w = np.random.default_rng(14).uniform(-1, 2, len(frac))
        p = problem(cell_batch(frac, elem, off, cells, origins, w))
    else:
        wl, w = weighted_workload()
        p = oracle.Problem(wl.batch, wl.nx, wl.ny, wl.nz, wl.n_channels, wl.sigma, wl.cutoff,
                           wl.cutoff_k, wl.periodic, weight=w)
    W = np.random.default_rng(15).standard_normal(p.shape)
    gw = oracle.gradient_weight(p, W)
    L = oracle.loss(p, W)
    # L is linear and homogeneous in w: L = sum_a w_a dL/dw_a.
    assert abs(float(w @ gw) - L) <= 1e-12 * max(1.0, abs(L))
    # A unit step of one weight changes L by exactly that atom's dL/dw.
    a = 2
    w2 = w.copy()
    w2[a] += 1.0
    p.weight[:] = w2
    assert abs(oracle.loss(p, W) - L - gw[a]) <= 1e-12 * max(1.0, abs(L))
    assert np.max(np.abs(gw - oracle.gradient_weight(p, W, "brute"))) <= \
        1e-13 * np.max(np.abs(gw))


def test_coordinate_gradient_scales_with_the_weight(oracle_lib):
    wl, w = weighted_workload()
    args = (wl.batch, wl.nx, wl.ny, wl.nz, wl.n_channels, wl.sigma, wl.cutoff, wl.cutoff_k,
            wl.periodic)
    W = np.random.default_rng(16).standard_normal((wl.batch.n_mol, wl.n_channels, wl.nx,
                                                   wl.ny, wl.nz))
    g1 = oracle.gradient(oracle.Problem(*args, weight=np.ones_like(w)), W)
    gw = oracle.gradient(oracle.Problem(*args, weight=w), W)
    assert np.allclose(gw, w[:, None] * g1, rtol=1e-14, atol=1e-14 * np.abs(g1).max())


def test_refinement_in_a_periodic_cell_recovers_the_truth(oracle_lib):
    frac, elem, off, cells, origins = random_cells(17, n_mol=2, atoms=4)
    b = cell_batch(frac, elem, off, cells, origins)
    truth = problem(b, n=(16, 16, 16))
    T = oracle.voxelize(truth)
    start = b.coords + np.random.default_rng(18).normal(0, 0.08, b.coords.shape)
    x, loss, steps = oracle.refine(problem(b, n=(16, 16, 16), coords=start), T, 400, 0.02)
    assert np.max(np.abs(x - truth.coords)) < 1e-5
    assert np.all(loss < 1e-10)


def test_cells_reject_the_integral_and_separable_forms(oracle_lib):
    frac, elem, off, cells, origins = random_cells(19)
    b = cell_batch(frac, elem, off, cells, origins)
    with pytest.raises(ValueError):
        oracle.voxelize(problem(b, form="integral"))
    with pytest.raises(ValueError):
        oracle.separable(problem(b, cutoff="box"))


@pytest.mark.parametrize("cutoff", ["box", "none"])
@pytest.mark.parametrize("form", ["point", "integral"])
def test_weighted_separable_form_equals_the_direct_sum(oracle_lib, cutoff, form):
    wl, w = weighted_workload()
    p = oracle.Problem(wl.batch, wl.nx, wl.ny, wl.nz, wl.n_channels, wl.sigma, cutoff, 3.0,
                       False, form=form, weight=w)
    G = oracle.voxelize(p)
    assert np.max(np.abs(oracle.separable(p) - G)) < 1e-12 * np.abs(G).max()
