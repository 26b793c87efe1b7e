"""Pins for the oracle's voxel-integrated form (Sec. III-A, the gridding function after
Eq. 5: each voxel holds the normalised Gaussian integrated over it, a product of per-axis
erf differences).

They check closed forms that follow from integrating a normalised Gaussian over voxels
rather than re-evaluating the oracle's formula:

* a single voxel's integral is the product of three one-dimensional probabilities of a
  normal variable (math.erf);
* sums over contiguous voxel ranges telescope to the probability of the covered interval,
  so the total over a grid, over a box-cutoff range or over a periodic cell is known
  exactly, and deep inside a grid each atom contributes exactly one (the conservation law
  after Eq. 5);
* for small voxels the integral tends to h^3 times the normalised density;
* the coordinate derivative agrees with finite differences of the value, and the
  derivative of <v_x, G> is one.

A swapped edge order (negative values), the voxel centre used as the lower edge, sigma in
place of sqrt(2) sigma, a missing factor 1/2 or a transposed axis each fails one of them.
"""
import math

import numpy as np
import pytest

import oracle
import synth


def make(atoms, elems, n, C, sigma, origin=(0.0, 0.0, 0.0), spacing=(0.5, 0.5, 0.5),
         cutoff="none", k=3.0, periodic=False):
    batch = synth.single_atom_batch([atoms], [elems], origin, spacing)
    coords = np.asarray(atoms, float).reshape(-1, 3)
    batch.origin = np.asarray([origin], float)
    batch.spacing = np.asarray([spacing], float)
    return oracle.Problem(batch, *n, C, np.broadcast_to(np.asarray(sigma, float), (C,)),
                          cutoff, k, periodic, coords=coords, form="integral")


def normal_prob(a, b, mu, sigma):
    """P(a <= X <= b) for X ~ N(mu, sigma^2)."""
    s = math.sqrt(2.0) * sigma
    return 0.5 * (math.erf((b - mu) / s) - math.erf((a - mu) / s))


def test_voxel_values_are_normal_probabilities_of_the_voxel(oracle_lib):
    n, h, o = (9, 11, 13), (0.5, 0.25, 0.75), (-1.0, 2.0, 0.5)
    sigma = 0.6
    x = [o[0] + 3.3 * h[0], o[1] + 7.9 * h[1], o[2] + 5.5 * h[2]]
    G = oracle.voxelize(make([x], [0], n, 1, sigma, o, h))[0, 0]
    for ijk in [(3, 7, 5), (0, 0, 0), (8, 10, 12), (4, 6, 5), (2, 8, 6)]:
        want = 1.0
        for ax in range(3):
            lo = o[ax] + ijk[ax] * h[ax]
            want *= normal_prob(lo, lo + h[ax], x[ax], sigma)
        assert G[ijk] == pytest.approx(want, rel=1e-13, abs=1e-300)
    assert np.all(G >= 0.0)


def test_total_telescopes_to_probability_of_the_grid_box(oracle_lib):
    # Any atom position, even outside the grid: the grid total is the probability that the
    # atom's Gaussian lands inside the grid's box.
    rng = np.random.default_rng(5)
    n, h, o = (12, 10, 14), (0.5, 0.6, 0.4), (0.0, -1.0, 0.5)
    for trial in range(6):
        x = [o[a] + rng.uniform(-1.0, 1.0 + n[a] * h[a]) for a in range(3)]
        sigma = rng.uniform(0.3, 0.9)
        G = oracle.voxelize(make([x], [0], n, 1, sigma, o, h))[0, 0]
        want = 1.0
        for ax in range(3):
            want *= normal_prob(o[ax], o[ax] + n[ax] * h[ax], x[ax], sigma)
        assert G.sum() == pytest.approx(want, rel=1e-12, abs=1e-300)


def test_conservation_each_atom_contributes_one(oracle_lib):
    # The conservation law after Eq. 5: the grid sums to the number of atoms, and each
    # channel to the number of atoms of that element.
    rng = np.random.default_rng(8)
    atoms = 8.0 + rng.uniform(-2.0, 2.0, (7, 3))
    elems = [0, 1, 1, 2, 0, 1, 1]
    G = oracle.voxelize(make(atoms, elems, (32, 32, 32), 3, 0.5))[0]
    per_channel = G.reshape(3, -1).sum(axis=1)
    assert per_channel == pytest.approx([2.0, 4.0, 1.0], abs=1e-12)
    assert G.sum() == pytest.approx(7.0, abs=1e-12)


def test_box_cutoff_sums_telescope_over_the_kept_centres(oracle_lib):
    # With a box cutoff the kept voxels on each axis are those whose centre lies within
    # r_c; their values telescope to the probability of the union of their intervals.
    n, h, o = (24, 20, 28), (0.5, 0.55, 0.45), (0.0, 0.0, 0.0)
    x = [6.13, 5.02, 6.71]
    sigma, k = 0.6, 2.0
    G = oracle.voxelize(make([x], [0], n, 1, sigma, o, h, cutoff="box", k=k))[0, 0]
    want = 1.0
    for ax in range(3):
        c = o[ax] + (np.arange(n[ax]) + 0.5) * h[ax]
        kept = np.nonzero(np.abs(c - x[ax]) <= k * sigma)[0]
        assert np.all(np.diff(kept) == 1)
        want *= normal_prob(o[ax] + kept[0] * h[ax], o[ax] + (kept[-1] + 1) * h[ax], x[ax],
                            sigma)
    assert G.sum() == pytest.approx(want, rel=1e-12)


def test_periodic_cell_sums_to_one_per_atom(oracle_lib):
    # Minimum image over a cell much wider than sigma: every voxel of the cell sees the
    # nearest image, the per-axis ranges tile one period around the atom, and the total is
    # one up to the Gaussian mass beyond half a cell.
    n, h = (16, 18, 20), (0.5, 0.5, 0.45)
    for x in ([0.1, 8.7, 4.4], [7.99, 0.01, 8.9], [-3.0, 12.0, 30.0]):
        G = oracle.voxelize(make([x], [0], n, 1, 0.5, (0, 0, 0), h, periodic=True))[0, 0]
        assert G.sum() == pytest.approx(1.0, abs=1e-12)


def test_small_voxels_tend_to_density_times_volume(oracle_lib):
    # h -> 0: G / h^3 -> the normalised density; the midpoint error is O(h^2 / sigma^2).
    sigma = 0.5
    for h in (0.1, 0.05):
        n = int(round(4.0 / h))
        x = [2.0, 2.0, 2.0]
        G = oracle.voxelize(make([x], [0], (n, n, n), 1, sigma, (0, 0, 0), (h, h, h)))[0, 0]
        i = n // 2
        c = (i + 0.5) * h
        d2 = 3 * (c - 2.0) ** 2
        dens = math.exp(-d2 / (2 * sigma ** 2)) / (2 * math.pi * sigma ** 2) ** 1.5
        assert G[i, i, i] / h ** 3 == pytest.approx(dens, rel=(h / sigma) ** 2 / 4)


@pytest.mark.parametrize("cutoff,periodic", [("none", False), ("box", False), ("box", True),
                                             ("none", True)])
def test_separable_equals_direct(oracle_lib, cutoff, periodic):
    rng = np.random.default_rng(9)
    atoms = 4.0 + rng.uniform(-1.5, 1.5, (6, 3))
    prob = make(atoms, [0, 1, 0, 1, 1, 0], (16, 14, 18), 2, [0.5, 0.7], cutoff=cutoff,
                periodic=periodic)
    assert np.allclose(oracle.separable(prob), oracle.voxelize(prob), rtol=0, atol=1e-15)


@pytest.mark.parametrize("cutoff,periodic", [("sphere", False), ("box", True), ("none", False)])
def test_brute_force_equals_support_box_bitwise(oracle_lib, cutoff, periodic):
    rng = np.random.default_rng(10)
    atoms = 3.0 + rng.uniform(-1.5, 1.5, (5, 3))
    prob = make(atoms, [0, 1, 0, 1, 0], (12, 12, 12), 2, [0.4, 0.6], cutoff=cutoff,
                periodic=periodic)
    assert np.array_equal(oracle.voxelize(prob, "brute"), oracle.voxelize(prob, "bbox"))


@pytest.mark.parametrize("cutoff,periodic", [("none", False), ("sphere", False), ("box", True)])
def test_gradient_matches_finite_differences_of_the_value(oracle_lib, cutoff, periodic):
    rng = np.random.default_rng(12)
    atoms = 4.0 + rng.uniform(-1.0, 1.0, (5, 3))
    prob = make(atoms, [0, 1, 1, 0, 1], (16, 16, 16), 2, [0.5, 0.6], cutoff=cutoff,
                periodic=periodic)
    W = np.random.default_rng(13).standard_normal(prob.shape)
    g = oracle.gradient(prob, W)
    fd = oracle.fd_gradient_frozen(prob, W, step=1e-4)
    assert np.max(np.abs(g - fd)) <= 1e-7 * np.max(np.abs(g))
    if cutoff == "none":
        # Raw central differences of the whole forward pass (no support to freeze).
        base = prob.coords.copy()
        for a in range(base.shape[0]):
            for ax in range(3):
                lp, lm = base.copy(), base.copy()
                lp[a, ax] += 1e-4
                lm[a, ax] -= 1e-4
                Lp = oracle.loss(make(lp, [0, 1, 1, 0, 1], (16, 16, 16), 2, [0.5, 0.6]), W)
                Lm = oracle.loss(make(lm, [0, 1, 1, 0, 1], (16, 16, 16), 2, [0.5, 0.6]), W)
                assert (Lp - Lm) / 2e-4 == pytest.approx(g[a, ax], rel=1e-6, abs=1e-9)


def test_gradient_of_first_moment_is_one(oracle_lib):
    # L = <v_x, G> = E[centre_x(X)] for the atom's Gaussian X, which is mu_x up to the
    # aliasing term ~ exp(-2 pi^2 sigma^2 / h^2); dL/dmu = (1, 0, 0).
    n, h = (40, 40, 40), 0.5
    x = [10.07, 9.93, 10.21]
    prob = make([x], [0], n, 1, 0.5, (0, 0, 0), (h, h, h))
    cx = (np.arange(n[0]) + 0.5) * h
    W = np.broadcast_to(cx[:, None, None], n)[None, None].copy()
    g = oracle.gradient(prob, W)[0]
    assert g == pytest.approx([1.0, 0.0, 0.0], abs=1e-7)
