"""Pins for the FP64 oracle against facts the paper and the mathematics fix.

None of these compare the oracle with a retyped copy of its own formula.  They check
closed forms (lattice sums of a Gaussian, the normalisation constant of Eq. 1, the
gradient of <v_x, G>), invariants (translation, linearity, permutation, channel
separation, the point-sampled analog of the conservation law after Eq. 5), special cases
(an atom on a voxel centre, inclusive cutoffs hitting lattice points, periodic images as
explicit copies) and brute force on tiny inputs.  A dropped factor of two, sigma used as
a variance, a transposed axis, a wrong voxel-centre offset, a sign error in the gradient
or a broken minimum image each fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle
import synth


def make(atoms, elems, n, C, sigma, origin=(0.0, 0.0, 0.0), spacing=(0.5, 0.5, 0.5),
         cutoff="none", k=3.0, periodic=False, mols=None):
    """Problem with FP64 coordinates (no float32 rounding of the positions)."""
    if mols is None:
        mols = [(atoms, elems)]
    batch = synth.single_atom_batch([m[0] for m in mols], [m[1] for m in mols], origin, spacing)
    coords = np.concatenate([np.asarray(m[0], float).reshape(-1, 3) for m in mols])
    batch.origin = np.tile(np.asarray(origin, float), (len(mols), 1))
    batch.spacing = np.tile(np.asarray(spacing, float), (len(mols), 1))
    return oracle.Problem(batch, *n, C, np.broadcast_to(np.asarray(sigma, float), (C,)),
                          cutoff, k, periodic, coords=coords)


def centres(o, h, n):
    return o + (np.arange(n) + 0.5) * h


# --- P1: an atom on a voxel centre --------------------------------------------------

def test_atom_on_voxel_centre_peaks_at_one_on_the_right_index(oracle_lib):
    n, h, o = (9, 11, 13), (0.5, 0.25, 0.75), (-1.0, 2.0, 0.5)
    ijk = (3, 7, 5)
    x = [o[a] + (ijk[a] + 0.5) * h[a] for a in range(3)]
    G = oracle.voxelize(make([x], [0], n, 1, 0.6, o, h))[0, 0]
    assert G.shape == n
    assert G[ijk] == 1.0
    assert np.unravel_index(np.argmax(G), n) == ijk
    # One voxel along each axis decays with that axis's own spacing (axis order pin).
    s2 = 2 * 0.6 ** 2
    for ax in range(3):
        e = list(ijk)
        e[ax] += 1
        f = list(ijk)
        f[ax] -= 1
        assert G[tuple(e)] == pytest.approx(math.exp(-h[ax] ** 2 / s2), rel=1e-15)
        assert G[tuple(e)] == G[tuple(f)]
    # Distinct spacings must give distinct neighbour values, so a transposed axis shows.
    assert len({G[4, 7, 5], G[3, 8, 5], G[3, 7, 6]}) == 3


# --- P2: mass (point-sampled analog of "sum = number of atoms", after Eq. 5) ------------

def test_mass_without_cutoff_matches_gaussian_normalisation(oracle_lib):
    # sum_v G h^3 -> (2 pi sigma^2)^{3/2}; by Poisson summation the relative error is
    # about 6 exp(-2 pi^2 sigma^2 / h^2) ~ 2e-8 at sigma = h = 0.5.
    rng = np.random.default_rng(1)
    for sigma in (0.5, 0.7):
        x = 8.0 + rng.uniform(-0.5, 0.5, 3)
        G = oracle.voxelize(make([x], [0], (32, 32, 32), 1, sigma))[0, 0]
        mass = G.sum() * 0.5 ** 3
        assert mass == pytest.approx((2 * math.pi * sigma ** 2) ** 1.5, rel=1e-7)


def test_second_moment_per_axis_is_sigma_squared(oracle_lib):
    # sigma is the standard deviation of the sampled Gaussian (reading of "variance").
    n, h, o = (40, 36, 44), (0.4, 0.45, 0.35), (0.0, 0.0, 0.0)
    x = np.array([8.03, 7.91, 7.77])
    sigma = 0.9
    G = oracle.voxelize(make([x], [0], n, 1, sigma, o, h))[0, 0]
    c = [centres(o[a], h[a], n[a]) - x[a] for a in range(3)]
    tot = G.sum()
    mx = (G.sum(axis=(1, 2)) * c[0] ** 2).sum() / tot
    my = (G.sum(axis=(0, 2)) * c[1] ** 2).sum() / tot
    mz = (G.sum(axis=(0, 1)) * c[2] ** 2).sum() / tot
    for m in (mx, my, mz):
        assert m == pytest.approx(sigma ** 2, rel=1e-6)


def test_per_channel_mass_counts_atoms(oracle_lib):
    # Each channel's mass / (2 pi sigma_c^2)^{3/2} equals that channel's atom count.
    rng = np.random.default_rng(2)
    sig = np.array([0.4, 0.6, 0.5])
    el = np.array([0, 1, 1, 2, 0, 1, 2, 2, 2])
    x = 9.0 + rng.uniform(-2.0, 2.0, (el.size, 3))
    # h = 0.25 keeps the Poisson alias term 2 exp(-2 pi^2 sigma^2/h^2) below 1e-13.
    G = oracle.voxelize(make(x, el, (72, 72, 72), 3, sig, spacing=(0.25,) * 3))[0]
    for c in range(3):
        count = G[c].sum() * 0.25 ** 3 / (2 * math.pi * sig[c] ** 2) ** 1.5
        assert count == pytest.approx((el == c).sum(), rel=1e-7)


def test_box_cutoff_mass_is_cube_of_trapezoid_sum(oracle_lib):
    # Atom on a voxel centre, r = k sigma an exact multiple of h: the box sum factorises
    # into three 1D sums over |i h| <= k sigma, whose Euler-Maclaurin expansion is
    # sqrt(2 pi) sigma erf(k/sqrt 2) + h e^{-k^2/2} - (h^2/6)(k/sigma) e^{-k^2/2} + O(h^4).
    # An exclusive cutoff would drop the end voxels and miss by ~h e^{-k^2/2}.
    sigma, k, h = 1.0, 3.0, 0.125
    n = 64
    x = [(30 + 0.5) * h] * 3
    G = oracle.voxelize(make([x], [0], (n, n, n), 1, sigma, spacing=(h, h, h),
                             cutoff="box", k=k))[0, 0]
    e = math.exp(-k * k / 2)
    s1 = math.sqrt(2 * math.pi) * sigma * math.erf(k / math.sqrt(2)) + h * e \
        - (h * h / 6) * (k / sigma) * e
    assert G.sum() * h ** 3 == pytest.approx(s1 ** 3, rel=2e-7)


def test_sphere_cutoff_mass_converges_to_truncated_gaussian(oracle_lib):
    # Fine grid limit of the sphere-truncated mass:
    # (2 pi sigma^2)^{3/2} [erf(k/sqrt 2) - sqrt(2/pi) k e^{-k^2/2}]  (~0.9707 at k = 3).
    sigma, k, h = 1.0, 3.0, 0.0625
    n = 112
    rng = np.random.default_rng(3)
    x = 3.5 + rng.uniform(-0.03, 0.03, 3)
    G = oracle.voxelize(make([x], [0], (n, n, n), 1, sigma, spacing=(h, h, h),
                             cutoff="sphere", k=k))[0, 0]
    frac = math.erf(k / math.sqrt(2)) - math.sqrt(2 / math.pi) * k * math.exp(-k * k / 2)
    assert frac == pytest.approx(0.9707, abs=1e-4)
    assert G.sum() * h ** 3 == pytest.approx((2 * math.pi * sigma ** 2) ** 1.5 * frac, rel=1e-3)


def test_sphere_cutoff_is_inclusive_on_lattice_points(oracle_lib):
    # sigma = 0.5, k = 3 -> r = 1.5 = 3 voxels: the nonzero voxels are the integer points
    # with p^2 + q^2 + s^2 <= 9, counted here by enumeration.
    h = 0.5
    x = [(8 + 0.5) * h] * 3
    G = oracle.voxelize(make([x], [0], (17, 17, 17), 1, 0.5, spacing=(h, h, h),
                             cutoff="sphere", k=3.0))[0, 0]
    r = range(-4, 5)
    count = sum(1 for p in r for q in r for s in r if p * p + q * q + s * s <= 9)
    assert count == 123
    assert int((G > 0).sum()) == count
    assert G[8 + 3, 8, 8] == pytest.approx(math.exp(-4.5), rel=1e-15)
    assert G[8 + 3, 8 + 1, 8] == 0.0


# --- P3: translation ------------------------------------------------------------------

def test_one_voxel_translation_shifts_grid_exactly(oracle_lib):
    rng = np.random.default_rng(4)
    x = np.round((6.0 + rng.uniform(0, 3, (5, 3))) * 64) / 64  # dyadic, exact shifts
    el = [0, 1, 0, 1, 1]
    for cutoff in ("sphere", "box", "none"):
        kw = dict(n=(24, 20, 22), C=2, sigma=[0.5, 0.7], cutoff=cutoff)
        G0 = oracle.voxelize(make(x, el, **kw))[0]
        for ax in range(3):
            xs = x.copy()
            xs[:, ax] += 0.5
            G1 = oracle.voxelize(make(xs, el, **kw))[0]
            sl0 = [slice(None)] * 4
            sl1 = [slice(None)] * 4
            sl0[ax + 1] = slice(0, -1)
            sl1[ax + 1] = slice(1, None)
            np.testing.assert_array_equal(G1[tuple(sl1)], G0[tuple(sl0)])


def test_periodic_lattice_translation_and_roll(oracle_lib):
    rng = np.random.default_rng(5)
    n, h = (16, 12, 20), (0.5, 0.625, 0.375)
    L = np.array(n) * np.array(h)
    x = np.round(rng.uniform(0, 1, (6, 3)) * L * 64) / 64
    el = [0, 1, 2, 0, 1, 2]
    kw = dict(n=n, C=3, sigma=[0.5, 0.6, 0.4], spacing=h, cutoff="sphere", periodic=True)
    G0 = oracle.voxelize(make(x, el, **kw))[0]
    G1 = oracle.voxelize(make(x + L * np.array([1, -2, 3]), el, **kw))[0]
    np.testing.assert_allclose(G1, G0, rtol=1e-13, atol=1e-15)
    for ax in range(3):
        xs = x.copy()
        xs[:, ax] += h[ax]
        G2 = oracle.voxelize(make(xs, el, **kw))[0]
        np.testing.assert_allclose(G2, np.roll(G0, 1, axis=ax + 1), rtol=1e-13, atol=1e-15)


def test_minimum_image_equals_sum_over_explicit_images(oracle_lib):
    # With r_c < L/2 the nearest-image grid equals the open-boundary grid of the cell's
    # atoms replicated at all 27 lattice translations (c7 reading of Sec. III-A).
    rng = np.random.default_rng(6)
    n, h = (14, 18, 16), (0.4, 0.35, 0.45)
    L = np.array(n) * np.array(h)
    x = rng.uniform(0, 1, (7, 3)) * L
    x[0] = [0.05, L[1] - 0.1, 0.02]  # near a corner so its images matter
    el = np.array([0, 1, 0, 1, 1, 0, 1])
    sig = [0.5, 0.6]
    assert 3 * max(sig) < L.min() / 2
    Gp = oracle.voxelize(make(x, el, n, 2, sig, spacing=h, cutoff="sphere",
                              periodic=True))[0]
    shifts = np.array([[a, b, c] for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)])
    xi = np.concatenate([x + s * L for s in shifts])
    ei = np.tile(el, len(shifts))
    Go = oracle.voxelize(make(xi, ei, n, 2, sig, spacing=h, cutoff="sphere"))[0]
    np.testing.assert_allclose(Gp, Go, rtol=1e-12, atol=1e-15)


# --- P4: linearity, permutation, channel separation -----------------------------------

def test_linearity_permutation_and_channels(oracle_lib):
    rng = np.random.default_rng(7)
    x = 8.0 + rng.uniform(-3, 3, (8, 3))
    el = np.array([0, 1, 2, 1, 0, 2, 2, 1])
    kw = dict(n=(32, 32, 32), C=3, sigma=[0.4, 0.6, 0.5], cutoff="sphere")
    G = oracle.voxelize(make(x, el, **kw))[0]
    parts = sum(oracle.voxelize(make(x[i:i + 1], el[i:i + 1], **kw))[0] for i in range(8))
    np.testing.assert_allclose(G, parts, rtol=1e-13, atol=1e-16)
    perm = rng.permutation(8)
    Gp = oracle.voxelize(make(x[perm], el[perm], **kw))[0]
    np.testing.assert_allclose(Gp, G, rtol=1e-13, atol=1e-16)
    for c in range(3):
        Gc = oracle.voxelize(make(x[el == c], el[el == c], **kw))[0]
        np.testing.assert_array_equal(Gc[c], G[c])
        assert not np.any(np.delete(Gc, c, axis=0))


# --- P5 / P6: separable = direct, brute force = support box ---------------------------

@pytest.mark.parametrize("cutoff", ["none", "box"])
@pytest.mark.parametrize("periodic", [False, True])
def test_separable_equals_direct(oracle_lib, cutoff, periodic):
    wl = synth.plain_small(n_mol=4)
    p = oracle.Problem(wl.batch, 20, 24, 16, 5, [0.4, 0.5, 0.6, 0.55, 0.45], cutoff, 2.5,
                       periodic)
    np.testing.assert_allclose(oracle.separable(p), oracle.voxelize(p, "brute"),
                               rtol=1e-12, atol=1e-15)


def test_separable_rejects_sphere(oracle_lib):
    wl = synth.plain_small(n_mol=1)
    with pytest.raises(ValueError):
        oracle.separable(oracle.Problem.from_workload(wl))


@pytest.mark.parametrize("cutoff", ["sphere", "box", "none"])
@pytest.mark.parametrize("periodic", [False, True])
def test_brute_force_equals_support_box_bitwise(oracle_lib, cutoff, periodic):
    wl = synth.plain_small(n_mol=6)
    # Odd shapes, atoms partly outside the grid (non-periodic), non-cubic voxels.
    batch = wl.batch
    batch.spacing = np.tile(np.array([0.55, 0.5, 0.6], np.float32), (6, 1))
    p = oracle.Problem(batch, 19, 23, 17, 5, [0.4, 0.5, 0.6, 0.55, 0.45], cutoff, 3.0,
                       periodic)
    np.testing.assert_array_equal(oracle.voxelize(p, "brute"), oracle.voxelize(p, "bbox"))
    W = np.random.default_rng(8).standard_normal(p.shape)
    np.testing.assert_allclose(oracle.gradient(p, W, "brute"), oracle.gradient(p, W, "bbox"),
                               rtol=1e-12, atol=1e-14)


def test_band_split_brackets_the_grid(oracle_lib):
    wl = synth.plain_small(n_mol=3)
    p = oracle.Problem.from_workload(wl)
    G = oracle.voxelize(p)
    g_in, g_band = oracle.voxelize_band(p, 1e-5)
    assert np.all(g_in <= G + 1e-15) and np.all(G <= g_in + g_band + 1e-15)
    # Lattice-point case: sigma = 0.5, r = 1.5 = 3 voxels exactly.  The 30 voxels with
    # p^2 + q^2 + s^2 = 9 (6 axial, 24 of type (2,2,1)) sit exactly on the cutoff surface:
    # all of them land in the band and none counts as strictly inside.
    x = [[8.25, 8.25, 8.25]]
    p2 = make(x, [0], (33, 33, 33), 1, 0.5, cutoff="sphere")
    gi, gb = oracle.voxelize_band(p2, 1e-9)
    assert int((gb > 0).sum()) == 30
    assert np.all(gi[gb > 0] == 0.0)


def test_invalid_element_is_rejected(oracle_lib):
    wl = synth.plain_small(n_mol=2)
    wl.batch.elem[3] = 7
    with pytest.raises(ValueError):
        oracle.voxelize(oracle.Problem.from_workload(wl))


# --- P7: gradient ---------------------------------------------------------------------

def test_gradient_vanishes_at_symmetric_centre(oracle_lib):
    # W = 1, no cutoff, atom at the exact centre of a box of voxels: dL/dx = 0.
    n, h = (20, 20, 20), (0.5, 0.5, 0.5)
    p = make([[5.0, 5.0, 5.0]], [0], n, 1, 0.7, spacing=h)
    g = oracle.gradient(p, np.ones(p.shape))
    assert np.abs(g).max() < 1e-12


def test_gradient_of_first_moment_is_normalisation(oracle_lib):
    # L = sum_v v_x G(v) = x (2 pi s^2)^{3/2} / h^3 up to aliasing, so
    # dL/dx = (2 pi s^2)^{3/2} / (h_x h_y h_z) and dL/dy = dL/dz = 0.  A flipped sign
    # of d or a wrong 1/sigma^2 factor fails this.
    n, h = (40, 40, 40), (0.4, 0.4, 0.4)
    sigma = 0.6
    x = [8.13, 7.94, 8.02]
    p = make([x], [0], n, 1, sigma, spacing=h)
    vx = centres(0.0, h[0], n[0])
    W = np.broadcast_to(vx[:, None, None], n)[None, None]
    g = oracle.gradient(p, W)[0]
    expect = (2 * math.pi * sigma ** 2) ** 1.5 / (h[0] * h[1] * h[2])
    assert g[0] == pytest.approx(expect, rel=1e-7)
    assert abs(g[1]) < 1e-6 * expect and abs(g[2]) < 1e-6 * expect


@pytest.mark.parametrize("cutoff,periodic", [("none", False), ("sphere", False),
                                             ("box", False), ("sphere", True)])
def test_gradient_matches_frozen_support_finite_differences(oracle_lib, cutoff, periodic):
    wl = synth.plain_small(n_mol=3)
    p = oracle.Problem(wl.batch, 24, 24, 24, 5, [0.5, 0.6, 0.4, 0.55, 0.45], cutoff, 3.0,
                       periodic)
    W = np.random.default_rng(9).standard_normal(p.shape)
    g = oracle.gradient(p, W)
    fd = oracle.fd_gradient_frozen(p, W, 1e-4)
    scale = np.abs(g).max()
    np.testing.assert_allclose(fd, g, rtol=0, atol=1e-6 * scale)


def test_gradient_matches_raw_finite_differences_of_forward(oracle_lib):
    # Raw central differences of L(x) = <W, G(x)> computed from the forward oracle alone,
    # for coordinates whose stencil does not move any voxel across the cutoff.
    rng = np.random.default_rng(10)
    n, C = (20, 20, 20), 2
    sig = [0.5, 0.6]
    step = 1e-4
    checked = 0
    for cutoff in ("none", "sphere"):
        x = 5.0 + rng.uniform(-1, 1, (1, 3))
        el = np.array([1])
        p = make(x, el, n, C, sig, cutoff=cutoff)
        W = rng.standard_normal(p.shape)
        g = oracle.gradient(p, W)[0]
        for ax in range(3):
            xp, xm = x.copy(), x.copy()
            xp[0, ax] += step
            xm[0, ax] -= step
            Gp = oracle.voxelize(make(xp, el, n, C, sig, cutoff=cutoff))
            Gm = oracle.voxelize(make(xm, el, n, C, sig, cutoff=cutoff))
            if not np.array_equal(Gp > 0, Gm > 0):
                continue  # a voxel crossed the cutoff: raw FD picks up the jump
            fd = ((W * Gp).sum() - (W * Gm).sum()) / (2 * step)
            assert fd == pytest.approx(g[ax], rel=1e-6, abs=1e-6 * np.abs(g).max())
            checked += 1
    assert checked >= 4


# --- P8: sanity statistic (context only) ------------------------------------------------

def test_nonzero_fraction_is_sparse_like_the_paper(oracle_lib):
    # The paper reports ~1% non-zero cells at 64^3 on drug-like molecules (Sec. VI-B).
    # QM9-shaped molecules with a 3 sigma cutoff on 5 channels are in the same regime.
    wl = synth.qm9_shaped(n_mol=8)
    G = oracle.voxelize(oracle.Problem.from_workload(wl))
    frac = (G > 0).mean()
    assert 0.001 < frac < 0.05
