"""Seeded synthetic batches shaped like the workloads of the ParticleGrid paper.

The paper measures on MOSES molecules with RDKit conformers (Sec. VI-D) and trains on
PCQM4Mv2 (Sec. VII); neither dataset is available here, so these generators stand in for
them with the shapes, atom-count distributions and element mixes of small organic
molecules (QM9-like) and of periodic crystals.

This module holds none of the voxelization arithmetic: it only samples geometry
(random walks, random crystal cells), draws element ids, and packs the result into the
CSR layout that both the CUDA path and the CPU oracle consume.  Every draw comes from
``numpy.random.default_rng`` seeded with ``SEED_BASE + workload index`` (optionally mixed
with a shard index), so a batch is reproducible on any machine.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

SEED_BASE = 20221115

# Channel order: one channel per element (Sec. III-A); H, C, N, O, F for molecules.
MOLECULE_ELEMENTS = ("H", "C", "N", "O", "F")

CUTOFF_SPHERE = "sphere"
CUTOFF_NONE = "none"
CUTOFF_BOX = "box"


@dataclass
class Batch:
    """CSR-packed atoms of B molecules (or cells).

    coords  float32 [N, 3]  Cartesian positions (Angstrom)
    elem    int32   [N]     channel id of each atom
    mol_off int32   [B+1]   atoms of molecule b are rows mol_off[b] .. mol_off[b+1]-1
    origin  float32 [B, 3]  lower corner of molecule b's grid box
    spacing float32 [B, 3]  voxel edge lengths of molecule b's grid
    weight  float32 [N]     optional per-atom weights (weighted grids); None means ones
    cell    float32 [B,3,3] optional box edges a, b, c (rows) along the grid's x, y, z
                            axes, replacing the axis-aligned box of `spacing`; None if unused
    """

    coords: np.ndarray
    elem: np.ndarray
    mol_off: np.ndarray
    origin: np.ndarray
    spacing: np.ndarray
    info: dict = field(default_factory=dict)
    weight: np.ndarray | None = None
    cell: np.ndarray | None = None

    @property
    def n_mol(self) -> int:
        return int(self.mol_off.shape[0] - 1)

    @property
    def n_atoms(self) -> int:
        return int(self.coords.shape[0])

    def atoms_of(self, b: int) -> slice:
        return slice(int(self.mol_off[b]), int(self.mol_off[b + 1]))

    def subset(self, idx) -> "Batch":
        """Batch made of molecules ``idx`` (in that order)."""
        idx = [int(i) for i in idx]
        parts = [self.atoms_of(b) for b in idx]
        counts = [p.stop - p.start for p in parts]
        off = np.zeros(len(idx) + 1, np.int32)
        off[1:] = np.cumsum(counts)
        cat = lambda a: (np.concatenate([a[p] for p in parts]) if parts else a[:0])
        return Batch(
            coords=np.ascontiguousarray(cat(self.coords), dtype=np.float32).reshape(-1, 3),
            elem=np.ascontiguousarray(cat(self.elem), dtype=np.int32),
            mol_off=off,
            origin=np.ascontiguousarray(self.origin[idx], dtype=np.float32).reshape(-1, 3),
            spacing=np.ascontiguousarray(self.spacing[idx], dtype=np.float32).reshape(-1, 3),
            weight=(None if self.weight is None else
                    np.ascontiguousarray(cat(self.weight), dtype=np.float32)),
            cell=(None if self.cell is None else
                  np.ascontiguousarray(self.cell[idx], dtype=np.float32).reshape(-1, 3, 3)),
        )


@dataclass
class Workload:
    """A batch plus the grid description it is voxelized on."""

    name: str
    batch: Batch
    nx: int
    ny: int
    nz: int
    n_channels: int
    sigma: np.ndarray          # float32 [C], Gaussian width (standard deviation, Angstrom)
    cutoff: str                # "sphere" | "none" | "box"
    cutoff_k: float            # r_c = cutoff_k * sigma_c
    periodic: bool
    out_dtype: str             # "f32" | "f16" | "bf16"
    description: str = ""
    form: str = "point"        # "point" (sampled at voxel centres) | "integral" (erf form)

    @property
    def voxels_per_grid(self) -> int:
        return self.n_channels * self.nx * self.ny * self.nz

    def out_bytes(self, dtype: str | None = None) -> int:
        size = {"f32": 4, "f16": 2, "bf16": 2}[dtype or self.out_dtype]
        return self.batch.n_mol * self.voxels_per_grid * size


def _rng(index: int, shard: int | None = None) -> np.random.Generator:
    seed = SEED_BASE + index
    return np.random.default_rng(seed if shard is None else [seed, shard])


def _unit_vectors(rng: np.random.Generator, n: int) -> np.ndarray:
    v = rng.standard_normal((n, 3))
    return v / np.sqrt((v * v).sum(axis=1, keepdims=True))


def random_walk(rng: np.random.Generator, n: int, step_lo=1.0, step_hi=1.5) -> np.ndarray:
    """3D random walk of n points; step length U[step_lo, step_hi], direction uniform on the
    sphere, no self-avoidance."""
    pos = np.zeros((n, 3))
    if n > 1:
        steps = rng.uniform(step_lo, step_hi, size=(n - 1, 1)) * _unit_vectors(rng, n - 1)
        pos[1:] = np.cumsum(steps, axis=0)
    return pos


def _pack(coord_list, elem_list, origins, spacings, info=None) -> Batch:
    counts = [len(e) for e in elem_list]
    off = np.zeros(len(counts) + 1, np.int64)
    off[1:] = np.cumsum(counts)
    if off[-1] >= 2**31:
        raise ValueError("batch too large for int32 offsets")
    coords = (np.concatenate(coord_list) if coord_list else np.zeros((0, 3)))
    elem = (np.concatenate(elem_list) if elem_list else np.zeros(0))
    return Batch(
        coords=np.ascontiguousarray(coords, dtype=np.float32).reshape(-1, 3),
        elem=np.ascontiguousarray(elem, dtype=np.int32),
        mol_off=off.astype(np.int32),
        origin=np.ascontiguousarray(origins, dtype=np.float32).reshape(-1, 3),
        spacing=np.ascontiguousarray(spacings, dtype=np.float32).reshape(-1, 3),
        info=info or {},
    )


def _centred_box(pos: np.ndarray, n: tuple, h: float):
    """Origin that puts the centroid of pos at the centre of an n*h box."""
    centroid = pos.mean(axis=0)
    return centroid - 0.5 * np.asarray(n, float) * h


def plain_small(shard: int | None = None, n_mol: int = 16) -> Workload:
    """Plain method, small: 16 molecules of U{5..20} atoms, elements uniform over
    H,C,N,O,F, random-walk geometry (bond 1.0-1.5 A) centred in a 32^3 grid at 0.5 A,
    sigma 0.5 A for every element, spherical cutoff 3 sigma, FP32 output."""
    rng = _rng(0, shard)
    n = (32, 32, 32)
    h = 0.5
    coords, elems, origins = [], [], []
    for _ in range(n_mol):
        na = int(rng.integers(5, 21))
        pos = random_walk(rng, na)
        coords.append(pos)
        elems.append(rng.integers(0, 5, size=na))
        origins.append(_centred_box(pos, n, h))
    batch = _pack(coords, elems, origins, np.full((n_mol, 3), h))
    return Workload("plain_small", batch, *n, 5, np.full(5, 0.5, np.float32),
                    CUTOFF_SPHERE, 3.0, False, "f32",
                    "16 random-walk molecules, 5-20 atoms, 5ch 32^3 @0.5A, sigma 0.5, sphere 3sigma")


def _qm9_molecule(rng: np.random.Generator):
    """QM9-like composition: k ~ U{1..9} heavy atoms from {C,N,O,F}, H count
    U{max(0,3-k) .. 2k+2}, total capped at 29; atoms placed on one random walk in a
    random order."""
    k = int(rng.integers(1, 10))
    n_h = int(rng.integers(max(0, 3 - k), 2 * k + 3))
    n_h = min(n_h, 29 - k)
    heavy = rng.integers(1, 5, size=k)
    el = np.concatenate([heavy, np.zeros(n_h, np.int64)])
    el = el[rng.permutation(el.shape[0])]
    pos = random_walk(rng, el.shape[0])
    return pos, el


QM9_SIGMA = np.array([0.4, 0.6, 0.6, 0.6, 0.6], np.float32)


def qm9_batch(index: int, n_mol: int, n: tuple, h: float, shard: int | None = None) -> Batch:
    rng = _rng(index, shard)
    coords, elems, origins = [], [], []
    for _ in range(n_mol):
        pos, el = _qm9_molecule(rng)
        coords.append(pos)
        elems.append(el)
        origins.append(_centred_box(pos, n, h))
    return _pack(coords, elems, origins, np.full((n_mol, 3), h))


def qm9_shaped(shard: int | None = None, n_mol: int = 4096) -> Workload:
    """QM9-shaped batch: 4096 molecules, 3-29 atoms, 5ch 32^3 @0.5 A, per-element sigma
    {H .4, C/N/O/F .6}, spherical cutoff 3 sigma, FP32 direct path."""
    n = (32, 32, 32)
    batch = qm9_batch(1, n_mol, n, 0.5, shard)
    return Workload("qm9_shaped", batch, *n, 5, QM9_SIGMA.copy(), CUTOFF_SPHERE, 3.0,
                    False, "f32",
                    f"{n_mol} QM9-shaped molecules (3-29 atoms), 5ch 32^3 @0.5A, sigma H.4/CNOF.6, sphere 3sigma")


def precision_form(shard: int | None = None, n_mol: int = 4096) -> Workload:
    """Precision form: QM9-shaped molecules on a 64^3 grid at 0.25 A with no cutoff, so
    the separable contraction is dense; FP16 output."""
    n = (64, 64, 64)
    batch = qm9_batch(2, n_mol, n, 0.25, shard)
    return Workload("precision_form", batch, *n, 5, QM9_SIGMA.copy(), CUTOFF_NONE, 3.0,
                    False, "f16",
                    f"{n_mol} QM9-shaped molecules, 5ch 64^3 @0.25A, no cutoff")


def precision_form_integral(shard: int | None = None, n_mol: int = 4096) -> Workload:
    """The precision-form batch with the voxel-integrated (erf) voxel function of Sec. III-A:
    the same molecules and grid, each voxel holding the Gaussian's integral over it."""
    wl = precision_form(shard, n_mol)
    wl.name = "precision_form_integral"
    wl.form = "integral"
    wl.description = f"{n_mol} QM9-shaped molecules, 5ch 64^3 @0.25A, no cutoff, erf voxel integrals"
    return wl


ZIPF_EXPONENT = 1.2
CRYSTAL_ELEMENTS = 10
JAMMING_SKIP = 0.32


def crystal_cell(rng: np.random.Generator, n_atoms: int, edge_lo=5.0, edge_hi=15.0,
                 min_sep=1.2, max_tries=1000):
    """Random orthorhombic cell with n_atoms atoms placed by random sequential addition.

    Fractional coordinates are uniform; a proposal closer than min_sep (minimum image)
    to a placed atom is rejected.  After max_tries consecutive rejections for one atom
    the cell edges are redrawn and placement restarts with the same atom count.
    Returns (edges[3], frac[n,3], redraws)."""
    redraws = 0
    v_excl = math.pi / 6.0 * min_sep ** 3
    while True:
        edges = rng.uniform(edge_lo, edge_hi, size=3)
        # Above this packing fraction random sequential addition practically never
        # places every atom within max_tries, so the cell is redrawn at once.
        if n_atoms * v_excl / float(np.prod(edges)) > JAMMING_SKIP:
            redraws += 1
            continue
        placed = np.zeros((n_atoms, 3))
        ok = True
        for i in range(n_atoms):
            tries = 0
            done = False
            while tries < max_tries:
                # Small proposal blocks while most proposals succeed, larger ones after.
                m = min(4 if tries == 0 else 64, max_tries - tries)
                cand = rng.uniform(0.0, 1.0, size=(m, 3))
                if i == 0:
                    placed[0] = cand[0]
                    done = True
                    break
                diff = cand[:, None, :] - placed[None, :i, :]
                diff -= np.round(diff)
                dist2 = ((diff * edges) ** 2).sum(axis=2).min(axis=1)
                good = np.nonzero(dist2 >= min_sep * min_sep)[0]
                if good.size:
                    placed[i] = cand[good[0]]
                    done = True
                    break
                tries += m
            if not done:
                ok = False
                break
        if ok:
            return edges, placed, redraws
        redraws += 1


def crystal_shaped(shard: int | None = None, n_cells: int = 512, grid: int = 48) -> Workload:
    """Crystal-shaped uneven batch: orthorhombic cells with edges U[5,15] A, atom counts
    log-uniform in 20..500, 10 element channels with Zipf(1.2) frequencies, 1.2 A minimum
    separation, periodic minimum image, sigma 0.5 A, spherical cutoff 3 sigma, 48^3 grid
    spanning each cell, FP16 output."""
    rng = _rng(3, shard)
    p = (np.arange(1, CRYSTAL_ELEMENTS + 1, dtype=float)) ** (-ZIPF_EXPONENT)
    p /= p.sum()
    coords, elems, origins, spacings = [], [], [], []
    redraws = 0
    for _ in range(n_cells):
        na = int(round(math.exp(rng.uniform(math.log(20.0), math.log(500.0)))))
        edges, frac, r = crystal_cell(rng, na)
        redraws += r
        h = (edges / grid).astype(np.float32)
        cell = h.astype(np.float64) * grid
        coords.append(frac * cell)
        elems.append(rng.choice(CRYSTAL_ELEMENTS, size=na, p=p))
        origins.append(np.zeros(3))
        spacings.append(h)
    batch = _pack(coords, elems, origins, spacings, info={"cell_redraws": redraws})
    return Workload("crystal_shaped", batch, grid, grid, grid, CRYSTAL_ELEMENTS,
                    np.full(CRYSTAL_ELEMENTS, 0.5, np.float32), CUTOFF_SPHERE, 3.0, True,
                    "f16",
                    f"{n_cells} periodic orthorhombic cells 5-15A, 20-500 atoms, 10ch Zipf1.2, 48^3, sigma .5, sphere 3sigma")


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation (QR of a Gaussian matrix, signs fixed, det +1)."""
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def triclinic_cell(rng: np.random.Generator, n_atoms: int, edge_lo=5.0, edge_hi=15.0,
                   angle_lo=60.0, angle_hi=120.0, min_width=3.2, min_sep=1.2,
                   max_tries=1000):
    """Random triclinic cell with n_atoms atoms placed by random sequential addition.

    Edge lengths a, b, c are U[edge_lo, edge_hi] A and the angles alpha, beta, gamma
    U[angle_lo, angle_hi] degrees.  Cells that are not valid, or whose distance between
    opposite faces is below min_width on some axis, are redrawn.  The cell is then turned
    by a uniform random rotation.  Fractional coordinates are uniform; a proposal closer
    than min_sep to a placed atom is rejected, and after max_tries rejections for one atom
    the cell is redrawn.  Since every width exceeds 2 min_sep, only the image at the rounded
    fractional difference can come that close.
    Returns (M [3, 3] with rows a, b, c, frac [n, 3], redraws)."""
    redraws = 0
    v_excl = math.pi / 6.0 * min_sep ** 3
    assert min_width > 2.0 * min_sep
    while True:
        a, b, c = rng.uniform(edge_lo, edge_hi, size=3)
        al, be, ga = np.radians(rng.uniform(angle_lo, angle_hi, size=3))
        cy = (math.cos(al) - math.cos(be) * math.cos(ga)) / math.sin(ga)
        cz2 = 1.0 - math.cos(be) ** 2 - cy ** 2
        if cz2 <= 0.0:
            redraws += 1
            continue
        M = np.array([[a, 0.0, 0.0],
                      [b * math.cos(ga), b * math.sin(ga), 0.0],
                      [c * math.cos(be), c * cy, c * math.sqrt(cz2)]])
        width = 1.0 / np.linalg.norm(np.linalg.inv(M), axis=0)
        vol = abs(float(np.linalg.det(M)))
        if width.min() < min_width or n_atoms * v_excl / vol > JAMMING_SKIP:
            redraws += 1
            continue
        M = M @ _random_rotation(rng).T
        placed = np.zeros((n_atoms, 3))
        ok = True
        for i in range(n_atoms):
            tries = 0
            done = False
            while tries < max_tries:
                m = min(4 if tries == 0 else 64, max_tries - tries)
                cand = rng.uniform(0.0, 1.0, size=(m, 3))
                if i == 0:
                    placed[0] = cand[0]
                    done = True
                    break
                diff = cand[:, None, :] - placed[None, :i, :]
                diff -= np.round(diff)
                dist2 = ((diff @ M) ** 2).sum(axis=2).min(axis=1)
                good = np.nonzero(dist2 >= min_sep * min_sep)[0]
                if good.size:
                    placed[i] = cand[good[0]]
                    done = True
                    break
                tries += m
            if not done:
                ok = False
                break
        if ok:
            return M, placed, redraws
        redraws += 1


def crystal_triclinic(shard: int | None = None, n_cells: int = 512, grid: int = 48) -> Workload:
    """Weighted triclinic crystal batch: cells with edges U[5,15] A, angles U[60,120] deg,
    every face-to-face width at least 3.2 A, random orientation; atom counts log-uniform in
    20..500; 10 element channels with Zipf(1.2) frequencies; 1.2 A minimum separation;
    per-atom weights U[0.5,1.5]; periodic nearest image; sigma 0.5 A; spherical cutoff
    3 sigma; a 48^3 grid along the cell edges; FP16 output."""
    rng = _rng(7, shard)
    p = (np.arange(1, CRYSTAL_ELEMENTS + 1, dtype=float)) ** (-ZIPF_EXPONENT)
    p /= p.sum()
    coords, elems, origins, spacings, cells, weights = [], [], [], [], [], []
    redraws = 0
    for _ in range(n_cells):
        na = int(round(math.exp(rng.uniform(math.log(20.0), math.log(500.0)))))
        M, frac, r = triclinic_cell(rng, na)
        redraws += r
        M32 = M.astype(np.float32)
        cells.append(M32)
        coords.append(frac @ M32.astype(np.float64))
        elems.append(rng.choice(CRYSTAL_ELEMENTS, size=na, p=p))
        weights.append(rng.uniform(0.5, 1.5, size=na))
        origins.append(np.zeros(3))
        spacings.append(np.linalg.norm(M32, axis=1) / grid)
    batch = _pack(coords, elems, origins, spacings, info={"cell_redraws": redraws})
    batch.cell = np.ascontiguousarray(np.stack(cells), dtype=np.float32)
    batch.weight = np.ascontiguousarray(np.concatenate(weights), dtype=np.float32)
    return Workload("crystal_triclinic", batch, grid, grid, grid, CRYSTAL_ELEMENTS,
                    np.full(CRYSTAL_ELEMENTS, 0.5, np.float32), CUTOFF_SPHERE, 3.0, True,
                    "f16",
                    f"{n_cells} weighted periodic triclinic cells 5-15A 60-120deg, 20-500 atoms, "
                    "10ch Zipf1.2, 48^3, sigma .5, sphere 3sigma")


def differentiation(shard: int | None = None, n_mol: int = 1024) -> Workload:
    """Differentiation workload: 1024 QM9-shaped molecules on 5ch 32^3 @0.5 A, per-element
    sigma, spherical cutoff 3 sigma; the loss is <W, G> with W from ``loss_weights``."""
    n = (32, 32, 32)
    batch = qm9_batch(4, n_mol, n, 0.5, shard)
    return Workload("differentiation", batch, *n, 5, QM9_SIGMA.copy(), CUTOFF_SPHERE, 3.0,
                    False, "f32",
                    f"{n_mol} QM9-shaped molecules, 5ch 32^3 @0.5A, loss <W,G>, W~N(0,1)")


def loss_weights(wl: Workload, molecules=None, shard: int | None = None) -> np.ndarray:
    """Seeded N(0,1) float32 weights W with the grid's shape, one independent stream per
    molecule so any subset can be regenerated on its own.  Returns [len(molecules), C,
    nx, ny, nz]."""
    if molecules is None:
        molecules = range(wl.batch.n_mol)
    shape = (wl.n_channels, wl.nx, wl.ny, wl.nz)
    base = SEED_BASE + 4 if shard is None else SEED_BASE + 4 + 1000003 * (shard + 1)
    out = np.empty((len(molecules),) + shape, np.float32)
    for i, b in enumerate(molecules):
        out[i] = np.random.default_rng([base, int(b)]).standard_normal(shape, dtype=np.float32)
    return out


def _pcqm_molecule(rng: np.random.Generator):
    """PCQM4Mv2-like size: k ~ U{3..25} heavy atoms and U{k/2 .. k+4} hydrogens, at most 51
    atoms, placed on one random walk (bond 1.0-1.5 A)."""
    k = int(rng.integers(3, 26))
    n_h = int(rng.integers(k // 2, k + 5))
    n = min(k + n_h, 51)
    return random_walk(rng, n)


def pipeline_single_channel(shard: int | None = None, n_mol: int = 16384) -> Workload:
    """The training-input use case of Sec. VII: every atom in one channel, a 32^3 grid whose
    spatial resolution adapts to each molecule's bounding box, sigma 0.4, generated on the
    fly for a 3D CNN (training batches of 256; one step here covers 64 of them so the output
    exceeds L2).  The voxel function is the paper's erf integral, with a box cutoff of
    3 sigma, stored as BF16."""
    rng = _rng(6, shard)
    n = (32, 32, 32)
    sigma = 0.4
    coords, elems, origins, spacings = [], [], [], []
    for _ in range(n_mol):
        pos = _pcqm_molecule(rng)
        lo, hi = pos.min(axis=0), pos.max(axis=0)
        extent = float((hi - lo).max()) + 2 * 3.0 * sigma   # the box keeps every support
        h = extent / n[0]
        coords.append(pos)
        elems.append(np.zeros(pos.shape[0], np.int64))
        origins.append(0.5 * (lo + hi) - 0.5 * n[0] * h)
        spacings.append((h, h, h))
    batch = _pack(coords, elems, origins, spacings)
    return Workload("pipeline_single_channel", batch, *n, 1, np.full(1, sigma, np.float32),
                    CUTOFF_BOX, 3.0, False, "bf16",
                    f"{n_mol} PCQM4Mv2-sized molecules (4-51 atoms), 1 channel, 32^3 adaptive box, "
                    f"sigma 0.4, erf voxel integrals, box 3 sigma, BF16",
                    form="integral")


REFINE_ITERS = 50      # descent steps per grid reversal
REFINE_LR = 0.02       # step size (A^2 per unit of the squared grid error's gradient)
REFINE_NOISE = 0.1     # A, standard deviation of the start's displacement from the truth


def refinement(shard: int | None = None, n_mol: int = 1024) -> Workload:
    """Grid reversal (Sec. IV-A): 1024 QM9-shaped molecules on 5ch 32^3 @0.5 A with
    per-element sigma and a spherical 3 sigma cutoff.  The grid to reverse is that of the
    true coordinates; descent starts from them displaced by N(0, 0.1 A) per coordinate
    (``refinement_start``) and takes REFINE_ITERS steps of REFINE_LR."""
    n = (32, 32, 32)
    batch = qm9_batch(5, n_mol, n, 0.5, shard)
    return Workload("refinement", batch, *n, 5, QM9_SIGMA.copy(), CUTOFF_SPHERE, 3.0, False,
                    "f32",
                    f"{n_mol} QM9-shaped molecules, 5ch 32^3 @0.5A, start = truth + N(0, "
                    f"{REFINE_NOISE} A), {REFINE_ITERS} descent steps of {REFINE_LR}")


def refinement_start(wl: Workload, shard: int | None = None) -> np.ndarray:
    """Seeded starting coordinates for grid reversal: the true coordinates plus N(0,
    REFINE_NOISE) per coordinate (float32 [N, 3])."""
    rng = np.random.default_rng([SEED_BASE + 5, 1] if shard is None
                                else [SEED_BASE + 5, 1, shard])
    noise = rng.normal(0.0, REFINE_NOISE, wl.batch.coords.shape)
    return (wl.batch.coords.astype(np.float64) + noise).astype(np.float32)


WORKLOADS = {
    "plain_small": plain_small,
    "qm9_shaped": qm9_shaped,
    "precision_form": precision_form,
    "precision_form_integral": precision_form_integral,
    "crystal_shaped": crystal_shaped,
    "differentiation": differentiation,
    "refinement": refinement,
    "pipeline_single_channel": pipeline_single_channel,
    "crystal_triclinic": crystal_triclinic,
}


def workload(name: str, **kw) -> Workload:
    return WORKLOADS[name](**kw)


def single_atom_batch(positions, elems, origin, spacing) -> Batch:
    """One molecule per row of ``positions`` (each a list of atoms) - for small pins."""
    coords, el, orig, sp = [], [], [], []
    for pos, e in zip(positions, elems):
        coords.append(np.asarray(pos, float).reshape(-1, 3))
        el.append(np.asarray(e, np.int64).reshape(-1))
        orig.append(origin)
        sp.append(spacing)
    return _pack(coords, el, orig, sp)
