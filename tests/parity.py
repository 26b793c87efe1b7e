"""Helpers shared by the GPU parity tests: compare CUDA grids and gradients with the oracle.

Tolerances (per molecule, relative to that molecule's largest oracle voxel value):
  f32  1e-5   the stated FP32 bar.  Sources of error: fp32 voxel-centre and displacement
              rounding (~1e-6 A of position, i.e. ~2e-6 of the peak through the slope
              1/(sigma sqrt e) of the Gaussian), the ex2.approx argument/result error
              (~3e-7 relative), and fp32 summation of a handful of terms.
  f16  1e-3   round-to-nearest-even on store adds 2^-11 = 4.9e-4 relative per voxel.
  bf16 5e-3   round-to-nearest-even on store adds 2^-8 = 3.9e-3 relative per voxel.
The stated bar for the half formats is 1e-2; these are tighter.
Voxels within a relative 1e-5 of the cutoff surface (the "band") may legitimately flip
between inside and outside in fp32; each voxel is accepted anywhere in
[G_in - tol, G_in + G_band + tol] and the band population is reported.
"""
from __future__ import annotations

import numpy as np

import oracle

TOL = {"f32": 1e-5, "f16": 1e-3, "bf16": 5e-3}
# Absolute floor: the spacing of the output format near zero.  FP16 cannot represent values
# below its smallest subnormal 2^-24; FP32/BF16 kernels flush results below 2^-126 to zero.
ABS_TOL = {"f32": 2.0 ** -120, "f16": 2.0 ** -24, "bf16": 2.0 ** -120}
SEPARABLE_TOL = 1e-2  # BF16 operands (2 x 2^-9 relative per term) + FP16 store
GRAD_TOL = 1e-4       # GPU gradient vs oracle, relative to max |g| per molecule


def grid_check(G_gpu, prob: "oracle.Problem", rel_tol: float, eps: float = 1e-5,
               abs_tol: float = 2.0 ** -120):
    """Assert the CUDA grids lie within rel_tol * max + abs_tol of the oracle; return error
    stats."""
    G = np.asarray(G_gpu, dtype=np.float64).reshape(prob.shape)
    if prob.c.cutoff == oracle.CUTOFFS["none"]:
        g_in = oracle.voxelize(prob)
        g_band = np.zeros_like(g_in)
    else:
        g_in, g_band = oracle.voxelize_band(prob, eps)
    ref = g_in + g_band
    worst_abs, worst_l2, band_voxels = 0.0, 0.0, int((g_band > 0).sum())
    for b in range(prob.shape[0]):
        m = float(np.abs(ref[b]).max())
        if m == 0.0:
            assert np.all(G[b] == 0.0), f"molecule {b}: oracle grid is zero, CUDA is not"
            continue
        tol = rel_tol * m + abs_tol
        lo = g_in[b] - tol
        hi = g_in[b] + g_band[b] + tol
        bad = (G[b] < lo) | (G[b] > hi) | ~np.isfinite(G[b])
        if bad.any():
            idx = np.argwhere(bad)[0]
            raise AssertionError(
                f"molecule {b}: {int(bad.sum())} voxels outside tolerance {rel_tol} "
                f"(first at {tuple(idx)}: cuda {G[b][tuple(idx)]!r}, oracle in "
                f"{g_in[b][tuple(idx)]!r} band {g_band[b][tuple(idx)]!r}, max {m})")
        # Error outside the cutoff-band ambiguity: distance from [G_in, G_in + G_band].
        err = np.maximum(np.maximum(g_in[b] - G[b], G[b] - (g_in[b] + g_band[b])), 0.0)
        worst_abs = max(worst_abs, float(err.max()) / m)
        worst_l2 = max(worst_l2, float(np.linalg.norm(err) / np.linalg.norm(ref[b])))
    return {"max_abs_rel": worst_abs, "rel_l2": worst_l2, "band_voxels": band_voxels}


def grad_check(g_gpu, g_ref, mol_off, rel_tol=GRAD_TOL):
    """Per molecule: max |g_gpu - g_ref| <= rel_tol * max |g_ref| (all components)."""
    g_gpu = np.asarray(g_gpu, np.float64)
    g_ref = np.asarray(g_ref, np.float64)
    worst = 0.0
    for b in range(len(mol_off) - 1):
        s = slice(int(mol_off[b]), int(mol_off[b + 1]))
        if s.stop == s.start:
            continue
        m = float(np.abs(g_ref[s]).max())
        d = float(np.abs(g_gpu[s] - g_ref[s]).max())
        if m == 0.0:
            assert d == 0.0
            continue
        assert d <= rel_tol * m, f"molecule {b}: gradient error {d / m:.3e} > {rel_tol}"
        worst = max(worst, d / m)
    return worst
