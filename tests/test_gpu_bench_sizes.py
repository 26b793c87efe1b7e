"""GPU parity at the benchmark's full batch sizes, in the launch configuration the benchmark
times: the same autotuner call (same dtype, path and output buffer) followed by the same
forward call, then a seeded sample of the grids checked against the FP64 oracle.

Batches: the precision form (4096 x 5 x 64^3, no cutoff) as the FP16 form (BF16 tcgen05
separable contraction) and as the plain FP32 direct path, the 512-cell crystal batch
(periodic, Zipf elements, 20-500 atoms, FP16), the 16384-molecule single-channel pipeline
batch (erf form, box cutoff, BF16) and the 512 weighted triclinic cells.  The tuner's choice
of chunk size, order, scatter or gather mode, and the separable kernel's resident K slots
all depend on the batch, so the smaller parity cases elsewhere do not reach these branches.
The autotuner's reference candidate (the default launch, which every other candidate is
compared against) is checked against the oracle on the same sample.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.parity import ABS_TOL, SEPARABLE_TOL, TOL, grid_check

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2211_08506_gb300 as pkg
    pkg.build()
    from paper_2211_08506_gb300 import api
    return api


def tuned_and_sampled(pg, wl, dtype, path, n_sample, seed, tol, reference=False):
    """Autotune and run as the benchmark does; check a seeded sample against the oracle.
    With reference=True also run the tuner's reference candidate (the default launch of
    the chosen path) and check it on the same sample."""
    db = pg.DeviceBatch.from_numpy(wl.batch)
    grid = pg.Grid.from_workload(wl)
    out = torch.empty(grid.out_shape(wl.batch.n_mol), dtype=pg.DTYPES[dtype][1], device="cuda")
    tuning = pg.autotune(db, grid, dtype=dtype, path=path, out=out)
    pg.voxelize(db, grid, dtype=dtype, path=path, out=out)
    assert pg.sync_status() == 0
    idx = np.sort(np.random.default_rng(seed).choice(wl.batch.n_mol, n_sample, replace=False))
    sel = torch.as_tensor(idx, device="cuda")
    prob = oracle.Problem.from_workload(wl, batch=wl.batch.subset(idx))
    stats = grid_check(out[sel].float().cpu().numpy(), prob, tol, abs_tol=ABS_TOL[dtype])
    if reference:
        pg.voxelize_tuned(db, grid, {"path": tuning["path"]}, dtype=dtype, out=out)
        assert pg.sync_status() == 0
        grid_check(out[sel].float().cpu().numpy(), prob, tol, abs_tol=ABS_TOL[dtype])
    del out
    torch.cuda.empty_cache()
    return tuning, stats


def test_precision_form_fp16_form_tuned_full_batch(pg):
    wl = synth.precision_form()
    tuning, stats = tuned_and_sampled(pg, wl, "f16", "separable", 8, 31, SEPARABLE_TOL,
                                      reference=True)
    assert tuning["path"] == 2
    assert stats["max_abs_rel"] < SEPARABLE_TOL


def test_precision_form_fp32_direct_tuned_full_batch(pg):
    # The denominator of the FP16 form's speedup: 21.5 GB of FP32 grids, no cutoff.
    wl = synth.precision_form()
    tuning, stats = tuned_and_sampled(pg, wl, "f32", "direct", 8, 32, TOL["f32"],
                                      reference=True)
    assert tuning["path"] == 1
    assert stats["max_abs_rel"] < TOL["f32"]


def test_crystal_shaped_tuned_full_batch(pg):
    wl = synth.crystal_shaped()
    assert wl.batch.n_mol == 512
    tuned_and_sampled(pg, wl, "f16", "auto", 16, 33, TOL["f16"], reference=True)


def test_crystal_triclinic_tuned_full_batch(pg):
    wl = synth.crystal_triclinic()
    assert wl.batch.n_mol == 512
    tuned_and_sampled(pg, wl, "f16", "auto", 12, 34, TOL["f16"], reference=True)


def test_pipeline_single_channel_tuned_full_batch(pg):
    wl = synth.pipeline_single_channel()
    assert wl.batch.n_mol == 16384
    tuning, _ = tuned_and_sampled(pg, wl, "bf16", "auto", 24, 35, SEPARABLE_TOL,
                                  reference=True)


def test_precision_form_integral_fp32_direct_tuned_full_batch(pg):
    # The erf form's FP32 reference path (per-chunk factor tables) on the full batch.
    wl = synth.precision_form_integral()
    tuning, stats = tuned_and_sampled(pg, wl, "f32", "direct", 8, 36, TOL["f32"],
                                      reference=True)
    assert stats["max_abs_rel"] < TOL["f32"]
