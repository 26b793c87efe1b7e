"""Host logic of bench.py, on the CPU: the error stated with every result, the clock record
of a timed region, the gating of profiled DRAM traffic by kernel source, and the seeded
sample of molecules.  No GPU and no CUDA extension are needed."""
import json
import os

import numpy as np
import pytest

import bench
import oracle
import synth


def test_error_of_the_oracle_itself_is_zero_and_a_planted_error_is_reported():
    wl = synth.plain_small(n_mol=3)
    idx = np.arange(3)
    prob = oracle.Problem.from_workload(wl)
    g_in, g_band = oracle.voxelize_band(prob, 1e-5, 1)
    G = g_in.copy()
    e = bench.oracle_grid_error(wl, idx, G, "f32", 1, "direct")
    assert e["max_abs_rel"] == 0.0 and e["rel_l2"] == 0.0 and e["pass"]
    assert e["grids"] == 3 and e["bar"] == 1e-5
    # One voxel off by 1e-3 of its grid's maximum: reported as such, and above the FP32 bar.
    b = 1
    m = float(np.abs(g_in[b] + g_band[b]).max())
    pos = np.unravel_index(int(np.argmax(g_in[b])), g_in[b].shape)
    G[b][pos] += 1e-3 * m
    e = bench.oracle_grid_error(wl, idx, G, "f32", 1, "direct")
    assert e["max_abs_rel"] == pytest.approx(1e-3, rel=1e-6)
    assert not e["pass"]
    # The same error passes the FP16 bar, and the separable path is held to 1e-2.
    assert bench.oracle_grid_error(wl, idx, G, "f16", 1, "direct")["pass"]
    assert bench.oracle_grid_error(wl, idx, G, "f32", 1, "separable")["bar"] == 1e-2
    # A non-finite grid can never pass.
    G[0].flat[0] = np.nan
    e = bench.oracle_grid_error(wl, idx, G, "f32", 1, "direct")
    assert e["max_abs_rel"] == float("inf") and not e["pass"]


def test_clock_summary_uses_the_samples_inside_each_timed_region():
    s = bench.ClockSampler(0)
    s.max_mhz = 2070.0
    s.source = "test"
    cap = frozenset({"sw_power_cap"})
    hot = frozenset({"hw_thermal_slowdown"})
    s.rows = [(0.5, 1000.0, hot, 300.0), (1.1, 2070.0, frozenset(), 500.0),
              (1.2, 2040.0, cap, 700.0), (1.3, 2070.0, frozenset(), 600.0),
              (5.0, 900.0, hot, 200.0)]
    s.regions = {"headline": [1.0, 2.0], "short": [4.9, 4.901]}
    h = s.summary("headline")
    assert h["sm_mhz"] == 2070.0 and h["sm_max_mhz"] == 2070.0
    assert h["reasons"] == ["sw_power_cap"]      # samples outside the region do not count
    assert h["samples_in_timed_region"] == 3 and h["power_w_max"] == 700.0
    # A region shorter than the sampling period reports no sample inside it but takes the
    # nearest samples around it for the clock and the reasons.
    short = s.summary("short")
    assert short["samples_in_timed_region"] == 0
    assert short["reasons"] == ["hw_thermal_slowdown"]
    assert bench.ClockSampler(0).summary()["reasons"] == ["no clock samples"]


def test_profiled_traffic_is_reported_only_for_the_captured_kernel_source(tmp_path,
                                                                           monkeypatch):
    csrc = tmp_path / "paper_2211_08506_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in ("direct_kernel.cuh", "pg_internal.h"):
        (csrc / f).write_text("// kernel source " + f + "\n")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    sha = bench.kernel_source_sha("direct")
    entry = {"kernel_source_sha": sha, "dram_bytes_per_launch": 1234.0, "scaled_from": "x"}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"direct:qm9_shaped": entry}))
    assert bench.profiled_traffic("qm9_shaped", "direct") == 1234.0
    assert bench.profiled_traffic("crystal_shaped", "direct") is None
    # Any change to the kernel's sources (here a header it includes) voids the entry.
    (csrc / "pg_internal.h").write_text("// changed\n")
    assert bench.kernel_source_sha("direct") != sha
    assert bench.profiled_traffic("qm9_shaped", "direct") is None


def test_committed_traffic_entries_are_well_formed():
    path = os.path.join(os.path.dirname(bench.__file__), "profiles", "traffic.json")
    entries = json.load(open(path))
    assert entries
    for key, e in entries.items():
        kernel, workload = key.split(":")
        assert kernel in bench.KERNEL_SOURCES
        assert workload in synth.WORKLOADS
        assert len(e["kernel_source_sha"]) == 16
        assert e["dram_bytes_per_launch"] > 0
        assert e["scaled_from"].split(":")[0].endswith(".md")
        assert os.path.exists(os.path.join(os.path.dirname(path), e["scaled_from"].split(":")[0]))


def test_sample_indices_are_seeded_sorted_distinct_and_capped():
    a = bench.sample_indices(100, 16, 7)
    assert np.array_equal(a, bench.sample_indices(100, 16, 7))
    assert len(set(a.tolist())) == 16 and np.all(np.diff(a) > 0)
    assert not np.array_equal(a, bench.sample_indices(100, 16, 8))
    assert np.array_equal(bench.sample_indices(5, 16, 7), np.arange(5))
