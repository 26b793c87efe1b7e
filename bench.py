#!/usr/bin/env python
"""Throughput of batched Gaussian-density voxelization on GB300.

One step = one pass of the voxelization hot path over one batch.  Default workload: the
QM9-shaped batch (4096 molecules, 3-29 atoms, 5 channels of 32^3 at 0.5 A, per-element
sigma, spherical cutoff 3 sigma, FP32 grids; 2.68 GB written per step, larger than L2),
autotuned, CUDA-graph captured.  Prints one JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]
                  [--secondary core|all|none]

The line's headline (`value`, `roofline`, `e2e`) is the QM9-shaped FP32 direct path.  Every
result carries an `error` object: the max-abs (relative to each grid's maximum) and
relative-L2 error of a seeded sample of its grids against the FP64 oracle, computed after the
timed regions.  On one GPU the same line also holds `secondary` results measured the same way:
the precision-form batch (64^3, no cutoff) as the FP16 form (BF16 tcgen05 contraction, FP32
accumulation, FP16 store) and as the plain FP32 direct path, with the speedup between them
(`precision_speedup`); the crystal-shaped batch; and the differentiation batch (forward plus
adjoint, gradient checked against the oracle's gradient and frozen-support finite
differences).  `--secondary all` adds the erf-form, pipeline and triclinic batches.

Under torchrun one global batch (N times the single-GPU batch) is partitioned into contiguous
molecule ranges balanced by output bytes and atom work; each rank voxelizes its range on its
own GPU with no collective on the data path (weak scaling).  The timed region is bracketed by
barriers and the slowest rank's time is reported; only the headline runs.  --impl reference
times the FP64 CPU oracle on the host cores.
"""
from __future__ import annotations

import argparse
import copy
import ctypes
import hashlib
import inspect
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FALLBACK_HBM_GBS = 6800.0
METRIC = "grids/sec (and voxels/sec) at 32^3x5ch FP32 vs FP16/BF16 form; fraction of HBM roofline"
# Error bars stated for each output precision (relative to each grid's maximum): FP32 1e-5;
# FP16/BF16 stores and the BF16-operand separable form 1e-2.  Gradients: 1e-4 of max |g|.
ERROR_BAR = {"f32": 1e-5, "f16": 1e-2, "bf16": 1e-2}
GRAD_BAR = 1e-4
ERROR_SAMPLE = 16       # grids per result checked against the oracle
FD_SAMPLE = 4           # molecules whose gradient is also checked by finite differences
SECONDARY_SETS = {
    "none": [],
    "core": ["precision_form:f16:separable", "precision_form:f32:direct",
             "crystal_shaped:f16:auto", "differentiation:f32:auto"],
}
SECONDARY_SETS["all"] = SECONDARY_SETS["core"] + [
    "precision_form_integral:f16:separable", "precision_form_integral:f32:direct",
    "pipeline_single_channel:bf16:auto",
    "crystal_triclinic:f16:auto"]
SLOW_TO_GENERATE = ("crystal_shaped", "crystal_triclinic")


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def _make_workload(name):
    """Generate a seeded workload (runs in a spawned helper process for the slow crystal
    generators, overlapping the GPU measurements)."""
    import synth
    return synth.workload(name)


class ClockSampler:
    """SM clock, power and throttle reasons of one GPU, sampled every 2 ms through NVML while
    running (every 200 ms through nvidia-smi if NVML cannot be loaded).  Timed regions are
    marked by tag; each tag's summary uses the samples taken inside its region."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}
    SMI_FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                  "clocks_event_reasons.hw_thermal_slowdown,"
                  "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, cuda_index: int):
        self.cuda_index = cuda_index
        self.rows = []          # (t, sm_mhz, reasons frozenset, power_w)
        self.max_mhz = None
        self.regions = {}       # tag -> [t0, t1]
        self.source = None
        self._stop = threading.Event()
        self._thread = None
        self._proc = None

    # -- NVML through ctypes (the library ships with the driver)
    def _nvml_handle(self):
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        h = ctypes.c_void_p()
        bus = None
        try:
            import torch
            p = torch.cuda.get_device_properties(self.cuda_index)
            bus = "%08X:%02X:%02X.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
        except Exception:
            bus = None
        if bus is None or lib.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(h)):
            vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
            idx = self.cuda_index
            parts = [x for x in vis.split(",") if x.strip()]
            if parts and all(x.strip().isdigit() for x in parts):
                idx = int(parts[self.cuda_index])
            if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(idx), ctypes.byref(h)):
                raise OSError("no NVML handle")
        return lib, h

    def start(self):
        try:
            lib, h = self._nvml_handle()
            mx = ctypes.c_uint()
            if lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:  # 1 = SM clock
                self.max_mhz = float(mx.value)
            get_reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                lib.nvmlDeviceGetCurrentClocksThrottleReasons
            self.source = "nvml, 2 ms"
            self._thread = threading.Thread(target=self._poll_nvml, args=(lib, h, get_reasons),
                                            daemon=True)
            self._thread.start()
            return
        except (OSError, AttributeError):
            pass
        try:
            self._proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.cuda_index), f"--query-gpu={self.SMI_FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.source = "nvidia-smi, 200 ms"
            self._thread = threading.Thread(target=self._read_smi, daemon=True)
            self._thread.start()
        except Exception:
            self._proc = None

    def _poll_nvml(self, lib, h, get_reasons):
        clk, pw, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        while not self._stop.is_set():
            ok = lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0
            reasons = frozenset()
            if get_reasons(h, ctypes.byref(rs)) == 0:
                reasons = frozenset(n for bit, n in self.REASONS.items() if rs.value & bit)
            power = pw.value / 1e3 if lib.nvmlDeviceGetPowerUsage(h, ctypes.byref(pw)) == 0 \
                else None
            if ok:
                self.rows.append((time.time(), float(clk.value), reasons, power))
            time.sleep(0.002)

    def _read_smi(self):
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self._proc.stdout:
            r = [x.strip() for x in line.split(",")]
            try:
                sm = float(r[0])
                self.max_mhz = max(self.max_mhz or 0.0, float(r[1]))
            except (ValueError, IndexError):
                continue
            try:
                power = float(r[2])
            except ValueError:
                power = None
            reasons = frozenset(n for n, v in zip(names, r[3:7]) if v.lower() == "active")
            self.rows.append((time.time(), sm, reasons, power))

    def mark(self, which, tag="headline"):
        reg = self.regions.setdefault(tag, [None, None])
        reg[0 if which == "start" else 1] = time.time()

    def stop(self):
        self._stop.set()
        if self._proc is not None:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except Exception:
                self._proc.kill()
        if self._thread is not None:
            self._thread.join(timeout=2)

    def summary(self, tag="headline"):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no clock samples"],
                    "samples_in_timed_region": 0, "sampler": self.source}
        t0, t1 = self.regions.get(tag, [None, None])
        inside = [r for r in self.rows if t0 and t1 and t0 <= r[0] <= t1]
        rows = inside
        if not rows and t0 and t1:   # nearest samples around a region shorter than a period
            rows = sorted(self.rows, key=lambda r: abs(r[0] - 0.5 * (t0 + t1)))[:2]
        sm = [r[1] for r in rows]
        power = [r[3] for r in rows if r[3] is not None]
        reasons = sorted(set().union(*[r[2] for r in rows])) if rows else []
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": self.max_mhz,
                "reasons": reasons, "samples_in_timed_region": len(inside),
                "power_w_max": max(power) if power else None, "sampler": self.source}


def write_probe_gbs(nbytes=4 << 30, reps=10):
    """Write-only bandwidth of plain device fills over >= 4 GB: torch fill kernels (byte and
    fp32 views) and, when the CUDA runtime is reachable, cudaMemsetAsync.  Returns
    (best GB/s, {method: GB/s})."""
    import torch

    buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    methods = {"torch_zero_u8": lambda: buf.zero_(),
               "torch_fill_f32": lambda: buf.view(torch.float32).fill_(0.0)}
    for name in ("libcudart.so.13", "/usr/local/cuda/lib64/libcudart.so.13"):
        try:
            rt = ctypes.CDLL(name)
            rt.cudaMemsetAsync.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t,
                                           ctypes.c_void_p]
            rt.cudaMemsetAsync.restype = ctypes.c_int
            stream = torch.cuda.current_stream().cuda_stream
            methods["cudaMemsetAsync"] = lambda rt=rt, stream=stream: rt.cudaMemsetAsync(
                ctypes.c_void_p(buf.data_ptr()), 0, ctypes.c_size_t(nbytes),
                ctypes.c_void_p(stream))
            break
        except (OSError, AttributeError):
            continue
    res = {}
    for name, fn in methods.items():
        for _ in range(3):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        res[name] = nbytes * reps / (e0.elapsed_time(e1) / 1e3) / 1e9
    del buf
    torch.cuda.empty_cache()
    return max(res.values()), res


KERNEL_SOURCES = {"direct": ("direct_kernel.cuh", "pg_internal.h"),
                  "separable": ("pg_separable.cu", "pg_internal.h"),
                  "backward": ("pg_backward.cu", "pg_internal.h"),
                  "cell": ("pg_cell.cu", "direct_kernel.cuh", "pg_internal.h")}
CELL_WORKLOADS = ("crystal_shaped", "crystal_triclinic")


def kernel_source_sha(kernel: str) -> str:
    """First 16 hex digits of the SHA-256 of the kernel's CUDA sources (the kernel's file and
    the headers it includes from the package)."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        p = os.path.join(ROOT, "paper_2211_08506_gb300", "csrc", f)
        if os.path.exists(p):
            h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(workload: str, kernel: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on the current
    kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            entries = json.load(f)
    except Exception:
        return None
    e = entries.get(f"{kernel}:{workload}")
    if not e or e.get("kernel_source_sha") != kernel_source_sha(kernel):
        return None
    return e.get("dram_bytes_per_launch")


def sample_indices(n_mol: int, k: int, seed: int):
    """Seeded sample of k distinct molecule indices, sorted."""
    import numpy as np
    k = min(k, n_mol)
    return np.sort(np.random.default_rng(seed).choice(n_mol, k, replace=False))


# ------------------------------------------------------------------------------------------
# Accuracy against the FP64 oracle.  The oracle (test infrastructure) only checks results
# here, after every timed region; nothing it computes reaches the measured path.

def oracle_grid_error(wl, idx, G, dtype, threads, path):
    """Worst per-grid max-abs error (relative to the grid's maximum) and relative-L2 error of
    the sampled CUDA grids G [k][C][nx][ny][nz] against the oracle.  With a spherical cutoff a
    voxel is measured from the interval [inside, inside + band] that the oracle brackets at
    the cutoff surface (an FP32 distance test may round either way within 1e-5 r_c^2)."""
    import numpy as np
    import oracle

    sub = wl.batch.subset(idx)
    prob = oracle.Problem.from_workload(wl, batch=sub)
    t = time.perf_counter()
    if wl.cutoff == "none":
        g_in = oracle.voxelize(prob, "bbox", threads)
        g_band = np.zeros_like(g_in)
    else:
        g_in, g_band = oracle.voxelize_band(prob, 1e-5, threads)
    oracle_s = time.perf_counter() - t
    G = np.asarray(G, np.float64).reshape(prob.shape)
    worst_abs = worst_l2 = 0.0
    for b in range(prob.shape[0]):
        ref = g_in[b] + g_band[b]
        m = float(np.abs(ref).max())
        err = np.maximum(np.maximum(g_in[b] - G[b], G[b] - ref), 0.0)
        if not np.all(np.isfinite(G[b])):
            worst_abs = worst_l2 = float("inf")
            continue
        if m == 0.0:
            worst_abs = max(worst_abs, float(err.max()))
            continue
        worst_abs = max(worst_abs, float(err.max()) / m)
        worst_l2 = max(worst_l2, float(np.linalg.norm(err) / np.linalg.norm(ref)))
    bar = ERROR_BAR[dtype] if path != "separable" else 1e-2
    return {"max_abs_rel": worst_abs, "rel_l2": worst_l2, "bar": bar,
            "pass": worst_abs <= bar, "grids": int(len(idx)),
            "sample": f"{len(idx)} seeded molecules of {wl.batch.n_mol}",
            "against": "FP64 oracle (support-box mode)",
            "band_voxels": int((g_band > 0).sum()),
            "oracle_grids_per_s": len(idx) / max(oracle_s, 1e-9)}


def oracle_grad_error(wl, idx, W, grad, threads, n_fd=FD_SAMPLE):
    """Worst per-molecule gradient error max|g - g_ref| / max|g_ref| of the sampled CUDA
    coordinate gradients against the oracle's adjoint and against FP64 central differences
    with frozen support (h = 1e-4 A) on the first n_fd sampled molecules."""
    import numpy as np
    import oracle

    def worst(g, g_ref, off):
        w = 0.0
        for b in range(len(off) - 1):
            s = slice(int(off[b]), int(off[b + 1]))
            if s.stop == s.start:
                continue
            m = float(np.abs(g_ref[s]).max())
            d = float(np.abs(g[s] - g_ref[s]).max())
            w = max(w, d / m if m > 0 else d)
        return w

    sub = wl.batch.subset(idx)
    prob = oracle.Problem.from_workload(wl, batch=sub)
    g_ref = oracle.gradient(prob, W, "bbox", threads)
    e_ref = worst(grad, g_ref, sub.mol_off)
    k = min(n_fd, len(idx))
    sub_fd = wl.batch.subset(idx[:k])
    prob_fd = oracle.Problem.from_workload(wl, batch=sub_fd)
    g_fd = oracle.fd_gradient_frozen(prob_fd, W[:k], 1e-4, threads)
    n_fd_atoms = int(sub_fd.mol_off[-1])
    e_fd = worst(grad[:n_fd_atoms], g_fd, sub_fd.mol_off)
    return {"vs_oracle_gradient": e_ref, "vs_frozen_support_fd": e_fd, "bar": GRAD_BAR,
            "pass": e_ref <= GRAD_BAR and e_fd <= GRAD_BAR,
            "sample": f"{len(idx)} seeded molecules (finite differences on {k})"}


def cpu_baseline(wl, budget_s=12.0, reps_cap=4):
    """Time the FP64 oracle (support-box mode, all host cores) on a bounded sample."""
    import oracle

    oracle.build()
    threads = os.cpu_count() or 1
    n = wl.batch.n_mol
    calib = wl.batch.subset(range(min(n, 64)))
    prob = oracle.Problem.from_workload(wl, batch=calib)
    t = time.perf_counter()
    oracle.voxelize(prob, "bbox", threads)
    per_mol = (time.perf_counter() - t) / max(1, calib.n_mol)
    n_sample = max(1, min(n, int(budget_s / max(per_mol, 1e-9) / 2)))
    sub = wl.batch.subset(range(n_sample))
    prob = oracle.Problem.from_workload(wl, batch=sub)
    times = []
    for _ in range(reps_cap):
        t = time.perf_counter()
        oracle.voxelize(prob, "bbox", threads)
        times.append(time.perf_counter() - t)
        if sum(times) > budget_s:
            break
    best = min(times)
    # The same oracle on one core, on a sample of about 3 s.
    probe = wl.batch.subset(range(min(n, 4)))
    t = time.perf_counter()
    oracle.voxelize(oracle.Problem.from_workload(wl, batch=probe), "bbox", 1)
    per_mol_1 = (time.perf_counter() - t) / max(1, probe.n_mol)
    n1 = max(1, min(n, int(3.0 / max(per_mol_1, 1e-9))))
    sub1 = wl.batch.subset(range(n1))
    t = time.perf_counter()
    oracle.voxelize(oracle.Problem.from_workload(wl, batch=sub1), "bbox", 1)
    one = n1 / (time.perf_counter() - t)
    return {"value": n_sample / best, "unit": "grids/s", "cores": threads, "kind": "oracle",
            "sample": f"first {n_sample} molecules of the {wl.name} batch, FP64 support-box "
                      f"oracle, OpenMP over molecules, best of {len(times)}",
            "single_core": {"value": one, "unit": "grids/s", "cores": 1,
                            "sample": f"first {n1} molecules, one thread"}}


def run_reference(args):
    """Reference arm: the FP64 oracle as it stands, on the host cores, rank 0 only."""
    rank = _env_int("RANK", 0)
    if rank != 0:
        return
    import oracle
    import synth

    oracle.build()
    wl = synth.workload(args.workload)
    threads = os.cpu_count() or 1
    if wl.name == "refinement":
        return run_reference_refinement(args, wl, threads)
    n = wl.batch.n_mol
    calib = wl.batch.subset(range(min(n, 32)))
    t = time.perf_counter()
    oracle.voxelize(oracle.Problem.from_workload(wl, batch=calib), "bbox", threads)
    per_mol = (time.perf_counter() - t) / calib.n_mol
    steps = args.steps + args.warmup
    budget = 150.0
    per_step = max(1, min(n, int(budget / steps / max(per_mol, 1e-9))))
    sub = wl.batch.subset(range(per_step))
    prob = oracle.Problem.from_workload(wl, batch=sub)
    for _ in range(args.warmup):
        oracle.voxelize(prob, "bbox", threads)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle.voxelize(prob, "bbox", threads)
    dt = time.perf_counter() - t
    value = per_step * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "grids/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "description": wl.description,
                   "batch_per_step": per_step},
        "cpu_baseline": {"value": value, "unit": "grids/s", "cores": threads, "kind": "oracle",
                         "sample": f"{per_step} molecules of the {wl.name} batch per step"},
        "e2e": {"value": value, "unit": "grids/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_reference_refinement(args, wl, threads):
    """Reference arm for grid reversal: the oracle's FP64 descent on a sample per step."""
    import numpy as np
    import oracle
    import synth

    iters, lr = synth.REFINE_ITERS, synth.REFINE_LR
    start = synth.refinement_start(wl)

    def problem(n):
        sub = wl.batch.subset(range(n))
        s = slice(0, int(sub.mol_off[-1]))
        T = oracle.voxelize(oracle.Problem.from_workload(wl, batch=sub), "bbox", threads)
        return oracle.Problem.from_workload(wl, batch=sub, coords=start[s].astype(np.float64)), T

    prob, T = problem(min(wl.batch.n_mol, threads))
    t = time.perf_counter()
    oracle.refine(prob, T, iters, lr, 0.0, threads)
    per_mol = (time.perf_counter() - t) / prob.shape[0]
    steps = args.steps + args.warmup
    per_step = max(1, min(wl.batch.n_mol, int(150.0 / steps / max(per_mol, 1e-9))))
    prob, T = problem(per_step)
    for _ in range(args.warmup):
        oracle.refine(prob, T, iters, lr, 0.0, threads)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle.refine(prob, T, iters, lr, 0.0, threads)
    dt = time.perf_counter() - t
    value = per_step * iters * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "molecule-iterations/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "description": wl.description,
                   "batch_per_step": per_step, "iters": iters, "lr": lr},
        "cpu_baseline": {"value": value, "unit": "molecule-iterations/s", "cores": threads,
                         "kind": "oracle",
                         "sample": f"{per_step} molecules of the refinement batch per step"},
        "e2e": {"value": value, "unit": "molecule-iterations/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)




class Session:
    """What every measurement shares: torch, the API, the process group and the stream."""

    def __init__(self, args):
        import torch

        import paper_2211_08506_gb300 as pkg

        self.args = args
        self.torch = torch
        self.rank = _env_int("RANK", 0)
        self.world = _env_int("WORLD_SIZE", 1)
        self.local = _env_int("LOCAL_RANK", 0)
        torch.cuda.set_device(self.local)
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group("nccl", device_id=torch.device("cuda", self.local))
            self.dist = dist
        pkg.build()
        from paper_2211_08506_gb300 import api
        self.api = api
        self.stream = torch.cuda.Stream()
        self.sampler = ClockSampler(self.local)
        self.peak, self.peak_src = load_peaks()

    def barrier(self):
        if self.dist:
            self.dist.barrier()

    def max_over_ranks(self, x: float) -> float:
        if not self.dist:
            return x
        t = self.torch.tensor([x], device="cuda")
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def sum_over_ranks(self, x: float) -> float:
        if not self.dist:
            return x
        t = self.torch.tensor([x], device="cuda", dtype=self.torch.float64)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        self.sampler.stop()
        if self.dist:
            self.dist.destroy_process_group()


def rank_workload(ses, name, n_mol=0):
    """This rank's share of the run: on one GPU the whole seeded batch; under torchrun one
    global batch of world x the single-GPU size, cut into contiguous molecule ranges balanced
    by output bytes plus atom work (shard.partition).  Returns (this rank's workload, the
    global index of its first molecule, the global workload)."""
    import synth
    from paper_2211_08506_gb300 import shard

    size_arg = "n_cells" if name in CELL_WORKLOADS else "n_mol"
    base = n_mol or inspect.signature(synth.WORKLOADS[name]).parameters[size_arg].default
    kw = {size_arg: base * ses.world} if (ses.world > 1 or n_mol) else {}
    whole = synth.workload(name, **kw)
    wl, first = whole, 0
    if ses.world > 1:
        esz = {"f32": 4, "f16": 2, "bf16": 2}[whole.out_dtype]
        wl = copy.copy(whole)
        wl.batch, (first, _) = shard.shard(whole.batch, ses.rank, ses.world,
                                           whole.voxels_per_grid * esz)
    return wl, first, whole


def _nvtx(torch, name):
    """Open (name given) or close an NVTX range for profiler timelines; a no-op where torch
    has no NVTX support."""
    try:
        if name is None:
            torch.cuda.nvtx.range_pop()
        else:
            torch.cuda.nvtx.range_push(name)
    except Exception:
        pass


def measure(ses, wl, dtype, path, tag, W=None, e2e=True):
    """Autotune, capture and time one workload: K graph replays of the forward launch (and
    of the adjoint when W, the upstream gradient, is given) after W warm-up replays, on the
    session stream with CUDA events; then the same step end to end through the public API.
    Returns (result dict, output grids, coordinate gradient or None)."""
    torch, api = ses.torch, ses.api
    args = ses.args
    grid = api.Grid.from_workload(wl)
    db = api.DeviceBatch.from_numpy(wl.batch)
    B = wl.batch.n_mol
    esz = 4 if dtype == "f32" else 2
    out_bytes = B * wl.voxels_per_grid * esz
    out = torch.empty(grid.out_shape(B), dtype=api.DTYPES[dtype][1], device="cuda")
    stream = ses.stream
    Wd = grad = None
    if W is not None:
        Wd = torch.from_numpy(W).cuda()
        grad = torch.empty((wl.batch.n_atoms, 3), dtype=torch.float32, device="cuda")

    # Untimed: autotune the launch for this bucket, then capture the step in graphs (forward,
    # and adjoint if any, so the forward kernel's own time is visible between them).
    with torch.cuda.stream(stream):
        tuning = api.autotune(db, grid, dtype=dtype, path=path, out=out)
        api.voxelize(db, grid, dtype=dtype, path=path, out=out)
        if Wd is not None:
            api.voxelize_backward(db, grid, Wd, grad_coords=grad)
    api.sync_status(stream)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        api.voxelize(db, grid, dtype=dtype, path=path, out=out)
    graph_bwd = None
    if Wd is not None:
        graph_bwd = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph_bwd, stream=stream):
            api.voxelize_backward(db, grid, Wd, grad_coords=grad)
    torch.cuda.synchronize()

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            graph.replay()
            if graph_bwd is not None:
                graph_bwd.replay()
    torch.cuda.synchronize()
    ses.barrier()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev_mid = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ses.sampler.mark("start", tag)
    _nvtx(torch, "timed_" + tag.replace(":", "_"))
    with torch.cuda.stream(stream):
        ev[0].record(stream)
        for i in range(args.steps):
            graph.replay()
            ev_mid[i].record(stream)
            if graph_bwd is not None:
                graph_bwd.replay()
            ev[i + 1].record(stream)
    torch.cuda.synchronize()
    _nvtx(torch, None)
    ses.sampler.mark("stop", tag)
    ses.barrier()
    per_fwd = [ev[i].elapsed_time(ev_mid[i]) for i in range(args.steps)]
    per_bwd = [ev_mid[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    total_ms = ses.max_over_ranks(ev[0].elapsed_time(ev[-1]))
    assert api.sync_status(stream) == 0
    del graph, graph_bwd
    ms = total_ms / args.steps
    units = ses.sum_over_ranks(float(B))
    value = units / (ms / 1e3)

    # End to end through the public API: pinned host inputs -> plan (graph: H2D + kernel)
    # -> device error word back to the host, every step.  A differentiation step then runs
    # the adjoint and reads the coordinate gradient back into pinned host memory.
    e2e_res = None
    if e2e:
        import numpy as np
        b = wl.batch
        pin = lambda a: None if a is None else torch.from_numpy(
            np.ascontiguousarray(a)).pin_memory()
        host = [pin(a) for a in (b.coords, b.elem, b.mol_off, b.origin,
                                 None if b.cell is not None else b.spacing)]
        extra = {"weight": pin(b.weight), "cell": pin(b.cell)}
        h2d = sum(t.numel() * t.element_size() for t in host + list(extra.values())
                  if t is not None)
        # Two plans alternate (double buffering, as a data loader runs them): step i's batch
        # is copied in and launched before step i - 1's results are waited for and read.
        plans = [api.Plan(grid, dtype, max_mol=B, max_atoms=b.n_atoms, path=path)
                 for _ in range(2)]
        outs = [out, torch.empty_like(out)]
        d2h = 4
        grads = grad_hosts = None
        if Wd is not None:
            grads = [grad, torch.empty_like(grad)]
            grad_hosts = [torch.empty((b.n_atoms, 3), dtype=torch.float32).pin_memory()
                          for _ in range(2)]
            d2h += grad_hosts[0].numel() * grad_hosts[0].element_size()
        done = [torch.cuda.Event(), torch.cuda.Event()]

        # Each plan runs on a stream of its own, so that one step's host-to-device copies
        # overlap the previous step's kernels (the two steps share no buffer).
        e2e_streams = [stream, torch.cuda.Stream()]

        def launch(i):
            k = i % 2
            s = e2e_streams[k]
            plans[k].launch(*host, out=outs[k], stream=s, **extra)
            if Wd is not None:
                # The adjoint of the step's forward pass and its gradient back to the host.
                api.voxelize_backward(db, grid, Wd, grad_coords=grads[k], stream=s)
                with torch.cuda.stream(s):
                    grad_hosts[k].copy_(grads[k], non_blocking=True)
            done[k].record(s)

        def finish(i):
            k = i % 2
            plans[k].wait(e2e_streams[k])   # the error word of step i's forward pass
            done[k].synchronize()   # and, with the adjoint, its gradient on the host

        def run(n):
            launch(0)
            for i in range(1, n):
                launch(i)
                finish(i - 1)
            finish(n - 1)

        with torch.cuda.stream(stream):
            run(max(3, args.warmup))
        e2e_steps = max(3, min(args.steps, 200))
        ses.barrier()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            run(e2e_steps)
        e2e_s = ses.max_over_ranks((time.perf_counter() - t0) / e2e_steps)
        for pl in plans:
            pl.close()
        del outs
        e2e_res = {"value": units / e2e_s, "unit": "grids/s", "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": d2h,
                   "api": "two pg_plan_* plans alternating on two streams: pg_plan_launch "
                          "(pinned host CSR "
                          "batch -> graph: H2D + kernel -> error word D2H)"
                          + (" + pg_voxelize_backward + gradient D2H" if Wd is not None
                             else "")
                          + ", then pg_plan_wait for the previous step"}

    kernel = ("separable" if tuning.get("path") == 2
              else "cell" if wl.batch.cell is not None else "direct")
    launch_ms = statistics.mean(per_fwd)
    achieved = out_bytes / (launch_ms / 1e3) / 1e9
    res = {
        "workload": wl.name, "description": wl.description,
        "value": value, "unit": "grids/s", "ms_per_step": ms,
        "voxels_per_sec": units * wl.voxels_per_grid / (ms / 1e3),
        "dtype": dtype, "path": kernel, "tuning": tuning,
        "batch_per_gpu": B, "grid": [wl.n_channels, wl.nx, wl.ny, wl.nz],
        "voxel_form": wl.form, "cutoff": wl.cutoff, "periodic": bool(wl.periodic),
        "step": "forward + adjoint" if Wd is not None else "forward",
        "adjoint_ms_per_step": statistics.mean(per_bwd) if Wd is not None else None,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": ses.peak, "unit": "GB/s",
                     "frac": achieved / ses.peak,
                     "traffic": profiled_traffic(wl.name, kernel),
                     "peak_source": f"{ses.peak_src} hbm_gbs (copy)",
                     "algorithmic_bytes_per_launch": out_bytes,
                     "kernel": f"{kernel} voxelization kernel"},
        "e2e": e2e_res,
        "gpu_launches": args.steps * (2 if Wd is not None else 1),
        "l2": f"output {out_bytes / 1e9:.2f} GB per step > 129 MB L2; no flush",
        "clocks": ses.sampler.summary(tag),
    }
    return res, out, grad


def sample_result(ses, wl, out, grad, seed):
    """Host copies of a seeded sample of grids (and their atoms' gradients) for the oracle
    check after the timed regions."""
    import numpy as np
    idx = sample_indices(wl.batch.n_mol, ERROR_SAMPLE, seed)
    G = out[ses.torch.as_tensor(idx, device="cuda")].float().cpu().numpy()
    g = None
    if grad is not None:
        rows = np.concatenate([np.arange(wl.batch.mol_off[i], wl.batch.mol_off[i + 1])
                               for i in idx])
        g = grad[ses.torch.as_tensor(rows, device="cuda", dtype=ses.torch.long)].cpu().numpy()
    return idx, G, g


def run_ours(args):
    import numpy as np

    import synth

    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    secondary = SECONDARY_SETS[args.secondary] if world == 1 else []
    # The crystal generators take tens of seconds of host time: start them in spawned helper
    # processes so that they overlap the GPU measurements.
    pool, pending = None, {}
    slow = sorted({s.split(":")[0] for s in secondary} & set(SLOW_TO_GENERATE))
    if slow:
        import concurrent.futures
        import multiprocessing
        pool = concurrent.futures.ProcessPoolExecutor(
            max_workers=len(slow), mp_context=multiprocessing.get_context("spawn"))
        pending = {n: pool.submit(_make_workload, n) for n in slow}

    ses = Session(args)
    torch = ses.torch
    if args.profile:
        wl, _, _ = rank_workload(ses, args.workload, args.n_mol)
        return run_profile(args, wl, args.dtype or wl.out_dtype)

    ses.sampler.start()
    time.sleep(0.3)
    wl, first, _ = rank_workload(ses, args.workload, args.n_mol)
    dtype = args.dtype or wl.out_dtype
    W = None
    if wl.name == "differentiation":
        W = synth.loss_weights(wl, molecules=range(first, first + wl.batch.n_mol))
    head, out, grad = measure(ses, wl, dtype, args.path, "headline", W=W)
    samples = {"headline": (wl, dtype, args.path, W) + sample_result(ses, wl, out, grad, 12)}
    del out, grad
    torch.cuda.empty_cache()

    sec = []
    for spec in secondary:
        name, sdtype, spath = spec.split(":")
        swl = pending[name].result() if name in pending else synth.workload(name)
        sW = synth.loss_weights(swl) if name == "differentiation" else None
        res, out, grad = measure(ses, swl, sdtype, spath, spec, W=sW)
        sec.append(res)
        samples[spec] = (swl, sdtype, spath, sW) + sample_result(ses, swl, out, grad, 12)
        del out, grad
        torch.cuda.empty_cache()
    if pool is not None:
        pool.shutdown()

    # Write-only reference: plain device fills of at least 4 GB.
    probe, probe_all = (None, None)
    if rank == 0:
        probe, probe_all = write_probe_gbs()
    ses.sampler.stop()
    if rank != 0:
        ses.close()
        return

    # Accuracy of every result against the FP64 oracle (host cores, after the GPU work).
    import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    errors = {}
    for key, (swl, sdtype, spath, sW, idx, G, g) in samples.items():
        err = oracle_grid_error(swl, idx, G, sdtype, threads, spath)
        if g is not None:
            err["gradient"] = oracle_grad_error(swl, idx, sW[idx], g, threads)
        errors[key] = err
    for res, spec in zip(sec, secondary):
        res["error"] = errors[spec]

    head["roofline"]["write_probe_gbs"] = probe
    head["roofline"]["write_probe_methods"] = probe_all
    head["roofline"]["frac_of_write_probe"] = head["roofline"]["achieved"] / probe
    base = cpu_baseline(wl) if world == 1 and not args.no_cpu_baseline else None
    line = {
        "metric": METRIC,
        "value": head["value"],
        "unit": "grids/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": head["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": dtype,
        "data": "synthetic",
        "config": {
            "workload": wl.name,
            "description": wl.description,
            "batch_per_gpu": wl.batch.n_mol,
            "grid": head["grid"],
            "voxel_form": wl.form,
            "cell_matrices": wl.batch.cell is not None,
            "weighted": wl.batch.weight is not None,
            "out_dtype": dtype,
            "path": head["path"],
            "tuning": head["tuning"],
            "parallelism": f"dp{world}" if world > 1 else "single",
            "sharding": ("one global batch, contiguous molecule ranges balanced by output "
                         "bytes + atom work" if world > 1 else None),
            "l2": head["l2"],
            "cuda_graph": True,
        },
        "voxels_per_sec": head["voxels_per_sec"],
        "step": head["step"],
        "adjoint_ms_per_step": head["adjoint_ms_per_step"],
        "roofline": head["roofline"],
        "e2e": head["e2e"],
        "error": errors["headline"],
        "gpu_launches": head["gpu_launches"],
        "clocks": head["clocks"],
        "cpu_baseline": base,
    }
    by = {s: r for s, r in zip(secondary, sec)}
    f16 = by.get("precision_form:f16:separable")
    f32 = by.get("precision_form:f32:direct")
    if f16 and f32:
        line["precision_speedup"] = {
            "value": f16["value"] / f32["value"],
            "what": "precision_form batch (4096 x 5 x 64^3, no cutoff): FP16 form (BF16 "
                    "tcgen05 separable contraction, FP32 accumulation, FP16 store) over the "
                    "plain FP32 direct path, same GPU",
            "fp16_form": {"grids_per_s": f16["value"], "error": f16["error"]},
            "fp32_direct": {"grids_per_s": f32["value"], "error": f32["error"]},
            "e2e_value": (f16["e2e"]["value"] / f32["e2e"]["value"]
                          if f16["e2e"] and f32["e2e"] else None),
        }
    if sec:
        line["secondary"] = sec
    print(json.dumps(line), flush=True)
    ses.close()


def run_refinement(args):
    """Grid reversal (Sec. IV-A/IV-C): a step is one pg_refine call of REFINE_ITERS descent
    iterations over the whole batch, from the seeded start (reset by a device copy inside the
    step).  value = molecule-iterations per second over all ranks."""
    import numpy as np

    import synth

    ses = Session(args)
    torch, api, rank, world, dist = ses.torch, ses.api, ses.rank, ses.world, ses.dist
    wl, first, whole = rank_workload(ses, "refinement", args.n_mol)
    iters, lr = synth.REFINE_ITERS, synth.REFINE_LR
    grid = api.Grid.from_workload(wl)
    db = api.DeviceBatch.from_numpy(wl.batch)
    B = wl.batch.n_mol
    stream = torch.cuda.Stream()
    s0, s1 = int(whole.batch.mol_off[first]), int(whole.batch.mol_off[first + B])
    start_h = np.ascontiguousarray(synth.refinement_start(whole)[s0:s1])
    start = torch.as_tensor(start_h, device="cuda")
    x = start.clone()
    work = torch.empty(max(1, B * wl.voxels_per_grid + 3 * wl.batch.n_atoms),
                       dtype=torch.float32, device="cuda")
    with torch.cuda.stream(stream):
        # The grid to reverse: the true coordinates' own grid (input preparation, untimed).
        api.autotune(db, grid, dtype="f32", path="direct")
        target = api.voxelize(db, grid, dtype="f32", path="direct")
        for _ in range(args.warmup):
            x.copy_(start)
            api.refine(db, grid, target, x, iters, lr, 0.0, work=work, stream=stream)
    api.sync_status(stream)
    sampler = ses.sampler
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler.mark("start")
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(args.steps):
            x.copy_(start)
            loss, steps = api.refine(db, grid, target, x, iters, lr, 0.0, work=work,
                                     stream=stream)
        e1.record(stream)
    torch.cuda.synchronize()
    sampler.mark("stop")
    total_ms = ses.max_over_ranks(e0.elapsed_time(e1))
    sampler.stop()
    assert api.sync_status(stream) == 0
    ms = total_ms / args.steps
    units = ses.sum_over_ranks(float(B))
    value = units * iters / (ms / 1e3)

    # End to end: the grid to reverse and the start come from pinned host memory, the refined
    # coordinates and losses go back, every step.
    target_h = target.cpu().pin_memory()
    start_p = torch.from_numpy(start_h).pin_memory()
    x_h = torch.empty_like(start_p).pin_memory()
    loss_h = torch.empty(B, dtype=torch.float32).pin_memory()
    tgt_d = torch.empty_like(target)
    e2e_steps = max(3, min(args.steps, 20))
    with torch.cuda.stream(stream):
        for it in range(2 + e2e_steps):
            if it == 2:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
            tgt_d.copy_(target_h, non_blocking=True)
            x.copy_(start_p, non_blocking=True)
            loss, _ = api.refine(db, grid, tgt_d, x, iters, lr, 0.0, work=work, stream=stream)
            x_h.copy_(x, non_blocking=True)
            loss_h.copy_(loss, non_blocking=True)
            stream.synchronize()
    e2e_s = ses.max_over_ranks((time.perf_counter() - t0) / e2e_steps)
    if rank != 0:
        ses.close()
        return
    peak, peak_src = load_peaks()
    grid_bytes = B * wl.voxels_per_grid * 4
    # Per step: iters + 1 forward passes (grid written) and residual passes (grid and target
    # read, upstream gradient written); the adjoint's reads of the cutoff boxes are small.
    algo = (iters + 1) * 4 * grid_bytes
    achieved = algo / (ms / 1e3) / 1e9
    base = None
    if world == 1 and not args.no_cpu_baseline:
        base = refinement_cpu_baseline(wl, start_h)
    line = {
        "metric": METRIC, "value": value, "unit": "molecule-iterations/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": wl.name, "description": wl.description, "batch_per_gpu": B,
                   "grid": [wl.n_channels, wl.nx, wl.ny, wl.nz], "iters": iters, "lr": lr,
                   "parallelism": f"dp{world}" if world > 1 else "single",
                   "l2": f"grid {grid_bytes / 1e9:.2f} GB > 129 MB L2; no flush"},
        "final_loss_median": float(torch.median(loss).item()),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None,
                     "peak_source": f"{peak_src} hbm_gbs (copy)",
                     "algorithmic_bytes_per_step": algo,
                     "kernel": "refinement step (forward, residual, adjoint, update kernels)"},
        "e2e": {"value": units * iters / e2e_s, "unit": "molecule-iterations/s",
                "h2d_bytes_per_step": target_h.numel() * 4 + start_p.numel() * 4,
                "d2h_bytes_per_step": x_h.numel() * 4 + B * 4,
                "api": "pg_refine with the target and start copied in and results copied out"},
        "gpu_launches": args.steps * (4 * iters + 2),
        "clocks": sampler.summary(),
        "cpu_baseline": base,
    }
    print(json.dumps(line), flush=True)
    ses.close()


def refinement_cpu_baseline(wl, start, budget_s=12.0):
    """The FP64 oracle's refinement on a bounded sample of the batch, all host cores."""
    import numpy as np
    import oracle
    import synth

    oracle.build()
    threads = os.cpu_count() or 1
    iters = synth.REFINE_ITERS

    def run(n):
        sub = wl.batch.subset(range(n))
        s = slice(0, int(sub.mol_off[-1]))
        T = oracle.voxelize(oracle.Problem.from_workload(wl, batch=sub), "bbox", threads)
        prob = oracle.Problem.from_workload(wl, batch=sub, coords=start[s].astype(np.float64))
        t = time.perf_counter()
        oracle.refine(prob, T, iters, synth.REFINE_LR, 0.0, threads)
        return time.perf_counter() - t

    n = min(wl.batch.n_mol, threads)
    dt = run(n)
    n2 = max(1, min(wl.batch.n_mol, int(n * budget_s / max(dt, 1e-6) / 2)))
    if n2 > n:
        n, dt = n2, run(n2)
    return {"value": n * iters / dt, "unit": "molecule-iterations/s", "cores": threads,
            "kind": "oracle",
            "sample": f"first {n} molecules of the refinement batch, {iters} FP64 descent "
                      f"iterations each, OpenMP over molecules"}


def run_profile(args, wl, dtype):
    """Plain launches for profiler captures: no tuning, no graph, no host-side extras.
    Prints a line marked "profile" (it is not a benchmark result)."""
    import torch

    import synth
    from paper_2211_08506_gb300 import api

    grid = api.Grid.from_workload(wl)
    db = api.DeviceBatch.from_numpy(wl.batch)
    out = torch.empty(grid.out_shape(wl.batch.n_mol), dtype=api.DTYPES[dtype][1], device="cuda")
    tuning = {"path": 2 if args.path == "separable" else 1, "block_threads": args.threads,
              "blocks_per_sm": 0, "store_hint": args.store_hint, "n_tile": args.n_tile,
              "chunk_planes": args.chunk_planes, "gather_only": args.gather_only,
              "chunk_order": args.chunk_order}
    W = grad = None
    if wl.name == "differentiation":
        W = torch.from_numpy(synth.loss_weights(wl)).cuda()
        grad = torch.empty((wl.batch.n_atoms, 3), dtype=torch.float32, device="cuda")
    for _ in range(args.warmup + args.steps):
        api.voxelize_tuned(db, grid, tuning, dtype=dtype, out=out)
        if W is not None:
            api.voxelize_backward(db, grid, W, grad_coords=grad)
    torch.cuda.synchronize()
    assert api.sync_status() == 0
    print(json.dumps({"profile": True, "workload": wl.name, "n_mol": wl.batch.n_mol,
                      "launches": args.warmup + args.steps, "tuning": tuning,
                      "out_bytes": out.numel() * out.element_size()}), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawTextHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="qm9_shaped",
                    choices=["qm9_shaped", "plain_small", "precision_form",
                             "precision_form_integral", "crystal_shaped", "differentiation",
                             "refinement", "pipeline_single_channel", "crystal_triclinic"])
    ap.add_argument("--secondary", choices=sorted(SECONDARY_SETS), default=None,
                    help="extra results on the same line (default: core with the default "
                         "workload, none otherwise)")
    ap.add_argument("--dtype", choices=["f32", "f16", "bf16"], default=None)
    ap.add_argument("--path", choices=["auto", "direct", "separable"], default="auto")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n-mol", type=int, default=0, help="override the batch size")
    ap.add_argument("--profile", action="store_true",
                    help="plain launches only (for ncu); prints a profile line, not a result")
    ap.add_argument("--threads", type=int, default=512, help="--profile: threads per CTA")
    ap.add_argument("--store-hint", type=int, default=1, help="--profile: 1 = streaming stores")
    ap.add_argument("--chunk-planes", type=int, default=8, help="--profile: planes per chunk")
    ap.add_argument("--chunk-order", type=int, default=0,
                    help="--profile: 0 = molecule-major chunks, 1 = channel-major")
    ap.add_argument("--gather-only", type=int, default=0, help="--profile: 1 = gather only (no lane lists or factor tables)")
    ap.add_argument("--n-tile", type=int, default=128, help="--profile: separable tile width")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.secondary is None:
        args.secondary = "core" if (args.workload == "qm9_shaped" and not args.n_mol
                                    and not args.profile) else "none"
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "refinement" and not args.profile:
        run_refinement(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
