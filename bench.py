#!/usr/bin/env python
"""Throughput of batched Gaussian-density voxelization on GB300.

One step = one pass of the voxelization hot path over one batch.  Default workload: the
QM9-shaped batch (4096 molecules, 3-29 atoms, 5 channels of 32^3 at 0.5 A, per-element
sigma, spherical cutoff 3 sigma, FP32 grids; 2.68 GB written per step, larger than L2),
autotuned, CUDA-graph captured.  Prints one JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Under torchrun each rank voxelizes its own batch of the same size (weak scaling, no
collective on the data path); the timed region is bracketed by barriers and the slowest
rank's time is reported.  --impl reference times the FP64 CPU oracle on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
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


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self._reader = threading.Thread(target=self._read, daemon=True)
        self._reader.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), [x.strip() for x in line.split(",")]))

    def mark(self, which):
        if which == "start":
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def stop(self):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self._reader.join(timeout=2)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"],
                    "samples": 0}
        inside = [r for t, r in self.rows if self.t0 and self.t1 and self.t0 <= t <= self.t1]
        rows = inside if inside else [r for _, r in self.rows]

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if len(r) > 8 and num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if len(r) > 8 and num(r[2]) is not None]
        reasons = set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            if len(r) > 8:
                for name, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons),
                "samples": len(rows),
                "samples_in_timed_region": len(inside)}


def write_probe_gbs(nbytes=4 << 30, reps=10):
    """Write-only bandwidth of plain device fills over >= 4 GB: torch fill kernels (byte and
    fp32 views) and, when the CUDA runtime is reachable, cudaMemsetAsync.  Returns
    (best GB/s, {method: GB/s})."""
    import ctypes
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


KERNEL_SOURCES = {"direct": ("direct_kernel.cuh",), "separable": ("pg_separable.cu",),
                  "backward": ("pg_backward.cu",), "cell": ("pg_cell.cu",)}
CELL_WORKLOADS = ("crystal_shaped", "crystal_triclinic")


def kernel_source_sha(kernel: str) -> str:
    """First 16 hex digits of the SHA-256 of the kernel's CUDA source."""
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


def run_ours(args):
    import numpy as np
    import torch

    import synth
    import paper_2211_08506_gb300 as pkg

    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    pkg.build()
    from paper_2211_08506_gb300 import api

    kw = {"shard": rank if world > 1 else None}
    if args.n_mol:
        kw["n_cells" if args.workload in CELL_WORKLOADS else "n_mol"] = args.n_mol
    wl = synth.workload(args.workload, **kw)
    dtype = args.dtype or wl.out_dtype
    if args.profile:
        return run_profile(args, wl, dtype)
    path = args.path
    grid = api.Grid.from_workload(wl)
    db = api.DeviceBatch.from_numpy(wl.batch)
    B = wl.batch.n_mol
    esz = 4 if dtype == "f32" else 2
    out_bytes = B * wl.voxels_per_grid * esz
    out = torch.empty(grid.out_shape(B), dtype=api.DTYPES[dtype][1], device="cuda")
    stream = torch.cuda.Stream()

    # Differentiation: a step is the forward pass plus the adjoint for L = <W, G>.
    W = grad = None
    if wl.name == "differentiation":
        W = torch.from_numpy(synth.loss_weights(wl, shard=rank if world > 1 else None)).cuda()
        grad = torch.empty((wl.batch.n_atoms, 3), dtype=torch.float32, device="cuda")

    # Untimed: autotune the launch for this bucket, then capture the step in graphs (forward,
    # and adjoint if any, so the forward kernel's own time is visible between them).
    with torch.cuda.stream(stream):
        tuning = api.autotune(db, grid, dtype=dtype, path=path, out=out)
        api.voxelize(db, grid, dtype=dtype, path=path, out=out)
        if W is not None:
            api.voxelize_backward(db, grid, W, grad_coords=grad)
    api.sync_status(stream)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        api.voxelize(db, grid, dtype=dtype, path=path, out=out)
    graph_bwd = None
    if W is not None:
        graph_bwd = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph_bwd, stream=stream):
            api.voxelize_backward(db, grid, W, grad_coords=grad)
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.4)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            graph.replay()
            if graph_bwd is not None:
                graph_bwd.replay()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev_mid = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    sampler.mark("start")
    with torch.cuda.stream(stream):
        ev[0].record(stream)
        for i in range(args.steps):
            graph.replay()
            ev_mid[i].record(stream)
            if graph_bwd is not None:
                graph_bwd.replay()
            ev[i + 1].record(stream)
    torch.cuda.synchronize()
    sampler.mark("stop")
    if dist:
        dist.barrier()
    # Forward kernel time per launch (the step's dominant kernel) and the adjoint's.
    per_step = [ev[i].elapsed_time(ev_mid[i]) for i in range(args.steps)]
    per_bwd = [ev_mid[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    if dist:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    sampler.stop()
    assert api.sync_status(stream) == 0

    ms = total_ms / args.steps
    value = world * B / (ms / 1e3)
    voxels = world * B * wl.voxels_per_grid / (ms / 1e3)

    # End to end through the public API: pinned host inputs -> plan (graph: H2D + kernel)
    # -> device error word back to the host, every step.  A differentiation step then runs
    # the adjoint and reads the coordinate gradient back into pinned host memory.
    b = wl.batch
    pin = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    host = [pin(a) for a in (b.coords, b.elem, b.mol_off, b.origin,
                             None if b.cell is not None else b.spacing)]
    extra = {"weight": pin(b.weight), "cell": pin(b.cell)}
    h2d = sum(t.numel() * t.element_size() for t in host + list(extra.values())
              if t is not None)
    plan = api.Plan(grid, dtype, max_mol=B, max_atoms=b.n_atoms, path=path)
    grad_host = None
    d2h = 4
    if W is not None:
        grad_host = torch.empty((b.n_atoms, 3), dtype=torch.float32).pin_memory()
        d2h += grad_host.numel() * grad_host.element_size()

    def e2e_step():
        plan.run(*host, out=out, **extra)
        if W is not None:
            api.voxelize_backward(db, grid, W, grad_coords=grad, stream=stream)
            grad_host.copy_(grad, non_blocking=True)
            stream.synchronize()

    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            e2e_step()
    e2e_steps = max(3, min(args.steps, 200))
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for _ in range(e2e_steps):
            e2e_step()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    if dist:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    plan.close()

    # Write-only reference: plain device fills of at least 4 GB.
    probe, probe_all = None, None
    if rank == 0:
        probe, probe_all = write_probe_gbs()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    peak, peak_src = load_peaks()
    kernel = ("separable" if tuning.get("path") == 2
              else "cell" if wl.batch.cell is not None else "direct")
    launch_ms = statistics.mean(per_step)
    achieved = out_bytes / (launch_ms / 1e3) / 1e9
    traffic = profiled_traffic(wl.name, kernel)
    base = None
    if world == 1 and not args.no_cpu_baseline:
        base = cpu_baseline(wl)
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "grids/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if dtype == "f32" else dtype,
        "data": "synthetic",
        "config": {
            "workload": wl.name,
            "description": wl.description,
            "batch_per_gpu": B,
            "grid": [wl.n_channels, wl.nx, wl.ny, wl.nz],
            "voxel_form": wl.form,
            "cell_matrices": wl.batch.cell is not None,
            "weighted": wl.batch.weight is not None,
            "out_dtype": dtype,
            "path": kernel,
            "tuning": tuning,
            "parallelism": f"dp{world}" if world > 1 else "single",
            "l2": f"output {out_bytes / 1e9:.2f} GB per step > 129 MB L2; no flush",
            "cuda_graph": True,
        },
        "voxels_per_sec": voxels,
        "step": "forward + adjoint" if graph_bwd is not None else "forward",
        "adjoint_ms_per_step": statistics.mean(per_bwd) if graph_bwd is not None else None,
        "roofline": {
            "bound": "hbm",
            "achieved": achieved,
            "peak": peak,
            "unit": "GB/s",
            "frac": achieved / peak,
            "traffic": traffic,
            "peak_source": f"{peak_src} hbm_gbs (copy)",
            "algorithmic_bytes_per_launch": out_bytes,
            "kernel": f"{kernel} voxelization kernel",
            "write_probe_gbs": probe,
            "write_probe_methods": probe_all,
            "frac_of_write_probe": (achieved / probe) if probe else None,
        },
        "e2e": {
            "value": world * B / e2e_s,
            "unit": "grids/s",
            "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h,
            "api": "pg_plan_run (pinned host CSR batch -> graph: H2D + kernel -> error word D2H)"
                   + (" + pg_voxelize_backward -> gradient D2H" if W is not None else ""),
        },
        "gpu_launches": args.steps * (2 if graph_bwd is not None else 1),
        "clocks": sampler.summary(),
        "cpu_baseline": base,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_refinement(args):
    """Grid reversal (Sec. IV-A/IV-C): a step is one pg_refine call of REFINE_ITERS descent
    iterations over the whole batch, from the seeded start (reset by a device copy inside the
    step).  value = molecule-iterations per second over all ranks."""
    import numpy as np
    import torch

    import synth
    import paper_2211_08506_gb300 as pkg

    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    pkg.build()
    from paper_2211_08506_gb300 import api

    shard = rank if world > 1 else None
    wl = synth.workload("refinement", shard=shard, **({"n_mol": args.n_mol} if args.n_mol else {}))
    iters, lr = synth.REFINE_ITERS, synth.REFINE_LR
    grid = api.Grid.from_workload(wl)
    db = api.DeviceBatch.from_numpy(wl.batch)
    B = wl.batch.n_mol
    stream = torch.cuda.Stream()
    start_h = synth.refinement_start(wl, shard)
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
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.4)
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
    total_ms = e0.elapsed_time(e1)
    if dist:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    sampler.stop()
    assert api.sync_status(stream) == 0
    ms = total_ms / args.steps
    value = world * B * iters / (ms / 1e3)

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
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    if rank != 0:
        if dist:
            dist.destroy_process_group()
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
        "e2e": {"value": world * B * iters / e2e_s, "unit": "molecule-iterations/s",
                "h2d_bytes_per_step": target_h.numel() * 4 + start_p.numel() * 4,
                "d2h_bytes_per_step": x_h.numel() * 4 + B * 4,
                "api": "pg_refine with the target and start copied in and results copied out"},
        "gpu_launches": args.steps * (4 * iters + 2),
        "clocks": sampler.summary(),
        "cpu_baseline": base,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


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
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="qm9_shaped",
                    choices=["qm9_shaped", "plain_small", "precision_form",
                             "precision_form_integral", "crystal_shaped", "differentiation",
                             "refinement", "pipeline_single_channel", "crystal_triclinic"])
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
    ap.add_argument("--gather-only", type=int, default=0, help="--profile: 1 = no scatter mode")
    ap.add_argument("--n-tile", type=int, default=128, help="--profile: separable tile width")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "refinement" and not args.profile:
        run_refinement(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
