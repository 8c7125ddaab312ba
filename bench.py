#!/usr/bin/env python3
"""Benchmark of the MBS hot path: voxel-iterations per second on one GB300.

Workload (default, C5): the domain-decomposed MBS problem at the paper's
320^3-wavelength scale, a 1280^3 grid at lambda/4 split 4x4x4 into 320^3
subdomains with t = 8 edge corrections, seeded random spheres (radius 5-40 px,
n in [1.0, 1.5]) added until 30 % of the volume is filled, 8-px absorbing
layers, point source at the centre. One step = one iteration of
Eq. wavesim_iter over the whole grid (all 64 subdomains).

Printed JSON line (one, from rank 0):
  value        voxel-iterations/s with every buffer resident in HBM, timed with
               CUDA events on the plan's stream over K graph-replayed iterations
               (FP32 edge corrections on the CUDA cores)
  mixed        the same with the 3xTF32 tensor-core edge corrections
  e2e          the same metric through the C ABI call mbs_solve with pinned host
               source/output buffers, host<->device copies inside the timed region
  roofline     the dominant kernel's algorithmic bytes per launch / its average
               CUDA-event duration, against the measured HBM copy bandwidth
  error        relative L2 distance to the FP64 oracle at equal iteration counts,
               per form, on the workload's recipe at a size the oracle runs
  cpu_baseline the FP64 oracle timed on the host cores (all of them, and one
               thread) on a bounded sample of the workload's recipe
  workloads    value and mixed value of the other single-grid workloads (C2, C3)
  activation   time to tolerance with and without subdomain activation on a long
               domain with the source in its first subdomain

With --gpus N > 1 (under torchrun) every rank runs an independent replica of
the workload on its own GPU (the path has no data exchange on one GPU);
value = total voxel-iterations of all ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "C5"
WORKLOAD_TEXT = {
    "C1": "C1: 64^3 grid at lambda/4, one periodic subdomain, 6 spheres, 8-px absorbing layers, point source",
    "C2": "C2: 256^3 grid at lambda/4, 2x2x2 subdomains of 128^3, t=8, 40 spheres, 8-px absorbing layers, point source",
    "C3": "C3: 512^3 grid at lambda/4, 4x4x4 subdomains of 128^3, t=8, n = 1.33 + Gaussian random field, "
          "Gaussian-beam plane source",
    "C4": "C4: 64 independent frequency solves, lambda uniform in [0.8,1.2] on one 24-unit box at lambda/4 "
          "(grids 80^3-120^3), each split 2x2x2 into 7-smooth halves, t=8, same spheres, point sources; "
          "advanced together as one batch",
    "C5": "C5: 1280^3 grid at lambda/4, 4x4x4 subdomains of 320^3, t=8, spheres to 30% fill, point source",
    "C2P": "C2P: the C2 recipe on a 246^3 grid, 2x2x2 subdomains of 123^3 (123 = 3 x 41: Bluestein transforms "
           "on every axis), t=8",
    "P43": "P43: the geometry of the paper's large example, 1320x1280x1280 at lambda/4, 20-px absorbing layers on "
           "the x faces only, y and z periodic, packed spheres r = 24 px with 24-px clearance (n = 1.33 + 0.01i), "
           "plane source at x = 20; 5x4x4 subdomains (x: 280, 280, 256, 252, 252; y, z: 320 with periodic seams), t=8",
}
METRIC = "voxel-iterations/s on 1 GB300 (mixed vs plain FP32, ≤1e-4 vs FP64); time-to-tol"
UNIT = "voxel-iterations/s"

# Algorithmic bytes per voxel and iteration of each kernel kind (summed over its
# launches in one iteration; complex64 = 8 B). fr holds layer fractions:
#   L   = sum over corrected axes of 2t*S_d/N_d,  L01 the same over axes 0 and 1,
#   sh  = fraction of voxels in any boundary layer, g01 = in an axis-0/1 layer.
#   When an axis-2 edge has a prime factor above 7 (Bluestein transforms) the
#   first pass does not compute E_2 x: the correction launches on x then cover
#   axis 2 too, and the first pass reads E x on every boundary-layer voxel.
def kernel_bytes_per_voxel(kind, fr):
    f = 8.0
    x_layers, first_layers = (fr["L01"], fr["g01"]) if fr["fused2"] else (fr["L"], fr["sh"])
    return {
        "corr_x": 2 * x_layers * f,            # layers of x in, E x out on them
        "rows_first": 3 * f + first_layers * f,  # x, B in, FFT buffer out, E x in on the layer voxels it needs
        "strided_fwd": 2 * f,
        "mid_axis0": 2 * f,
        "strided_inv": 2 * f,
        "rows_last": 4 * f,                    # FFT buffer, x, B in; x (or e on the layers) out
        # axis-0/1 layers of e in, E e out on them (axis 2 is computed inside the layer update)
        "corr_e": 2 * fr["L01"] * f,
        # e, x, B in and x out on the layer voxels; E_0 e + E_1 e in on the axis-0/1 layer rows
        "shell_update": 4 * fr["sh"] * f + fr["g01"] * f,
    }[kind]


def layer_fractions(info):
    t = info["t"]
    fd = [min(1.0, 2.0 * t * len(s) / sum(s)) if info["a"][d] > 0 else 0.0 for d, s in enumerate(info["sizes"])]
    sh = 1.0 - (1.0 - fd[0]) * (1.0 - fd[1]) * (1.0 - fd[2])
    g01 = 1.0 - (1.0 - fd[0]) * (1.0 - fd[1])

    def smooth7(v):
        for q in (2, 3, 5, 7):
            while v % q == 0:
                v //= q
        return v == 1

    fused2 = all(smooth7(n) for n in info["sizes"][2])
    return {"L": sum(fd), "L01": fd[0] + fd[1], "sh": sh, "g01": g01, "fused2": fused2}


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# dominant kernels, from ncu captures summarised under profiles/. The 1280^3
# workload is too large to capture under ncu's replay: its last pass is the
# 320^3 one-subdomain capture (the same kernel, per-voxel work and layer
# fractions) scaled by the 64 subdomains one launch covers.
MEASURED_TRAFFIC = {("C2", "rows_last"): 509084160, ("C2", "rows_first"): 418301696,
                    ("C5", "rows_last"): 64 * (786526464 + 247341568)}


def max_over_ranks(x, ws, device=None):
    """The largest x over the ranks: the job's time is its slowest rank's."""
    if ws <= 1:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, ws, seconds):
    """Units processed by all ranks (replicas of the same work) per second of the slowest rank."""
    return units_per_rank * ws / seconds


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clocks and throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < 3.0:  # the first sample before the timed region
                time.sleep(0.02)
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def build_problem(name):
    from synth import config_problem

    return config_problem(name)


# Bounded samples of a workload's recipe for the oracle on the host: the recipe
# on a sub-box with one subdomain of the workload's subdomain edge (wrap-removal
# corrections on every axis), so that the per-voxel work matches.
CPU_SAMPLE = {"C5": (320, 320, 320), "P43": (320, 320, 320), "C3": (128, 128, 128), "C2": (128, 128, 128), "C2P": (123, 123, 123),
              "C1": (64, 64, 64)}
REFERENCE_SAMPLE = (128, 128, 128)  # per step of the reference arm (a few seconds each)


def oracle_iterations(workload, shape, iters, warm):
    """The FP64 oracle as it stands: `warm` untimed then `iters` timed iterations of
    the workload's recipe on `shape` (one subdomain); returns (seconds, cpu seconds)."""
    import numpy as np

    from oracle import Problem
    from synth import config_problem

    params, n, src = config_problem(workload, shape=shape)
    periodic = params["periodic"]
    p = Problem(n, params["pixel"], params["wavelength"], widths=params["widths"], split=(1, 1, 1),
                periodic=periodic, t=params["t"])
    y = p.scaled_source(src)
    x = np.zeros(p.shape, dtype=complex)
    for _ in range(warm):
        x, _ = p.iteration(x, y)
    c0, t0 = time.process_time(), time.perf_counter()
    for _ in range(iters):
        x, _ = p.iteration(x, y)
    return time.perf_counter() - t0, time.process_time() - c0


def cpu_child(args):
    """Entry of the child process that times the oracle (its thread count is set
    in its environment before numpy loads): prints one JSON line."""
    shape = tuple(int(v) for v in args.cpu_shape.split("x"))
    dt, cpu = oracle_iterations(args.workload, shape, args.cpu_iters, 0)
    vox = float(shape[0] * shape[1] * shape[2])
    print(json.dumps({"value": vox * args.cpu_iters / dt, "seconds": dt, "cpu_seconds": cpu,
                      "shape": list(shape), "iters": args.cpu_iters}), flush=True)
    return 0


def run_cpu_child(workload, shape, iters, threads, timeout=900):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = str(threads)
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--cpu-child", "--workload", workload,
           "--cpu-shape", "x".join(map(str, shape)), "--cpu-iters", str(iters)]
    r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=timeout)
    if r.returncode != 0:
        return {"error": r.stderr[-500:]}
    return json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1])


def cpu_baseline(workload):
    """The oracle on all host cores and on one thread, on a bounded sample."""
    shape = CPU_SAMPLE.get(workload, (128, 128, 128))
    ncores = os.cpu_count() or 1
    allc = run_cpu_child(workload, shape, 1, ncores)
    one = run_cpu_child(workload, shape, 1, 1)
    if "error" in allc:
        return {"value": None, "unit": UNIT, "cores": ncores, "kind": "oracle", "error": allc["error"]}
    sample = ("%s recipe on a %s sub-box (one subdomain of the workload's subdomain edge, wrap-removal corrections "
              "on every axis), 1 MBS iteration of the FP64 numpy oracle, %.1f s" % (
                  workload, "x".join(map(str, shape)), allc["seconds"]))
    return {"value": allc["value"], "unit": UNIT, "cores": ncores, "kind": "oracle", "sample": sample,
            "nproc": ncores, "cpu_utilisation": allc["cpu_seconds"] / allc["seconds"],
            "threads_note": "OMP/OPENBLAS/MKL thread counts set to nproc; the oracle's FFT is numpy code, so only "
                            "its small matrix products can use more than one core",
            "single_thread": None if "error" in one else {"value": one["value"], "unit": UNIT, "cores": 1,
                                                          "seconds": one["seconds"]}}


def run_reference(args):
    """The oracle as it stands, timed on the host cores (rank 0 only): each step
    one MBS iteration of the workload's recipe on a 128^3 sub-box."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np

    from oracle import Problem
    from synth import config_problem

    shape = REFERENCE_SAMPLE
    params, n, src = config_problem(args.workload, shape=shape)
    p = Problem(n, params["pixel"], params["wavelength"], widths=params["widths"], split=(1, 1, 1),
                periodic=params["periodic"], t=params["t"])
    y = p.scaled_source(src)
    x = np.zeros(p.shape, dtype=complex)
    for _ in range(args.warmup):
        x, _ = p.iteration(x, y)
    c0, t0 = time.process_time(), time.perf_counter()
    for _ in range(args.steps):
        x, _ = p.iteration(x, y)
    dt = time.perf_counter() - t0
    cpu = time.process_time() - c0
    vox = float(np.prod(shape))
    v = vox * args.steps / dt
    ncores = os.cpu_count() or 1
    sample = ("one MBS iteration per step of the %s workload recipe on a %s sub-box (one subdomain, wrap-removal "
              "corrections on every axis), FP64 numpy oracle with numpy's default threading (%d host cores, "
              "CPU utilisation %.2f)" % (args.workload, "x".join(map(str, shape)), ncores, cpu / dt))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT[args.workload] + " (bounded CPU sample: %s sub-box)"
                       % "x".join(map(str, shape)), "grid": list(shape), "split": [1, 1, 1], "t": params["t"]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": ncores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_probe(args):
    """Per-kernel timing of one plan on a random medium (kernel studies and ncu
    captures of a chosen geometry): --probe N0xN1xN2 --probe-split S0xS1xS2
    [--probe-opts no_tma,force_tma,no_tune,corr_tf32]; 5 warm-up iterations,
    then K iterations one by one with CUDA events per kernel and K graph-replayed."""
    import torch

    import paper_2410_02395_gb300 as pkg

    shape = tuple(int(v) for v in args.probe.split("x"))
    split = tuple(int(v) for v in args.probe_split.split("x"))
    opts = {k: True for k in args.probe_opts.split(",") if k}
    g = torch.Generator(device="cuda").manual_seed(1)
    n = (1.0 + 0.5 * torch.rand(shape, generator=g, device="cuda")).to(torch.complex64)
    src = torch.zeros(shape, dtype=torch.complex64, device="cuda")
    src[tuple(v // 2 for v in shape)] = 1.0
    plan = pkg.Plan(shape, 0.25, 1.0, n, boundary_widths=((8, 8),) * 3, split=split, truncation=8, **opts)
    plan.set_source(src)
    plan.iterate(5, 0.0, no_poll=True)
    K = max(1, args.steps)
    prof = plan.profile(K)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    plan.iterate(K, 0.0, no_poll=True)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / K
    info = plan.info()
    print(json.dumps({"probe": list(shape), "split": list(split), "opts": sorted(opts), "ms_per_iter": ms,
                      "voxel_iterations_per_s": shape[0] * shape[1] * shape[2] / ms * 1e3,
                      "tuning": info["tuning"], "tma_groups": info["tma_groups"],
                      "kernels_ms_per_iter": {k: v[1] / K for k, v in prof.items()}}), flush=True)
    plan.close()
    return 0


def timed_iterations(plan, K, warmup, stream, dev, ws, torch, clocks=None):
    """CUDA-event milliseconds of K iterations (graph replays, no polling) after warm-up,
    max over ranks."""
    plan.iterate(max(warmup, 3), 0.0, no_poll=True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    if clocks is not None:
        clocks.start()
    ev0.record(stream)
    plan.iterate(K, 0.0, no_poll=True)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop() if clocks is not None else None
    ms = max_over_ranks(ev0.elapsed_time(ev1), ws, dev)
    if ws > 1:
        torch.distributed.barrier()
    return ms, clk


def error_vs_oracle(pkg, torch, dev, workload, shape=(96, 96, 96), iters=10):
    """Relative L2 distance (unsquared, and the paper's squared metric) of each form
    to the FP64 oracle at equal iteration counts, on the workload's recipe and
    split at a size the oracle runs in seconds."""
    from oracle import Problem, relative_l2
    from synth import config_problem

    params, n, src = config_problem(workload, shape=shape)
    kw = dict(widths=params["widths"], split=params["split"], periodic=params["periodic"], t=params["t"])
    ref = Problem(n, params["pixel"], params["wavelength"], **kw)
    xr, _, _ = ref.solve(src, tol=0.0, max_iter=iters)
    out = {"workload": "%s recipe on %s, split %s, %d iterations" % (
        workload, "x".join(map(str, shape)), "x".join(map(str, params["split"])), iters)}
    forms = {"fp32": {}, "mixed_3xtf32": {"corr_tf32": True}, "residual_form": {"residual_form": True},
             "plain_steps": {"plain_steps": True}}
    for name, fkw in forms.items():
        plan = pkg.Plan(shape, params["pixel"], params["wavelength"], torch.from_numpy(n).to(dev),
                        boundary_widths=params["widths"], split=params["split"], truncation=params["t"],
                        periodic=params["periodic"], **fkw)
        x, it, _ = plan.solve(torch.from_numpy(src).to(dev), tol=0.0, max_iter=iters)
        e = relative_l2(x.cpu().numpy(), xr)
        out[name] = {"rel_l2": e, "rel_l2_squared": e * e, "iterations": it}
        plan.close()
    return out


def cufft_comparison(torch, dev, info, prof, K, reps=5):
    """The vendor FFT (cuFFT through torch.fft) on the same subdomains, timed here
    only for comparison (the library never calls it): batched 3-D C2C forward
    transform, pointwise propagator-like multiply, inverse transform, against the
    CUDA-event time of the library's five transform passes of one iteration (which
    also carry the fused medium, source, correction and update work)."""
    sizes = info["sizes"]
    if any(len(set(s)) != 1 for s in sizes):
        return None  # uneven subdomains: no single batched transform
    nsub = len(sizes[0]) * len(sizes[1]) * len(sizes[2])
    shp = (nsub, sizes[0][0], sizes[1][0], sizes[2][0])
    g = torch.Generator(device=dev).manual_seed(7)
    a = torch.complex(torch.randn(shp, generator=g, device=dev), torch.randn(shp, generator=g, device=dev))
    mul = torch.complex(torch.rand(shp[1:], generator=g, device=dev), torch.rand(shp[1:], generator=g, device=dev))
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    fwd = inv = both = 0.0
    for r in range(reps + 2):
        ev[0].record()
        b = torch.fft.fftn(a, dim=(1, 2, 3))
        ev[1].record()
        b.mul_(mul)
        ev[2].record()
        c = torch.fft.ifftn(b, dim=(1, 2, 3))
        ev[3].record()
        torch.cuda.synchronize(dev)
        del b, c
        if r >= 2:
            fwd += ev[0].elapsed_time(ev[1]) / reps
            inv += ev[2].elapsed_time(ev[3]) / reps
            both += ev[0].elapsed_time(ev[3]) / reps
    del a, mul
    torch.cuda.empty_cache()
    ours = sum(prof[k][1] for k in ("rows_first", "strided_fwd", "mid_axis0", "strided_inv", "rows_last")) / K
    return {"batch": list(shp), "cufft_fwd_ms": fwd, "cufft_inv_ms": inv, "cufft_fwd_mul_inv_ms": both,
            "library_transform_passes_ms": ours,
            "ratio_library_over_cufft": ours / both if both > 0 else None,
            "how": "torch.fft.fftn / ifftn (cuFFT) on a contiguous batch of the subdomains, out of place, CUDA "
                   "events, %d repetitions after 2; the library's passes read and write the subdomains inside the "
                   "global grid and fuse the medium, source, corrections and update" % reps}


def activation_comparison(pkg, torch, dev, shape=(1024, 128, 128), split=(8, 1, 1), tol=1e-4, max_iter=40000):
    """Subdomain activation (Sec. 3.1): time to tolerance with and without it on a
    long domain (256 wavelengths along axis 0 at lambda/4, 8 subdomains of 128^3,
    the C2 sphere recipe, 8-px layers, t = 8) with the point source in the first
    subdomain, far from the others. Both solves are timed from mbs_set_source to
    the stop (x form, FP32 corrections)."""
    from synth import point_source, spheres_medium

    n = spheres_medium(shape, count=40, r_range=(4, 20), n_range=(1.0, 1.6), seed=106, margin=8)
    src = point_source(shape, (64, shape[1] // 2, shape[2] // 2))
    n_dev = torch.from_numpy(n).to(dev)
    s_dev = torch.from_numpy(src).to(dev)
    out = {"workload": "%s grid, split %s, t=8, 40 spheres, 8-px layers, point source at (64, %d, %d)" % (
        "x".join(map(str, shape)), "x".join(map(str, split)), shape[1] // 2, shape[2] // 2), "tol": tol}
    for name, kw in (("without", {}), ("with", {"activation": True})):
        p = pkg.Plan(shape, 0.25, 1.0, n_dev, boundary_widths=((8, 8),) * 3, split=split, truncation=8, **kw)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        p.set_source(s_dev)
        st, it, eps = p.iterate(max_iter, tol)
        torch.cuda.synchronize(dev)
        out[name] = {"status": st, "iterations": it, "residual": eps, "seconds": time.perf_counter() - t0}
        p.close()
    out["speedup"] = out["without"]["seconds"] / out["with"]["seconds"]
    del n_dev, s_dev
    torch.cuda.empty_cache()
    return out


def workload_values(pkg, torch, dev, names, steps, warmup, ws):
    """Device-timed value (and the mixed form's) of other single-grid workloads."""
    import numpy as np

    out = {}
    for name in names:
        params, n, src = build_problem(name)
        shape = params["shape"]
        vox = int(np.prod(shape))
        stream = torch.cuda.Stream(device=dev)
        n_dev = torch.from_numpy(n).to(dev)
        src_dev = torch.from_numpy(src).to(dev)
        rec = {"workload": WORKLOAD_TEXT[name]}
        for form, fkw in (("value", {}), ("mixed", {"corr_tf32": True})):
            with torch.cuda.stream(stream):
                p = pkg.Plan(shape, params["pixel"], params["wavelength"], n_dev, boundary_widths=params["widths"],
                             split=params["split"], truncation=params["t"], periodic=params["periodic"],
                             stream=stream.cuda_stream, **fkw)
                G = p.info()["graph_iters"]
                K = max(G, (max(steps, 100) // G) * G)
                p.set_source(src_dev)
                ms, _ = timed_iterations(p, K, warmup, stream, dev, ws, torch)
                p.close()
            rec[form] = whole_job_rate(vox * K, ws, ms / 1e3)
            rec[form + "_ms_per_step"] = ms / K
        out[name] = rec
        del n_dev, src_dev
        torch.cuda.empty_cache()
    return out


def run_batch(args, pkg, torch, ws, rank, dev):
    """The C4 workload: 64 solves advanced together by one graph per G iterations,
    against the same solves advanced one after another."""
    import numpy as np

    from synth import frequency_batch

    problems = frequency_batch(count=64, seed=104)
    stream = torch.cuda.Stream(device=dev)
    plans = []
    for params, n, src in problems:
        p = pkg.Plan(params["shape"], params["pixel"], params["wavelength"], torch.from_numpy(n).to(dev),
                     boundary_widths=params["widths"], split=params["split"], truncation=params["t"],
                     periodic=params["periodic"], split_sizes=params["split_sizes"])
        p.set_source(torch.from_numpy(src).to(dev))
        plans.append(p)
    vox = sum(int(np.prod(pp["shape"])) for pp, _, _ in problems)
    G = 10
    K = max(G, (args.steps // 10 // G) * G)
    b = pkg.Batch(plans, stream=stream.cuda_stream, graph_iters=G)
    b.iterate(max(args.warmup, 3), 0.0, no_poll=True)
    n_launch, fused = b.launches_per_iteration()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(dev.index)
    torch.cuda.synchronize(dev)
    clocks.start()
    ev0.record(stream)
    b.iterate(K, 0.0, no_poll=True)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1), ws, dev)
    value = whole_job_rate(vox * K, ws, ms / 1e3)
    # the other form of the batch (fused <-> graph of every plan's own launches)
    other = None
    b.set_fused(not fused)
    b.iterate(max(args.warmup, 3), 0.0, no_poll=True)
    n_launch2, fused2 = b.launches_per_iteration()
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    b.iterate(K, 0.0, no_poll=True)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    ms2 = max_over_ranks(ev0.elapsed_time(ev1), ws, dev)
    other = {"value": whole_job_rate(vox * K, ws, ms2 / 1e3), "unit": UNIT, "ms_per_step": ms2 / K, "fused": fused2,
             "launches_per_iteration": n_launch2}
    b.set_fused(fused)
    # the same solves one after another, each with its own graph replays
    t0 = time.perf_counter()
    for p in plans:
        p.iterate(K, 0.0, no_poll=True)
    torch.cuda.synchronize(dev)
    seq = time.perf_counter() - t0
    # time to tolerance of all 64 solves (residual form), batched
    ttt = None
    if not args.no_ttt:
        rplans = []
        for params, n, src in problems:
            p = pkg.Plan(params["shape"], params["pixel"], params["wavelength"], torch.from_numpy(n).to(dev),
                         boundary_widths=params["widths"], split=params["split"], truncation=params["t"],
                         periodic=params["periodic"], split_sizes=params["split_sizes"], residual_form=True)
            rplans.append(p)
        rb = pkg.Batch(rplans, graph_iters=G)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for p, (_, _, src) in zip(rplans, problems):
            p.set_source(torch.from_numpy(src).to(dev))
        res = rb.iterate(args.ttt_max_iter, problems[0][0]["tol"])
        torch.cuda.synchronize(dev)
        ttt = {"tol": problems[0][0]["tol"], "seconds": time.perf_counter() - t0,
               "converged": sum(1 for r in res if r[0] == "MBS_OK"), "solves": len(res),
               "iterations_max": max(r[1] for r in res), "iterations_min": min(r[1] for r in res),
               "form": "residual form, FP32 corrections, one batch"}
        rb.close()
        for p in rplans:
            p.close()
    b.close()
    for p in plans:
        p.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": args.warmup,
                "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "c64", "data": "synthetic",
                "config": {"workload": WORKLOAD_TEXT["C4"], "solves": len(problems), "voxels": vox,
                           "l2": "no flush: %.0f MB per field summed over the solves (> 129 MB L2)" % (vox * 8 / 1e6),
                           "parallelism": "replicas" if ws > 1 else "single GPU", "graph_iters": G},
                "clocks": clk,
                "gpu_launches": n_launch * K,
                "batch": {"fused": fused, "launches_per_iteration": n_launch,
                          "how": "one launch per pass and subdomain edge over the solves of each cluster "
                                 "(solves sharing an edge), clusters side by side" if fused else
                                 "one graph of every solve's own launches on forked streams"},
                "other_form": other,
                "sequential": {"value": vox * K / seq, "unit": UNIT,
                               "how": "the same 64 solves one after another, each with its own graph replays"},
                "time_to_tol": ttt}
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--e2e-iters", type=int, default=20, help="iterations per mbs_solve call in the e2e leg")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-error", action="store_true", help="skip the error-vs-oracle leg")
    ap.add_argument("--no-extra", action="store_true", help="skip the other single-grid workloads (C2, C3)")
    ap.add_argument("--no-activation", action="store_true", help="skip the subdomain-activation comparison")
    ap.add_argument("--ttt", action="store_true", help="run the time-to-tolerance leg (long at 1280^3)")
    ap.add_argument("--no-ttt", action="store_true", help="skip the time-to-tolerance leg of C4")
    ap.add_argument("--ttt-max-iter", type=int, default=40000)
    ap.add_argument("--ttt-chunk", type=int, default=0, help="print the --ttt leg's progress every N iterations")
    ap.add_argument("--ttt-history", default="", help="file (.npy) for the residual history of the --ttt leg")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOAD_TEXT),
                    help="benchmark workload (default: the 1280^3 configuration C5)")
    ap.add_argument("--no-mixed", action="store_true", help="skip the 3xTF32-correction timing")
    ap.add_argument("--t-sweep", default="", help="comma-separated truncation widths: ms per iteration for each "
                    "on the same workload (Sec. 4.2.1, Fig. 7c)")
    ap.add_argument("--probe", default="", help="per-kernel timing of one plan of this grid (N0xN1xN2)")
    ap.add_argument("--probe-split", default="1x1x1")
    ap.add_argument("--probe-opts", default="", help="comma-separated Plan flags, e.g. no_tma,force_tma")
    ap.add_argument("--cpu-child", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--cpu-shape", default="128x128x128", help=argparse.SUPPRESS)
    ap.add_argument("--cpu-iters", type=int, default=1, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.cpu_child:
        return cpu_child(args)
    if args.probe:
        return run_probe(args)
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    import paper_2410_02395_gb300 as pkg

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    assert args.warmup >= 3, "at least 3 warm-up steps"

    if args.workload == "C4":
        return run_batch(args, pkg, torch, ws, rank, dev)
    params, n, src = build_problem(args.workload)
    shape = params["shape"]
    vox = int(np.prod(shape))
    stream = torch.cuda.Stream(device=dev)
    n_dev = torch.from_numpy(n).to(dev)
    src_dev = torch.from_numpy(src).to(dev)
    kw = dict(boundary_widths=params["widths"], split=params["split"], truncation=params["t"],
              periodic=params["periodic"], stream=stream.cuda_stream)
    if params.get("split_sizes"):
        kw["split_sizes"] = params["split_sizes"]
    with torch.cuda.stream(stream):
        plan = pkg.Plan(shape, params["pixel"], params["wavelength"], n_dev, **kw)
        info = plan.info()
        G = info["graph_iters"]
        K = max(G, (args.steps // G) * G)  # whole graph replays
        plan.set_source(src_dev)

        # ---- device-resident timed region -------------------------------------
        ms, clk = timed_iterations(plan, K, args.warmup, stream, dev, ws, torch, ClockSampler(dev.index))
        value = whole_job_rate(vox * K, ws, ms / 1e3)

        # ---- per-kernel CUDA-event timing (same workload, kernels launched one by one)
        prof = plan.profile(K)
        launches_per_iter = sum(v[0] for v in prof.values()) / K
        tot = sum(v[1] for v in prof.values())
        dom = max(prof, key=lambda k: prof[k][1])
        fr = layer_fractions(info)
        peak, peak_src = read_peaks()
        dom_launches, dom_ms = prof[dom]
        bytes_per_launch = kernel_bytes_per_voxel(dom, fr) * vox / max(1.0, dom_launches / K)
        achieved = bytes_per_launch / (dom_ms / dom_launches / 1e3) / 1e9
        bytes_iter = sum(kernel_bytes_per_voxel(k, fr) for k in prof) * vox
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": MEASURED_TRAFFIC.get((args.workload, dom)), "kernel": dom, "peak_source": peak_src,
                    "share": prof[dom][1] / tot if tot else None,
                    "bytes_per_launch": bytes_per_launch,
                    "iteration": {"bytes_per_voxel": bytes_iter / vox,
                                  "GBps_graph_replayed": bytes_iter / (ms / K / 1e3) / 1e9,
                                  "frac_graph_replayed": bytes_iter / (ms / K / 1e3) / 1e9 / peak},
                    "kernels": {k: {"launches": v[0], "ms_per_iter": v[1] / K,
                                    "bytes_per_voxel": kernel_bytes_per_voxel(k, fr),
                                    "GBps": (kernel_bytes_per_voxel(k, fr) * vox * K / (v[1] / 1e3) / 1e9)
                                    if v[1] > 0 else None} for k, v in prof.items()}}

        # ---- end to end through the C ABI with pinned host buffers ------------
        e2e = None
        if not args.no_e2e:
            hsrc = torch.from_numpy(src).pin_memory()
            hout = torch.empty(shape, dtype=torch.complex64).pin_memory()
            plan.solve(hsrc, tol=0.0, max_iter=args.e2e_iters, out=hout)  # warm
            torch.cuda.synchronize(dev)
            if ws > 1:
                torch.distributed.barrier()
            t0 = time.perf_counter()
            for _ in range(args.e2e_steps):
                plan.solve(hsrc, tol=0.0, max_iter=args.e2e_iters, out=hout)
            dt = max_over_ranks(time.perf_counter() - t0, ws, dev)
            e2e = {"value": whole_job_rate(vox * args.e2e_iters * args.e2e_steps, ws, dt), "unit": UNIT,
                   "h2d_bytes_per_step": vox * 8, "d2h_bytes_per_step": vox * 8 + 8 * args.e2e_iters,
                   "step": "one mbs_solve call: pinned host source -> device, %d iterations, field -> pinned host"
                           % args.e2e_iters}
            del hsrc, hout
        plan.close()

        # ---- the mixed form: 3xTF32 tensor-core edge corrections ---------------
        mixed = None
        if not args.no_mixed and info["a"] != [0, 0, 0]:
            pm = pkg.Plan(shape, params["pixel"], params["wavelength"], n_dev, corr_tf32=True, **kw)
            pm.set_source(src_dev)
            msm, _ = timed_iterations(pm, K, args.warmup, stream, dev, ws, torch)
            pm.close()
            mixed = {"value": whole_job_rate(vox * K, ws, msm / 1e3), "unit": UNIT, "ms_per_step": msm / K,
                     "corrections": "3xTF32 mma.sync m16n8k8, FP32 accumulate"}

        # ---- the plain form: one launch per step, residual and stop test on the host
        Kp = max(5, K // 4)
        pp = pkg.Plan(shape, params["pixel"], params["wavelength"], n_dev, plain_steps=True, **kw)
        pp.set_source(src_dev)
        msp, _ = timed_iterations(pp, Kp, args.warmup, stream, dev, ws, torch)
        pp.close()
        plain = {"value": whole_job_rate(vox * Kp, ws, msp / 1e3), "unit": UNIT, "ms_per_step": msp / Kp,
                 "steps": Kp, "how": "MBS_FLAG_PLAIN_STEPS: every step of the iteration its own launch (about 16 "
                                     "per iteration), FP32 corrections on the CUDA cores, no CUDA graph, residual "
                                     "summed and stop test taken on the host after every iteration"}

        # ---- the same iterations launched kernel by kernel from the host -----
        Kn = max(10, K // 2)
        pn = pkg.Plan(shape, params["pixel"], params["wavelength"], n_dev, no_graph=True, **kw)
        pn.set_source(src_dev)
        msn, _ = timed_iterations(pn, Kn, args.warmup, stream, dev, ws, torch)
        pn.close()
        no_graph = {"value": whole_job_rate(vox * Kn, ws, msn / 1e3), "unit": UNIT, "ms_per_step": msn / Kn,
                    "steps": Kn, "how": "same kernels, launched one by one from the host (MBS_FLAG_NO_GRAPH)"}

        # ---- time to tolerance (residual form: no complex64 floor) -----------
        ttt_line = None
        if args.ttt:
            pr = pkg.Plan(shape, params["pixel"], params["wavelength"], n_dev, residual_form=True, **kw)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            pr.set_source(src_dev)
            if args.ttt_chunk > 0:  # progress on stderr every ttt_chunk iterations (same solve)
                it_tol = 0
                while it_tol < args.ttt_max_iter:
                    st_tol, it_tol, eps_tol = pr.iterate(min(args.ttt_chunk, args.ttt_max_iter - it_tol),
                                                         params["tol"])
                    print(json.dumps({"iterations": it_tol, "residual": eps_tol, "status": st_tol,
                                      "seconds": time.perf_counter() - t0}), file=sys.stderr, flush=True)
                    if st_tol != "MBS_ENOCONV":
                        break
            else:
                st_tol, it_tol, eps_tol = pr.iterate(args.ttt_max_iter, params["tol"])
            torch.cuda.synchronize(dev)
            secs = time.perf_counter() - t0
            ttt_line = {"tol": params["tol"], "status": st_tol, "iterations": it_tol, "residual": eps_tol,
                        "seconds": secs, "form": "residual form, FP32 corrections"}
            hist = pr.history(it_tol)
            if args.ttt_history:
                np.save(args.ttt_history, hist)
            if st_tol != "MBS_OK" and len(hist) >= 200:
                # extrapolation from the residual's slope over the last half of the run (log eps linear in n)
                h = np.log(np.maximum(hist, 1e-300))
                k = np.arange(len(h))
                half = len(h) // 2
                slope, icpt = np.polyfit(k[half:], h[half:], 1)
                if slope < 0:
                    n_tol = int(np.ceil((np.log(params["tol"]) - icpt) / slope))
                    ttt_line["extrapolated"] = {
                        "iterations": n_tol, "seconds": secs / it_tol * n_tol,
                        "how": "log eps fitted linearly over iterations %d-%d (slope %.3e per iteration); an "
                               "extrapolation, not a measurement" % (half, len(h) - 1, slope)}
            pr.close()

        # ---- truncation sweep: iteration time against t ------------------------
        tsweep = None
        if args.t_sweep:
            tsweep = []
            for tv in [int(v) for v in args.t_sweep.split(",") if v]:
                kt = dict(kw, truncation=tv)
                pt = pkg.Plan(shape, params["pixel"], params["wavelength"], n_dev, **kt)
                pt.set_source(src_dev)
                Kt = max(10, K // 4)
                mst, _ = timed_iterations(pt, Kt, args.warmup, stream, dev, ws, torch)
                tsweep.append({"t": tv, "ms_per_step": mst / Kt, "c_abs": abs(pt.info()["c"])})
                pt.close()
    del n_dev, src_dev, n, src
    torch.cuda.empty_cache()
    cufft = cufft_comparison(torch, dev, info, prof, K)

    error = None
    if rank == 0 and not args.no_error:
        error = error_vs_oracle(pkg, torch, dev, args.workload)
    extra = None
    if not args.no_extra and args.workload == "C5":
        extra = workload_values(pkg, torch, dev, ["C2", "C3"], args.steps, args.warmup, ws)
    activation = None
    if rank == 0 and not args.no_activation and args.workload == "C5":
        activation = activation_comparison(pkg, torch, dev)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": args.warmup,
            "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64", "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT[args.workload],
                       "grid": list(shape), "split": list(params["split"]), "t": params["t"],
                       "l2": ("no flush: x, B and the FFT buffer are %.0f MB each (> 129 MB L2)" % (vox * 8 / 1e6))
                       if vox * 8 > 129e6 else
                       ("working set of %.0f MB fits in L2 (not flushed): not a DRAM-bound measurement"
                        % (5 * vox * 8 / 1e6)),
                       "parallelism": "replicas" if ws > 1 else "single GPU",
                       "graph_iters": G},
            "clocks": clk,
            "gpu_launches": int(round(launches_per_iter * K)) + 1,
            "roofline": roofline,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "mixed": mixed,
            "plain": plain,
            "cufft": cufft,
            "no_graph": no_graph,
            "error": error,
            "workloads": extra,
            "activation": activation,
            "time_to_tol": ttt_line,
        }
        if args.t_sweep:
            line["t_sweep"] = tsweep
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
