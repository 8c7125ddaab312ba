#!/usr/bin/env python3
"""Benchmark of the MBS hot path: voxel-iterations per second on one GB300.

Workload (default): the domain-decomposed MBS problem on a 256^3 grid at
lambda/4, split 2x2x2 into 128^3 subdomains with t = 8 edge corrections, 40
seeded random spheres (radius 4-20 px, n in [1.0, 1.6]) in n = 1.0, 8-px
absorbing layers, point source at the centre. One step = one iteration of
Eq. wavesim_iter over the whole grid (all subdomains).

Printed JSON line (one, from rank 0):
  value       voxel-iterations/s with every buffer resident in HBM, timed with
              CUDA events on the plan's stream over K graph-replayed iterations
  e2e         the same metric through the C ABI call mbs_solve with pinned host
              source/output buffers, host<->device copies inside the timed region
  roofline    the dominant kernel's algorithmic bytes per launch / its average
              CUDA-event duration, against the measured HBM copy bandwidth
  cpu_baseline the FP64 oracle timed on the host cores on a bounded sample

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

WORKLOAD = "C2"
WORKLOAD_TEXT = {
    "C1": "C1: 64^3 grid at lambda/4, one periodic subdomain, 6 spheres, 8-px absorbing layers, point source",
    "C2": "C2: 256^3 grid at lambda/4, 2x2x2 subdomains of 128^3, t=8, 40 spheres, 8-px absorbing layers, point source",
    "C3": "C3: 512^3 grid at lambda/4, 4x4x4 subdomains of 128^3, t=8, n = 1.33 + Gaussian random field, "
          "Gaussian-beam plane source",
    "C4": "C4: 64 independent frequency solves, lambda uniform in [0.8,1.2] on one 24-unit box at lambda/4 "
          "(grids 80^3-120^3), each split 2x2x2 into 7-smooth halves, t=8, same spheres, point sources; "
          "one CUDA graph over all solves",
    "C5": "C5: 1280^3 grid at lambda/4, 4x4x4 subdomains of 320^3, t=8, spheres to 30% fill, point source",
    "C2P": "C2P: the C2 recipe on a 246^3 grid, 2x2x2 subdomains of 123^3 (123 = 3 x 41: Bluestein transforms "
           "on every axis), t=8",
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
# kernels that dominate the 256^3 workload, from one ncu capture of the current
# kernels (summarised under profiles/).
MEASURED_TRAFFIC = {("C2", "rows_last"): 509084160, ("C2", "rows_first"): 418301696}


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


def cpu_oracle_sample(iters=3, shape=(128, 128, 128)):
    """The FP64 oracle on the workload's recipe at a reduced grid (bounded sample)."""
    import numpy as np

    from oracle import Problem
    from synth import config_problem

    params, n, src = config_problem(WORKLOAD, shape=shape)
    p = Problem(n, params["pixel"], params["wavelength"], widths=params["widths"], split=params["split"],
                periodic=params["periodic"], t=params["t"])
    y = p.scaled_source(src)
    x = np.zeros(p.shape, dtype=complex)
    x, _ = p.iteration(x, y)  # untimed warm-up
    t0 = time.perf_counter()
    for _ in range(iters):
        x, _ = p.iteration(x, y)
    dt = time.perf_counter() - t0
    vox = float(np.prod(shape))
    return vox * iters / dt, dt, "C2 recipe (spheres, 8-px layers, point source, split 2x2x2, t=8) on a %s grid " \
                                 "(subdomains %s), %d iterations after 1 warm-up, %.1f s" % (
                                     "x".join(map(str, shape)), "x".join(str(s // 2) for s in shape), iters, dt)


def run_reference(args):
    """The oracle as it stands, timed on the host cores (rank 0 only)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import numpy as np

    from oracle import Problem
    from synth import config_problem

    shape = (128, 128, 128)
    params, n, src = config_problem(WORKLOAD, shape=shape)
    p = Problem(n, params["pixel"], params["wavelength"], widths=params["widths"], split=params["split"],
                periodic=params["periodic"], t=params["t"])
    y = p.scaled_source(src)
    x = np.zeros(p.shape, dtype=complex)
    for _ in range(args.warmup):
        x, _ = p.iteration(x, y)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        x, _ = p.iteration(x, y)
    dt = time.perf_counter() - t0
    vox = float(np.prod(shape))
    v = vox * args.steps / dt
    sample = ("one MBS iteration per step of the %s workload recipe on a 128^3 grid (split 2x2x2, t=8), "
              "FP64 numpy oracle, single thread" % WORKLOAD)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": {"workload": "C2 recipe at 128^3 (bounded CPU sample of the 256^3 C2 workload)",
                       "grid": list(shape), "split": [2, 2, 2], "t": 8},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


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
                "sequential": {"value": vox * K / seq, "unit": UNIT,
                               "how": "the same 64 solves one after another, each with its own graph replays"},
                "time_to_tol": ttt}
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--e2e-iters", type=int, default=100, help="iterations per mbs_solve call in the e2e leg")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-ttt", action="store_true", help="skip the time-to-tolerance leg")
    ap.add_argument("--ttt-max-iter", type=int, default=40000)
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOAD_TEXT),
                    help="benchmark workload (default: the C2 configuration)")
    ap.add_argument("--no-mixed", action="store_true", help="skip the 3xTF32-correction timing")
    ap.add_argument("--t-sweep", default="", help="comma-separated truncation widths: ms per iteration for each "
                    "on the same workload (Sec. 4.2.1, Fig. 7c)")
    args = ap.parse_args()
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
    with torch.cuda.stream(stream):
        plan = pkg.Plan(shape, params["pixel"], params["wavelength"], torch.from_numpy(n).to(dev),
                        boundary_widths=params["widths"], split=params["split"], truncation=params["t"],
                        periodic=params["periodic"], stream=stream.cuda_stream)
        info = plan.info()
        G = info["graph_iters"]
        K = max(G, (args.steps // G) * G)  # whole graph replays
        src_dev = torch.from_numpy(src).to(dev)
        plan.set_source(src_dev)
        plan.iterate(max(args.warmup, 3), 0.0, no_poll=True)

        # ---- device-resident timed region -------------------------------------
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        clocks = ClockSampler(dev.index)
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        clocks.start()
        ev0.record(stream)
        status, iters_done, eps = plan.iterate(K, 0.0, no_poll=True)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        clk = clocks.stop()
        ms = max_over_ranks(ev0.elapsed_time(ev1), ws, dev)
        if ws > 1:
            torch.distributed.barrier()
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
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": MEASURED_TRAFFIC.get((args.workload, dom)), "kernel": dom, "peak_source": peak_src,
                    "share": prof[dom][1] / tot if tot else None,
                    "bytes_per_launch": bytes_per_launch,
                    "kernels": {k: {"launches": v[0], "ms_per_iter": v[1] / K,
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

        plan.close()
        n_dev = torch.from_numpy(n).to(dev)
        kw = dict(boundary_widths=params["widths"], split=params["split"], truncation=params["t"],
                  periodic=params["periodic"], stream=stream.cuda_stream)

        # ---- the mixed form: 3xTF32 tensor-core edge corrections ---------------
        mixed = None
        if not args.no_mixed and info["a"] != [0, 0, 0]:
            pm = pkg.Plan(shape, params["pixel"], params["wavelength"], n_dev, corr_tf32=True, **kw)
            pm.set_source(src_dev)
            pm.iterate(max(args.warmup, 3), 0.0, no_poll=True)
            if ws > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize(dev)
            ev0.record(stream)
            pm.iterate(K, 0.0, no_poll=True)
            ev1.record(stream)
            torch.cuda.synchronize(dev)
            msm = max_over_ranks(ev0.elapsed_time(ev1), ws, dev)
            pm.close()
            mixed = {"value": whole_job_rate(vox * K, ws, msm / 1e3), "unit": UNIT, "ms_per_step": msm / K,
                     "corrections": "3xTF32 mma.sync m16n8k8, FP32 accumulate"}

        # ---- the same iterations launched kernel by kernel from the host -----
        # (no CUDA graph: one launch per pass and iteration, host launch cost included)
        Kn = max(10, K // 10)
        pn = pkg.Plan(shape, params["pixel"], params["wavelength"], n_dev, no_graph=True, **kw)
        pn.set_source(src_dev)
        pn.iterate(max(args.warmup, 3), 0.0, no_poll=True)
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        pn.iterate(Kn, 0.0, no_poll=True)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        msn = max_over_ranks(ev0.elapsed_time(ev1), ws, dev)
        pn.close()
        no_graph = {"value": whole_job_rate(vox * Kn, ws, msn / 1e3), "unit": UNIT, "ms_per_step": msn / Kn,
                    "steps": Kn, "how": "same kernels, launched one by one from the host (MBS_FLAG_NO_GRAPH)"}

        # ---- time to tolerance (residual form: no complex64 floor) -----------
        ttt_line = None
        if not args.no_ttt:
            pr = pkg.Plan(shape, params["pixel"], params["wavelength"], n_dev, residual_form=True, **kw)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            pr.set_source(src_dev)
            st_tol, it_tol, eps_tol = pr.iterate(args.ttt_max_iter, params["tol"])
            torch.cuda.synchronize(dev)
            ttt_line = {"tol": params["tol"], "status": st_tol, "iterations": it_tol, "residual": eps_tol,
                        "seconds": time.perf_counter() - t0, "form": "residual form, FP32 corrections"}
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
                pt.iterate(max(args.warmup, 3), 0.0, no_poll=True)
                torch.cuda.synchronize(dev)
                ev0.record(stream)
                pt.iterate(Kt, 0.0, no_poll=True)
                ev1.record(stream)
                torch.cuda.synchronize(dev)
                tsweep.append({"t": tv, "ms_per_step": ev0.elapsed_time(ev1) / Kt, "c_abs": abs(pt.info()["c"])})
                pt.close()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        os.environ.setdefault("OMP_NUM_THREADS", "1")
        v, dt, sample = cpu_oracle_sample()
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}

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
            "no_graph": no_graph,
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
