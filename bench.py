#!/usr/bin/env python3
"""Benchmark of the BME Godunov step on one or more GB300s.

Workload: the 3D turbulent periodic box, 256^3 cells, FP32 arithmetic (lognormal density,
k^-2 Gaussian random velocity, random SPD stress per cell; seeded synthetic input).  One
bench step = one full step of the hot path (boundary mapping, reconstruction, HLL fluxes
in x/y/z, unsplit update, CFL reduction, FP64 totals, realizability) on the whole grid.

Metric: cell-updates/s (whole job; N ranks each advance their own replica of the box, so
scaling is weak).  `value` is device time with the state resident in HBM (the 671 MB FP32
state is larger than the 129 MB L2, so no flush is needed between steps); `e2e` is the
same metric through the public C ABI with host buffers (pinned upload of the state, one
step, download of the result, every step).  `roofline` relates the step kernel's
algorithmic bytes (read U^n + write U^{n+1}: 80 B per cell in FP32) per launch to its
CUDA-event duration and the measured HBM bandwidth.

--impl reference times the FP64 CPU oracle on the same workload, full grid, every step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_BOX = 256
DATA = {"box": "synthetic (seeded k^-2 Gaussian random fields)",
        "blast": "synthetic (seeded 1% density noise)", "disc": "synthetic (seeded 1% density perturbation)"}
# name -> (cells per axis, description, timed kernel)
WORKLOADS = {
    "box": (256, "turbulent periodic box {n}^3, FP32, CFL 0.5", "step_tile_kernel<float,3>"),
    "blast": (1024, "anisotropic-stress blast {n}^2 periodic, FP32, CFL 0.5", "step_strip2d_kernel<float>"),
    "disc": (512, "stellar disc {n}^2 in a logarithmic potential, outflow, FP32, CFL 0.5",
             "step_strip2d_kernel<float>"),
}
BYTES_PER_CELL = {"f32": 80, "f64": 160}   # read U^n + write U^{n+1}, 10 fields each
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "step_tile_fp32_turb256.md")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="box", choices=sorted(WORKLOADS),
                    help="box: 3D turbulent box (the benchmark); blast, disc: the 2D workloads")
    ap.add_argument("--n", type=int, default=None, help="cells per axis (default: the workload's)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--fp32-only", action="store_true", help="skip the FP64 measurement")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the adjoint (disc 512^2 x 2000 steps) and batched-tubes measurements")
    ap.add_argument("--tiling", default=None, help="rows,zchunk instead of autotuning (e.g. 8,32)")
    ap.add_argument("--persistent-only", action="store_true",
                    help="with --suite --only tubes: skip the one-launch-per-step-per-tube baseline")
    ap.add_argument("--ctu", action="store_true",
                    help="the corner-transport-upwind form of the step (a profiling case, not the benchmark)")
    ap.add_argument("--suite", action="store_true", help="one JSON line per workload instead of the bench line")
    ap.add_argument("--only", default=None, choices=["sod", "blast", "box", "schemes", "ctu", "selfgrav", "tubes", "disc"],
                    help="with --suite: run one workload (--n and --steps then size it)")
    return ap.parse_args()


def dist_env():
    from paper_1210_5246_gb300 import replicas
    return replicas.dist_env()


def _code_only(text):
    """Source text without // comments and blank lines (a comment edit does not change the
    compiled kernel, so it keeps the record valid)."""
    out = []
    for line in text.splitlines():
        code = re.sub(r"//.*$", "", line).rstrip()
        if code:
            out.append(code)
    return "\n".join(out)


def kernel_source_hash():
    """Hash of the code the 3D step kernel is compiled from: the per-cell arithmetic
    (msh_device.cuh) and msh_step_kernels.cuh up to the 2D kernel (helpers and
    step_tile_kernel), comments left out."""
    csrc = os.path.join(ROOT, "paper_1210_5246_gb300", "csrc")
    step = open(os.path.join(csrc, "msh_step_kernels.cuh")).read()
    cut = step.find("// ---------------------------------------------------------------- 2D kernel")
    h = hashlib.sha256()
    h.update(_code_only(open(os.path.join(csrc, "msh_device.cuh")).read()).encode())
    h.update(_code_only(step[: cut if cut >= 0 else len(step)]).encode())
    return h.hexdigest()[:16]


def traffic_record():
    """The step kernel's ncu record in the committed summary (DRAM bytes and warp
    instructions per cell); None if absent or taken on different kernel sources."""
    try:
        txt = open(PROFILE_SUMMARY).read()
    except OSError:
        return None
    rec = None
    for line in txt.splitlines():
        if line.startswith("traffic_record:"):
            rec = json.loads(line.split(":", 1)[1])
    if not rec or rec.get("source_hash") != kernel_source_hash():
        return None
    return rec


def measured_traffic(n_cells):
    """DRAM bytes per launch of the step kernel from the committed ncu summary, scaled to
    the workload's cell count; None if absent or taken on different kernel sources."""
    rec = traffic_record()
    return None if rec is None else rec["dram_bytes_per_cell"] * n_cells


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]),
                "reasons": reasons, "samples": len(rows)}


def peaks():
    try:
        p = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def make_workload(kind, n):
    from paper_1210_5246_gb300 import inputs
    if kind == "box":
        return inputs.turb(n=n, nsteps=50)
    if kind == "blast":
        return inputs.blast(n=n)
    return inputs.disc(n=n)


# ----------------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_1210_5246_gb300 import replicas
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    replicas.init()
    import __graft_entry__
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        replicas.barrier()
        __graft_entry__.build()
    from paper_1210_5246_gb300 import msh

    n_axis, desc, kernel_name = WORKLOADS[args.workload]
    n_axis = args.n or n_axis
    p = make_workload(args.workload, n_axis)
    ncells = int(np.prod(p.n))
    state_mb = ncells * 10 * 4 / 1e6
    # one dedicated stream: the library launches on it and the CUDA events are recorded on it
    stream = torch.cuda.Stream()
    W32 = torch.from_numpy(p.W.astype(np.float32)).cuda()
    W64 = None if args.fp32_only else torch.from_numpy(p.W).cuda()
    torch.cuda.synchronize()

    def timed(precision, Wdev, steps, warmup, profile):
        g = msh.Grid.from_problem(p, precision, stream=stream.cuda_stream)
        if args.ctu:
            g.set_ctu(True)
        g.set_state(Wdev, msh.PRIMITIVE)
        if args.tiling:
            g.set_tiling(*[int(v) for v in args.tiling.split(",")])
        else:
            g.autotune()
        g.run(max_steps=warmup)
        g.set_state(Wdev, msh.PRIMITIVE)          # time the workload's first K steps
        g.set_time(0.0, 0)
        torch.cuda.synchronize()
        replicas.barrier()
        sampler = ClockSampler(local) if profile else None
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ns, _ = g.run(max_steps=steps)
        e1.record(stream)
        torch.cuda.synchronize()
        replicas.barrier()
        clocks = sampler.stop() if sampler else None
        ms = e0.elapsed_time(e1)
        kern_ms, kern_n = None, None
        if profile:
            # the same K steps again, launched eagerly with CUDA events around each step kernel
            g.set_state(Wdev, msh.PRIMITIVE)
            g.set_time(0.0, 0)
            g.set_profiling(True)
            e0.record(stream)
            g.run(max_steps=steps)
            e1.record(stream)
            torch.cuda.synchronize()
            kern_ms, fin_ms, kern_n = g.profile()
            timed.fin_ms = fin_ms / max(kern_n, 1)
            timed.eager_ms = e0.elapsed_time(e1)
        tiling = g.tiling()
        _, ok, _ = g.diagnostics()
        g.close()
        assert ns == steps and ok
        return ms, kern_ms, kern_n, clocks, tiling

    ms32, kms, kn, clocks, tiling = timed(msh.FP32, W32, args.steps, args.warmup, True)
    steps64 = max(1, min(args.steps, 20))
    if args.fp32_only:
        ms64, tiling64 = float("nan"), None
    else:
        ms64, _, _, _, tiling64 = timed(msh.FP64, W64, steps64, args.warmup, False)

    # end to end through the C ABI with host buffers: every step uploads its input state from
    # page-locked host memory, takes one CFL step and downloads the result.  msh_run_ensemble
    # overlaps the uploads, steps and downloads of different steps' states; the plain
    # per-call sequence (set_state, run, get_state) is reported beside it.
    e2e = None
    if not args.no_e2e:
        host_in = torch.from_numpy(p.W.astype(np.float32)).pin_memory()
        host_out = [torch.empty_like(host_in).pin_memory() for _ in range(2)]
        g = msh.Grid.from_problem(p, msh.FP32, stream=stream.cuda_stream)
        g.set_tiling(*tiling)
        k_e2e = max(3, args.steps)
        ins = [host_in.numpy()] * k_e2e
        outs = [host_out[k % 2].numpy() for k in range(k_e2e)]
        g.run_ensemble(ins[:3], outs[:3], kind=msh.PRIMITIVE, nsteps=1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.run_ensemble(ins, outs, kind=msh.PRIMITIVE, nsteps=1)
        torch.cuda.synchronize()
        dt_e2e = time.perf_counter() - t0

        def one():
            g.set_state(ins[0], msh.PRIMITIVE)
            g.run(max_steps=1)
            g.get_state(msh.PRIMITIVE, out=outs[0])
        k_seq = max(3, min(args.steps, 10))
        one()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k_seq):
            one()
        torch.cuda.synchronize()
        dt_seq = time.perf_counter() - t0
        g.close()
        nbytes = ncells * 10 * 4
        e2e = {"value": ncells * k_e2e / dt_e2e, "unit": "cell-updates/s",
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "steps": k_e2e,
               "api": "msh_run_ensemble (upload, step, download per step; overlapped)",
               "sequential": {"value": ncells * k_seq / dt_seq, "steps": k_seq,
                              "api": "msh_set_state + msh_run + msh_get_state per step"}}

    # max over ranks of the timed region; every rank advanced its own replica
    ms32 = replicas.max_over_ranks(ms32)
    value = replicas.whole_job_rate(ncells * args.steps, ms32 * 1e-3)
    value64 = ncells * steps64 / (ms64 * 1e-3) if not args.fp32_only else None

    hbm, peak_kind = peaks()
    avg_kernel_s = (kms / kn) * 1e-3
    achieved = BYTES_PER_CELL["f32"] * ncells / avg_kernel_s / 1e9
    traffic = measured_traffic(ncells) if args.workload == "box" else None
    # per step: step kernel, 4 fallback passes (idle unless cells were tagged), finalize;
    # the graphs hold 16 steps, plus the run-start kernel
    graph_launches = math.ceil(args.steps / 16) * 16 * 6 + 1
    out = {
        "metric": "cell-updates/s", "value": value, "unit": "cell-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms32 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": DATA[args.workload],
        "config": {"workload": desc.format(n=n_axis) + f", steps 1..{args.steps}",
                   "cells": ncells, "parallelism": f"replicas x{world}", "ctu": bool(args.ctu),
                   "l2": (f"state ({state_mb:.0f} MB per buffer) larger than L2; no flush" if state_mb > 129
                          else f"state ({state_mb:.0f} MB per buffer) fits in L2; no flush (L2-assisted)"),
                   "tiling": list(tiling)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic,
                     "kernel": kernel_name, "peak_source": peak_kind,
                     "kernel_ms": kms / kn, "bytes_per_cell": BYTES_PER_CELL["f32"],
                     "eager_ms_per_step": timed.eager_ms / args.steps, "finalize_ms": timed.fin_ms},
        "issue_roofline": (issue_roofline(ncells, avg_kernel_s, torch.cuda.get_device_properties(local).multi_processor_count,
                                          clocks) if args.workload == "box" else None),
        "fp64": None if args.fp32_only else {
            "value": value64, "unit": "cell-updates/s", "steps": steps64, "ms_per_step": ms64 / steps64,
            "tiling": list(tiling64), "hbm_frac": BYTES_PER_CELL["f64"] * value64 / 1e9 / hbm},
        "gpu_launches": graph_launches,
        "clocks": clocks,
        "e2e": e2e,
    }
    if rank == 0 and args.workload == "box" and not args.no_extras:
        # the adjoint and batching targets, measured in the same run (outside the timed region)
        from paper_1210_5246_gb300 import disc, inputs
        out["adjoint"] = adjoint_costs(msh, disc, stream)
        out["tubes"] = tubes_rates(msh, inputs, stream)
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(p)
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


def issue_roofline(ncells, kernel_s, sms, clocks):
    """The bound the step kernel actually meets: instruction issue.  Peak = the device's SM
    count `sms` (cudaDeviceProp.multiProcessorCount) x 4 warp schedulers x 1 warp
    instruction per cycle x the SM clock: the median sampled during the timed region (the
    maximum clock when no sample was taken, said so in `clock_source`); achieved = the warp
    instructions per cell of the committed ncu record x cells / the kernel's CUDA-event time
    (None without a record for the current source)."""
    rec = traffic_record()
    if rec is None or "warp_inst_per_cell" not in rec:
        return None
    if clocks and clocks.get("sm_mhz"):
        mhz, src = float(clocks["sm_mhz"]), "median SM clock sampled by nvidia-smi during the timed region"
    else:
        mhz, src = 2070.0, "maximum SM clock (no clock sample)"
    peak = sms * 4 * mhz * 1e6
    achieved = rec["warp_inst_per_cell"] * ncells / kernel_s
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "warp-instructions/s",
            "frac": achieved / peak, "warp_inst_per_cell": rec["warp_inst_per_cell"],
            "sms": sms, "sm_mhz": mhz, "clock_source": src,
            "peak_source": f"derived: {sms} SMs x 4 schedulers x {mhz:.0f} MHz"}


def cpu_baseline(p):
    """The oracle as it stands: one full-size FP64 step of the same workload."""
    from oracle import oracle
    og = oracle.Grid(p.n, p.lo, p.hi, p.bc, p.cfl)
    U = oracle.prim_to_cons(p.W)
    dt = oracle.cfl_dt(og, U)
    t0 = time.perf_counter()
    oracle.step(og, U, dt, phi=p.phi)
    el = time.perf_counter() - t0
    ncells = int(np.prod(p.n))
    return {"value": ncells / el, "unit": "cell-updates/s", "cores": oracle.num_threads(),
            "kind": "oracle", "sample": f"one FP64 step of the full {p.n[0]}^3 box ({el:.1f} s)"}


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    from oracle import oracle
    from paper_1210_5246_gb300 import inputs
    oracle.build()
    n_axis, desc, _ = WORKLOADS[args.workload]
    n_axis = args.n or n_axis
    p = make_workload(args.workload, n_axis)
    # every step is one FP64 step of the full workload (~3 s for the 256^3 box on 16 host
    # cores, so the default run of 20 timed and 5 warm-up steps takes a little over a minute)
    Wc = p.W
    og = oracle.Grid(p.n, p.lo, p.hi, p.bc, p.cfl)
    cells, sample = int(np.prod(p.n)), "the full grid"
    U = oracle.prim_to_cons(Wc)
    phi = p.phi if args.workload == "disc" else None
    for _ in range(args.warmup):
        U = oracle.step(og, U, oracle.cfl_dt(og, U), phi=phi)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        U = oracle.step(og, U, oracle.cfl_dt(og, U), phi=phi)
    el = time.perf_counter() - t0
    v = cells * args.steps / el
    cores = oracle.num_threads()
    print(json.dumps({
        "impl": "reference", "metric": "cell-updates/s", "value": v, "unit": "cell-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": DATA[args.workload],
        "config": {"workload": desc.format(n=n_axis).replace("FP32", "FP64 oracle") + f" (each step: {sample})",
                   "cells": cells},
        "cpu_baseline": {"value": v, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
                         "sample": f"{sample}, {args.steps} steps"},
        "e2e": {"value": v, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------------- the suite
def _oracle_rate(p, steps=1, crop=None):
    """Oracle cell-updates/s over `steps` FP64 steps of problem p (optionally a crop)."""
    from oracle import oracle
    W = p.W if crop is None else np.ascontiguousarray(p.W[(slice(None),) + crop])
    n = tuple(reversed(W.shape[1:]))[: p.ndim]
    og = oracle.Grid(n, p.lo, [p.lo[d] + (p.hi[d] - p.lo[d]) * n[d] / p.n[d] for d in range(p.ndim)], p.bc, p.cfl)
    U = oracle.prim_to_cons(W)
    phi = None
    if p.phi is not None and crop is None:
        phi = p.phi
    t0 = time.perf_counter()
    for _ in range(steps):
        U = oracle.step(og, U, oracle.cfl_dt(og, U), phi=phi)
    el = time.perf_counter() - t0
    return int(np.prod(n)) * steps / el, oracle.num_threads(), el


def _oracle_rate_1core(p, steps=1, crop=None):
    """The same on one host core (the oracle's OpenMP pool restored afterwards)."""
    from oracle import oracle
    n0 = oracle.num_threads()
    oracle.set_num_threads(1)
    try:
        v, _, el = _oracle_rate(p, steps=steps, crop=crop)
    finally:
        oracle.set_num_threads(n0)
    return v, el


def run_suite(args):
    """One JSON line per workload: GPU cell-updates/s in FP32/FP64, the HBM fraction of the
    step kernel, the oracle's rate on the host cores, and for the batched tubes and the disc
    the comparisons the workloads are about (persistent launch vs one launch per step per
    tube; adjoint vs forward cost)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1210_5246_gb300 import disc, inputs, msh
    hbm, _ = peaks()
    stream = torch.cuda.Stream()

    def emit(d):
        print(json.dumps(d), flush=True)

    def grid_rate(p, precision, steps, t_end=math.inf, scheme=0, ctu=False, cfl=None):
        if cfl is None:
            g = msh.Grid.from_problem(p, precision, stream=stream.cuda_stream)
        else:
            g = msh.Grid(p.n, p.lo, p.hi, p.bc, cfl, precision, stream=stream.cuda_stream)
        if scheme:
            g.set_scheme(scheme)
        if ctu:
            g.set_ctu(True)
        W = p.W.astype(np.float32) if precision == msh.FP32 else p.W
        g.set_state(W, msh.PRIMITIVE)
        if p.ndim > 1:
            g.autotune()
        g.run(t_end, min(steps, 3))
        g.set_state(W, msh.PRIMITIVE)
        g.set_time(0.0, 0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ns, t = g.run(t_end, steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        g.set_state(W, msh.PRIMITIVE)
        g.set_time(0.0, 0)
        g.set_profiling(True)
        g.run(t_end, steps)
        kms, _, kn = g.profile()
        g.close()
        cells = int(np.prod(p.n))
        bpc = 80 if precision == msh.FP32 else 160
        return {"value": cells * ns / (ms * 1e-3), "steps": ns, "ms_per_step": ms / ns, "t": t,
                "sim_time_per_s": t / (ms * 1e-3),
                "kernel_ms": kms / max(kn, 1), "hbm_frac": bpc * cells / (kms / max(kn, 1) * 1e-3) / 1e9 / hbm}

    only = args.only
    # 1D shock tube, FP64, to t = 0.2
    if only in (None, "sod"):
        p = inputs.sod(args.n or 256)
        r = grid_rate(p, msh.FP64, 1 << 20, p.t_end)
        orc, cores, _ = _oracle_rate(p, steps=r["steps"])
        orc1, _ = _oracle_rate_1core(p, steps=r["steps"])
        # the same problem as one tube of the batched kernel: every step in one persistent
        # launch (the grid path pays six launches per step, which a 256-cell step cannot hide)
        WL, WR = p.W[:, 0, 0, 0], p.W[:, 0, 0, -1]
        b = msh.Batch([p.n[0]], WL[None, :], WR[None, :], p.t_end, p.cfl, msh.FP64, stream=stream.cuda_stream)
        b.run()
        b.reset()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.run()
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        steps_b, _, cu = b.info()
        b.close()
        emit({"workload": f"sod {p.n[0]} cells FP64 to t=0.2", "gpu_fp64": r, "oracle": orc, "oracle_cores": cores,
              "oracle_1core": orc1,
              "gpu_fp64_one_tube_batch": {"value": cu / el, "steps": int(steps_b[0]), "ms_total": el * 1e3}})
    # 2D blast 1024^2, 200 steps
    if only in (None, "blast"):
        p = inputs.blast(n=args.n or 1024)
        steps = p.nsteps if only is None else args.steps
        r32 = grid_rate(p, msh.FP32, steps)
        r64 = grid_rate(p, msh.FP64, steps)
        orc, cores, _ = _oracle_rate(p, steps=2)
        crop = (slice(0, 1), slice(0, 256), slice(0, 256))
        orc_crop, _, _ = _oracle_rate(p, steps=1, crop=crop)
        orc1, _ = _oracle_rate_1core(p, steps=1, crop=crop)
        emit({"workload": f"blast {p.n[0]}^2, {steps} steps", "gpu_fp32": r32, "gpu_fp64": r64, "oracle": orc,
              "oracle_cores": cores, "oracle_sample": "2 FP64 steps of the full grid",
              "oracle_crop": orc_crop, "oracle_1core": orc1,
              "oracle_crop_sample": "1 FP64 step of a 256^2 periodic crop (oracle_crop: all cores, "
                                    "oracle_1core: one core)"})
    # 3D box 256^3, 50 steps
    if only in (None, "box"):
        p = inputs.turb(n=args.n or 256)
        steps = p.nsteps if only is None else args.steps
        r32 = grid_rate(p, msh.FP32, steps)
        r64 = grid_rate(p, msh.FP64, min(steps, 20))
        orc, cores, _ = _oracle_rate(p, steps=1)
        crop = (slice(0, 64), slice(0, 64), slice(0, 64))
        orc_crop, _, _ = _oracle_rate(p, steps=1, crop=crop)
        orc1, _ = _oracle_rate_1core(p, steps=1, crop=crop)
        emit({"workload": f"turb {p.n[0]}^3, {steps} steps (FP64: {min(steps, 20)})", "gpu_fp32": r32,
              "gpu_fp64": r64, "oracle": orc, "oracle_cores": cores, "oracle_sample": "1 FP64 step of the full grid",
              "oracle_crop": orc_crop, "oracle_1core": orc1,
              "oracle_crop_sample": "1 FP64 step of a 64^3 periodic crop (oracle_crop: all cores, "
                                    "oracle_1core: one core)",
              "gpu_fp32_over_oracle": r32["value"] / orc})
    # the two schemes at the same CFL number: time per step (Sec. 4.1 reports the central
    # scheme about 22 % cheaper than the characteristic one on the CPU)
    if only in (None, "schemes"):
        for name, p in (("box", inputs.turb(n=args.n or 256, cfl=0.4)), ("blast", inputs.blast(n=args.n or 1024, cfl=0.4))):
            steps = 50 if only is None else args.steps
            mh = grid_rate(p, msh.FP32, steps)
            roe = grid_rate(p, msh.FP32, steps, scheme=msh.MUSCL_HANCOCK_ROE)
            hllc = grid_rate(p, msh.FP32, steps, scheme=msh.MUSCL_HANCOCK_HLLC)
            kt = grid_rate(p, msh.FP32, steps, scheme=msh.KT)
            emit({"workload": f"{name} {p.n[0]}^{p.ndim} FP32, CFL 0.4, {steps} steps: MUSCL-Hancock (HLL, Roe-type, "
                              "HLLC) vs Kurganov-Tadmor",
                  "muscl_hancock": mh, "muscl_hancock_roe": roe, "muscl_hancock_hllc": hllc, "kurganov_tadmor": kt,
                  "kt_ms_over_mh_ms": kt["ms_per_step"] / mh["ms_per_step"],
                  "roe_ms_over_hll_ms": roe["ms_per_step"] / mh["ms_per_step"],
                  "hllc_ms_over_hll_ms": hllc["ms_per_step"] / mh["ms_per_step"]})
    # the corner-transport-upwind form: its max-form CFL rule allows longer steps than the
    # plain unsplit step's sum rule, at a higher cost per step; compared by simulated time
    # per second at the largest CFL number of a ladder whose run stays realizable (the
    # first-order faces of the fallback carry no transverse terms and need not restore
    # realizability at the longer steps)
    if only in (None, "ctu"):
        for name, p in (("box", inputs.turb(n=args.n or 256)), ("blast", inputs.blast(n=args.n or 1024))):
            steps = 50 if only is None else args.steps
            plain = grid_rate(p, msh.FP32, steps, cfl=0.5)
            ladder, ctu = {}, None
            for c in (0.8, 0.6, 0.5, 0.4, 0.3):
                try:
                    ctu = grid_rate(p, msh.FP32, steps, ctu=True, cfl=c)
                    ctu["cfl"] = c
                    break
                except msh.MshError as e:
                    ladder[str(c)] = str(e)
            line = {"workload": f"{name} {p.n[0]}^{p.ndim} FP32, {steps} steps: plain unsplit step (CFL 0.5, sum "
                                "rule) vs corner transport upwind (max rule, largest realizable CFL of 0.8 .. 0.3)",
                    "plain": plain, "ctu": ctu, "ctu_not_realizable": ladder}
            if ctu is not None:
                line["ctu_ms_over_plain_ms"] = ctu["ms_per_step"] / plain["ms_per_step"]
                line["ctu_sim_time_rate_over_plain"] = ctu["sim_time_per_s"] / plain["sim_time_per_s"]
            emit(line)
    # periodic self-gravity: the cost of the FFT Poisson solve and acceleration per step
    if only in (None, "selfgrav"):
        p = inputs.turb(n=args.n or 256)
        steps = 20 if only is None else args.steps
        base = grid_rate(p, msh.FP32, steps)
        g = msh.Grid.from_problem(p, msh.FP32, stream=stream.cuda_stream)
        g.set_self_gravity(1.0)
        W = p.W.astype(np.float32)
        g.set_state(W, msh.PRIMITIVE)
        g.set_tiling(16, 32)
        g.run(math.inf, 3)
        g.set_state(W, msh.PRIMITIVE)
        g.set_time(0.0, 0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ns, _ = g.run(math.inf, steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / ns
        g.close()
        emit({"workload": f"box {p.n[0]}^3 FP32 with periodic self-gravity (G = 1), {steps} steps",
              "ms_per_step": ms, "without_self_gravity_ms_per_step": base["ms_per_step"],
              "self_gravity_ms_per_step": ms - base["ms_per_step"],
              "cell_updates_per_s": int(np.prod(p.n)) * ns / (ms * ns * 1e-3)})
    if only in (None, "tubes"):
        run_suite_tubes(msh, inputs, stream, emit, per_tube=not args.persistent_only)
    if only in (None, "disc"):
        n = args.n or 512
        run_suite_disc(msh, disc, stream, emit, n, 2000 if only is None else args.steps)


def tubes_rates(msh, inputs, stream, per_tube=True):
    """Batched tubes (4096 tubes of 128..2048 cells, FP32, to t = 0.1): cell-updates/s of the
    persistent launch (the whole workload, wall time around msh_batch_run after its
    autotuning run) and, on 32 tubes spread over the length range, of one step-kernel launch
    per step per tube (msh_batch_run_per_tube)."""
    import torch
    tb = inputs.tubes()
    b = msh.Batch(tb.length, tb.WL, tb.WR, tb.t_end, tb.cfl, msh.FP32, stream=stream.cuda_stream)
    b.run()  # autotunes the block size
    b.reset()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.run()
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    _, _, cu = b.info()
    out = {"workload": "4096 tubes 128..2048 cells FP32 to t=0.1", "unit": "cell-updates/s",
           "persistent": cu / el, "cell_updates": cu, "seconds": el}
    if per_tube:
        sample = np.argsort(tb.length)[:: len(tb.length) // 32][:32]
        b.reset()
        b.run_per_tube(sample)  # builds the per-tube grids
        b.reset()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.run_per_tube(sample)
        torch.cuda.synchronize()
        el_pt = time.perf_counter() - t0
        steps_pt, _, _ = b.info()
        cu_pt = int((steps_pt[sample] * tb.length[sample]).sum())
        out.update({"per_tube_launches": cu_pt / el_pt,
                    "per_tube_sample": "32 tubes spread over the length range",
                    "speedup": (cu / el) / (cu_pt / el_pt)})
    b.close()
    return out


def run_suite_tubes(msh, inputs, stream, emit, per_tube=True):
    """Batched tubes: one persistent launch vs one launch per step per tube."""
    emit(tubes_rates(msh, inputs, stream, per_tube))


def adjoint_costs(msh, disc, stream, n=512, nsteps=2000, K=50, precisions=("fp32", "fp64")):
    """Differentiable disc (n^2, nsteps steps, checkpoints every K): wall time per step of the
    forward run (BMERun: the recorded graph-launched run) and of the backward
    (msh_adjoint_tape: segment recomputation from the checkpoints, reverse steps), each after
    one warm-up; backward cell-updates/s = cells x steps / backward time.  FP32 and FP64, and
    the FP32 loss and gradients' errors against FP64."""
    import torch
    from paper_1210_5246_gb300 import autograd as ag
    res, grads = {}, {}
    for name in precisions:
        prec = msh.FP32 if name == "fp32" else msh.FP64
        D = disc.DiscProblem(n=n, nsteps=nsteps, precision=prec, K=K, stream=stream.cuda_stream)
        D.value_and_grad()  # warm-up (builds graphs, allocates)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        W0 = D.initial_state(D.delta0, torch.tensor(0.0, dtype=torch.float64, device="cuda")).to(D.dtype).contiguous()
        ag.BMERun.apply(W0, D.grid, D.nsteps, D.K)
        torch.cuda.synchronize()
        t_fwd = time.perf_counter() - t0
        t0 = time.perf_counter()
        L, gd, gb = D.value_and_grad()
        torch.cuda.synchronize()
        t_both = time.perf_counter() - t0
        D.close()
        t_bwd = t_both - t_fwd
        cells = n * n
        res[name] = {"forward_ms_per_step": t_fwd * 1e3 / nsteps, "backward_ms_per_step": t_bwd * 1e3 / nsteps,
                     "backward_over_forward": t_bwd / t_fwd,
                     "forward_cell_updates_per_s": cells * nsteps / t_fwd,
                     "backward_cell_updates_per_s": cells * nsteps / t_bwd,
                     "loss": L, "dL_dbeta": gb}
        grads[name] = (L, gd, gb)
    out = {"workload": f"disc {n}^2, {nsteps} steps, checkpoints every K={K}", **res}
    if "fp32" in grads and "fp64" in grads:
        (L, gd, gb), (L64, gd64, gb64) = grads["fp32"], grads["fp64"]
        out["fp32_error_vs_fp64"] = {"loss_rel": abs(L - L64) / abs(L64), "dL_dbeta_rel": abs(gb - gb64) / abs(gb64),
                                     "dL_ddelta_rel_l2": float(torch.linalg.norm(gd - gd64) / torch.linalg.norm(gd64))}
    return out


def run_suite_disc(msh, disc, stream, emit, n, nsteps, K=50):
    """Differentiable disc: cost per step of the forward run and of the backward
    (msh_adjoint_run: checkpointed forward, segment recomputation, reverse steps)."""
    emit(adjoint_costs(msh, disc, stream, n, nsteps, K))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.suite:
        run_suite(a)
    else:
        run_gpu(a)
