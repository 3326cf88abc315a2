#!/usr/bin/env python
"""Benchmark: 3-D FADI cell-steps/s on one GB300 (FP32 fields with FP64-formed
coefficients; FP64 form alongside), with HBM roofline, end-to-end time through
the C ABI with host buffers, and the FP64 CPU oracle as the baseline.

Workload: 256^3-cell PEC cavity, 1 mm cells, vacuum, CFL 4, initial E = sum of
8 seeded cavity eigenmodes (N(0,1) amplitudes).  A step is one FADI time step:
procedures A and B, each three fused line-solve kernels over all six arrays.
The state (457 MB in FP32) exceeds the 129 MB L2, so no flush is needed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (torchrun): independent replicas, one grid per GPU, no collective
in the data path; value = all ranks' cell-steps / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "3D FADI cell-steps/s on 1 GB300, FP32 vs FP64 at stated error; % HBM peak"
UNIT = "cell-steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256, help="cells per axis")
    ap.add_argument("--cfl", type=float, default=4.0)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--tune", type=int, nargs=2, default=(0, 0), help="kernel-shape overrides (fdtd_desc.tune)")
    ap.add_argument("--no-batch", action="store_true", help="skip the many-cavity batch measurement")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the gradient (adjoint) measurement")
    ap.add_argument("--suite", action="store_true",
                    help="print throughput of every workload recipe (one JSON line each) instead of the bench line")
    ap.add_argument("--adjoint-n", type=int, default=192, help="cells per axis of the gradient run")
    ap.add_argument("--adjoint-steps", type=int, default=500)
    ap.add_argument("--adjoint-every", type=int, default=25, help="checkpoint spacing of the gradient run")
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--batch-steps", type=int, default=500)
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_fields(n):
    import workloads as W
    d = 1e-3
    modes = W.random_modes(2, n, n, n, d, d, d, count=8)
    return W.mode_sum_fields(modes, n, n, n)


def kernel_sources_sha1() -> str:
    """sha1 of the line kernels and of the host code that picks them."""
    import hashlib
    h = hashlib.sha1()
    for name in ("line_kernels.cuh", "fdtd.cu"):
        with open(os.path.join(ROOT, "paper_2011_14043_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def recorded_traffic(kernel_class: str, n: int):
    """DRAM bytes per launch of the kernel of one line direction from the
    committed ncu capture (profiles/dram_traffic.json), or None when the
    kernels or their launch choices changed since that capture, or when the
    grid is not the captured one."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))
        if kernel_sources_sha1() != rec["sources_sha1"] or n != rec["grid"]:
            return None
        return rec["classes"][kernel_class]["traffic_bytes_per_launch"]
    except Exception:
        return None


# The method's work per cell-step of FADI (Sec. IV, Table I): 42 flops of
# right-hand-side and explicit updates plus about 30 for the tridiagonal
# solves (5N per system of order N).  This is the basis of the FP64 form's
# ALU roofline.
FP64_FLOPS_PER_CELL_STEP = 42 + 30
# What the kernels issue per cell-step at 256^3, for context.  Per node of
# an x-line pair (segmented solve): RHS 1 sub + 1 FMA, forward sweep 1 FMA,
# forward carry fix 1 FMA, backward sweep 1 mul + 1 FMA, backward carry fix
# 1 FMA, H update 1 sub + 1 FMA, E update 1 sub: 16 flops (an FMA counts 2);
# per node of a y/z pair (one thread per line, no carry fixes or scans): 12.
# Two x pairs and four y/z pairs per step.
KERNEL_FP64_FLOPS_PER_CELL_STEP = 2 * 16 + 4 * 12


def fp64_alu_roofline(cell_steps_per_s: float) -> dict:
    """The FP64 form against the device's measured FP64 FMA rate, on the
    method's 72 flops per cell-step."""
    from paper_2011_14043_gb300 import probe_fp64_fma
    peak = probe_fp64_fma(20000) / 1e9
    achieved = FP64_FLOPS_PER_CELL_STEP * cell_steps_per_s / 1e9
    issued = KERNEL_FP64_FLOPS_PER_CELL_STEP * cell_steps_per_s / 1e9
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "GFLOP/s", "frac": achieved / peak,
            "peak_kind": "measured: FP64 FMA microbenchmark (fdtd_probe_fp64_fma)",
            "flops_per_cell_step": FP64_FLOPS_PER_CELL_STEP,
            "flops_basis": "the method's count, Table I: 42 RHS/explicit + 30 tridiagonal per cell-step",
            "kernel_issued": {"flops_per_cell_step": KERNEL_FP64_FLOPS_PER_CELL_STEP, "achieved": issued,
                              "frac": issued / peak,
                              "note": "FP64 flops the kernels issue at 256^3 (x lines: segmented Thomas with carry fixes; "
                                      "y/z lines: one thread per line)"}}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
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
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def run_gpu(args, prec, fields, time_kernels=True, keep_fields=False):
    """Device-resident timing of K steps on the library's default path (each
    step a replay of a captured graph whose three pair launches per procedure
    run on parallel branches), CUDA events on the handle's stream around the
    K steps.  With time_kernels, a second, serialised pass of the same
    kernels records a CUDA event pair around every line-solve launch: the
    per-kernel durations the roofline needs (a kernel's duration is not
    defined while the three pairs of a procedure share the GPU)."""
    import torch
    from paper_2011_14043_gb300 import Simulation
    n = args.n
    sim = Simulation(n, n, n, 1e-3, scheme="fadi", precision=prec, cfl=args.cfl, tune=tuple(args.tune))
    sim.set_fields(fields)
    sim.step(args.warmup)            # includes the Eq. 10 initialization and the graph capture
    sim.synchronize()
    stream = torch.cuda.ExternalStream(sim._stream.value) if sim._stream.value else torch.cuda.current_stream()
    sim.reset_stats()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = sim.stats()["launches"]
    st = None
    if time_kernels:
        sim.reset_stats()
        sim.set_timing(True)
        sim.step(max(4, min(args.steps, 40)))
        sim.synchronize()
        st = sim.stats()
        sim.set_timing(False)
    energy = sim.energy()
    out = None
    if keep_fields:
        out = {c: sim.get_field(c, device=True).clone() for c in fields}
    total_steps = sim.steps_done
    sim.close()
    return {"ms": ms, "launches": launches, "stats": st, "energy": energy, "fields": out,
            "total_steps": total_steps}


def device_rel_err(a: dict, b: dict) -> float:
    """Relative L2 of fields a against fields b (device tensors) in the vacuum
    energy norm: E weighted by eps0, H by mu0."""
    mu0 = 1.25663706212e-6
    eps0 = 1.0 / (mu0 * 299792458.0 ** 2)
    num = den = 0.0
    for c in a:
        w = eps0 if c.startswith("e") else mu0
        d = a[c].double() - b[c].double()
        num += w * float((d * d).sum())
        den += w * float((b[c].double() ** 2).sum())
    return math.sqrt(num / den)


def fp64_reference_fields(args, fields, steps):
    """The FP64 GPU path after `steps` steps of the same workload."""
    from paper_2011_14043_gb300 import Simulation
    n = args.n
    sim = Simulation(n, n, n, 1e-3, scheme="fadi", precision="f64", cfl=args.cfl, tune=tuple(args.tune))
    sim.set_fields(fields)
    sim.step(steps)
    out = {c: sim.get_field(c, device=True).clone() for c in fields}
    sim.close()
    return out


def run_e2e(args, prec, fields, reps=3):
    """Same metric through the C ABI with pinned host buffers: H2D of the
    initial fields, K steps, D2H of all six field components, all timed.
    One untimed round first, then `reps` timed rounds (a fresh handle each);
    the median is reported with every sample (the host-device link shows
    sporadic stalls of several milliseconds)."""
    import numpy as np
    import torch
    from paper_2011_14043_gb300 import Simulation
    n = args.n
    np_dtype = np.float32 if prec == "f32" else np.float64
    t_dtype = torch.float32 if prec == "f32" else torch.float64
    host_in = {}
    host_out = {}
    for c, v in fields.items():
        t = torch.empty(v.shape, dtype=t_dtype, pin_memory=True)
        t.numpy()[...] = v.astype(np_dtype)
        host_in[c] = t
        host_out[c] = torch.empty(v.shape, dtype=t_dtype, pin_memory=True)
    times = []
    for r in range(reps + 1):
        sim = Simulation(n, n, n, 1e-3, scheme="fadi", precision=prec, cfl=args.cfl, tune=tuple(args.tune))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for c in fields:
            sim.set_field(c, host_in[c].numpy())
        sim.step(args.steps)
        for c in fields:
            sim.get_field(c, out=host_out[c].numpy())
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        sim.close()
        if r > 0:
            times.append(t1 - t0)
    nbytes = sum(v.numel() * v.element_size() for v in host_in.values())
    return {"s": statistics.median(times), "samples_s": times, "h2d": nbytes, "d2h": nbytes}


def replica_throughput(local_ms: float, units_per_rank: float, ws: int, device: str):
    """Replicas (one independent grid per rank, no exchange in the data path):
    the job takes as long as its slowest rank, so the time is the MAX over
    ranks and the value all ranks' units over that time."""
    ms = local_ms
    if ws > 1:
        import torch
        t = torch.tensor([ms], device=device, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    return ms, ws * units_per_rank / (ms / 1e3)


def adjoint_section(args):
    """Gradient of the probe energy with respect to eps_r on the 192^3
    differentiable run (eps_r in [1, 6] in the central 64^3, dipole, 4^3 probe
    block, 500 steps, checkpoints every 25), FP32: forward (with checkpoints)
    and adjoint (recomputation + transposed procedures) timed separately."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2011_14043_gb300.adjoint import ProbeEnergyProblem
    wl = W.workload_adjoint(n=args.adjoint_n, steps=args.adjoint_steps, checkpoint_every=args.adjoint_every)
    n = wl.nx
    c0 = 299792458.0
    dt = wl.cfl / (c0 * math.sqrt(3.0 / wl.dx ** 2))
    cur = W.dipole_current((np.arange(wl.steps + 1) + 0.5) * dt)
    s = wl.source
    prob = ProbeEnergyProblem(n, n, n, wl.dx, steps=wl.steps, probe_block=wl.extra["probe_block"], dt=dt,
                              precision="f32", checkpoint_every=wl.extra["checkpoint_every"],
                              source=(s["comp"], s["i"], s["j"], s["k"], cur))
    from paper_2011_14043_gb300.adjoint import AdjointRun
    # warm-up: a 2-step run of the same grid fills the launch-shape caches
    warm = ProbeEnergyProblem(n, n, n, wl.dx, steps=2, probe_block=wl.extra["probe_block"], dt=dt,
                              precision="f32", checkpoint_every=1, source=prob.source)
    w = AdjointRun(warm, wl.eps_r)
    w.forward()
    w.backward(1.0)
    w.close()
    run = AdjointRun(prob, wl.eps_r)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J = run.forward()
    t1 = time.perf_counter()
    out = torch.empty((n, n, n), dtype=torch.float64, device="cuda")
    run.backward(1.0, out=out)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    mem = run.memory_bytes()
    run.close()
    cs = n ** 3 * wl.steps
    lo, hi = wl.extra["region"]
    return {"workload": f"FADI {n}^3, eps_r U[1,6] in the central {hi - lo}^3, z dipole, probe block, "
                        f"{wl.steps} steps, checkpoints every {wl.extra['checkpoint_every']}",
            "dtype": "f32", "objective": J, "forward_s": t1 - t0, "backward_s": t2 - t1,
            "forward_cell_steps_per_s": cs / (t1 - t0), "gradient_cell_steps_per_s": cs / (t2 - t0),
            "backward_over_forward": (t2 - t1) / (t1 - t0), "device_bytes": mem,
            "timing": "host wall clock around the synchronous C-ABI calls"}


def batch_rel_err(a: dict, b: dict) -> float:
    """Relative L2 in the vacuum energy norm (E weighted by eps0, H by mu0)."""
    import numpy as np
    eps0 = 1.0 / (1.25663706212e-6 * 299792458.0 ** 2)
    num = den = 0.0
    for c in a:
        w = eps0 if c.startswith("e") else 1.25663706212e-6
        num += w * float(np.sum((a[c].astype(np.float64) - b[c]) ** 2))
        den += w * float(np.sum(b[c].astype(np.float64) ** 2))
    return math.sqrt(num / den)


def run_batch(wls, prec, steps, warmup, want_fields):
    """Many cavities stepped as one batch (one CUDA graph per step); CUDA
    events on the handles' stream around ``steps`` steps."""
    import torch
    from paper_2011_14043_gb300 import Batch, Simulation
    sims = []
    for w in wls:
        s = Simulation(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, scheme="fadi", precision=prec, cfl=w.cfl)
        s.set_material(w.eps_r)
        s.set_fields(w.fields)
        sims.append(s)
    b = Batch(sims)
    b.step(warmup)
    b.synchronize()
    stream = torch.cuda.ExternalStream(sims[0]._stream.value) if sims[0]._stream.value \
        else torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    per_step = b.launches_per_step()
    cfg = b.config()
    cfg.update(b.mode())
    fields = [s.get_fields() for s in sims] if want_fields else None
    b.close()
    for s in sims:
        s.close()
    return {"ms": ms, "launches_per_step": per_step, "fields": fields, "config": cfg}


def batch_section(args):
    """64 seeded PEC cavities (32..160 x 32..96 x 32..128 cells, CFL in [2, 10],
    eps_r blocks in [1, 4], 8-mode initial field), FADI FP32, stepped together;
    per-instance error against the FP64 path after the same steps."""
    import workloads as W
    wls = W.workload_batch(seed=4, count=args.batch_count, steps=args.batch_steps)
    cells = sum(w.nx * w.ny * w.nz for w in wls)
    r32 = run_batch(wls, "f32", args.batch_steps, args.warmup, want_fields=not args.no_fp64)
    out = {"value": cells * args.batch_steps / (r32["ms"] / 1e3), "unit": UNIT,
           "ms_per_step": r32["ms"] / args.batch_steps, "steps": args.batch_steps, "warmup": args.warmup,
           "instances": len(wls), "cells": cells, "dtype": "f32",
           "workload": f"{len(wls)} seeded PEC cavities, 1 mm cells, sizes 32..160 x 32..96 x 32..128, "
                       f"CFL U[2,10], eps_r blocks U[1,4], 8 seeded modes, FADI",
           "gpu_launches": r32["launches_per_step"] * args.batch_steps,
           "launch_shape": r32["config"],
           "hbm_frac_step": 96.0 * cells * args.batch_steps / (r32["ms"] / 1e3) / 1e9
           / measured_peaks()[0]["hbm_gbs"]}
    # whole-step roofline on the algorithmic bytes of FADI with per-node
    # media: 96 B of fields + 2 procedures x 3 E unknowns x one 8 B FP64 pivot
    batch_gbs = 144.0 * cells * args.batch_steps / (r32["ms"] / 1e3) / 1e9
    peak = measured_peaks()[0]["hbm_gbs"]
    out["roofline"] = {"bound": "hbm", "achieved": batch_gbs, "peak": peak, "unit": "GB/s",
                       "frac": batch_gbs / peak,
                       "basis": "144 B per cell-step (96 B fields + 48 B FP64 pivots), whole batch step"}
    if not args.no_fp64:
        r64 = run_batch(wls, "f64", args.batch_steps, args.warmup, want_fields=True)
        errs = [batch_rel_err(a, b) for a, b in zip(r32["fields"], r64["fields"])]
        out["fp64_value"] = cells * args.batch_steps / (r64["ms"] / 1e3)
        out["max_rel_err_vs_fp64"] = max(errs)
        out["median_rel_err_vs_fp64"] = statistics.median(errs)
        out["error_norm"] = "per-instance relative L2, vacuum energy weights, FP32 vs FP64 path after the same steps"
    return out


def cpu_baseline(n, steps=1):
    """The FP64 numpy oracle timed on this host on a bounded sample."""
    import oracle.grid as G
    import oracle.schemes as S
    fields = workload_fields(n)
    g = G.Grid(n, n, n, 1e-3, 1e-3, 1e-3)
    P = S.Problem(g, 4.0 * g.dt_cfl())
    v = S.fadi_init(P, fields)
    t0 = time.perf_counter()
    for k in range(steps):
        v = S.fadi_step(P, v, k)
    dt = time.perf_counter() - t0
    return n ** 3 * steps / dt, dt


# Peak resident memory of one oracle FADI step at 256^3 (numpy FP64
# temporaries), measured: about 5.8 GB; it scales with the cell count.
ORACLE_BYTES_256 = 5.8e9


def host_memory_available() -> float:
    """Bytes this process may still use: MemAvailable, capped by a cgroup limit."""
    avail = float("inf")
    try:
        for ln in open("/proc/meminfo"):
            if ln.startswith("MemAvailable:"):
                avail = float(ln.split()[1]) * 1024
    except OSError:
        pass
    for path, used_path in (("/sys/fs/cgroup/memory.max", "/sys/fs/cgroup/memory.current"),
                            ("/sys/fs/cgroup/memory/memory.limit_in_bytes",
                             "/sys/fs/cgroup/memory/memory.usage_in_bytes")):
        try:
            lim = open(path).read().strip()
            if lim != "max" and float(lim) < 1e18:
                avail = min(avail, float(lim) - float(open(used_path).read().strip()))
        except (OSError, ValueError):
            pass
    return avail if avail != float("inf") else 8e9


def oracle_processes(n: int) -> tuple:
    """(processes, host cores): one oracle process per core, as many as fit
    in half of the memory available (each holds about ORACLE_BYTES_256 x
    (n/256)^3)."""
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    need = ORACLE_BYTES_256 * (n / 256.0) ** 3 + 3e8
    return max(1, min(cores, int(0.5 * host_memory_available() // need))), cores


def _oracle_worker(n, cfl, warm, steps, barrier, queue):
    """One process of oracle_replicas: the full FADI workload on one core."""
    import oracle.grid as G
    import oracle.schemes as S
    fields = workload_fields(n)
    g = G.Grid(n, n, n, 1e-3, 1e-3, 1e-3)
    P = S.Problem(g, cfl * g.dt_cfl())
    v = S.fadi_init(P, fields)
    for k in range(warm):
        v = S.fadi_step(P, v, k)
    barrier.wait()
    t0 = time.monotonic()
    for k in range(steps):
        v = S.fadi_step(P, v, warm + k)
    queue.put((t0, time.monotonic()))


def oracle_replicas(n, cfl, warm, steps, procs):
    """The FP64 numpy oracle on every core at once: `procs` spawned processes
    (numpy runs each on one core), each stepping its own copy of the full
    workload; all start their timed steps together (a barrier) and the wall
    time runs from the first start to the last end.  Returns (aggregate
    cell-steps/s, wall seconds)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")      # never fork a process that holds a CUDA context
    barrier = ctx.Barrier(procs)
    queue = ctx.Queue()
    ps = [ctx.Process(target=_oracle_worker, args=(n, cfl, warm, steps, barrier, queue)) for _ in range(procs)]
    for p in ps:
        p.start()
    res = [queue.get() for _ in ps]
    for p in ps:
        p.join()
    wall = max(r[1] for r in res) - min(r[0] for r in res)
    return procs * n ** 3 * steps / wall, wall


def reference_arm(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    n = args.n
    k_steps = max(1, min(args.steps, 3))
    w_steps = min(args.warmup, 1)
    procs, cores = oracle_processes(n)
    val, dt = oracle_replicas(n, args.cfl, w_steps, k_steps, procs)
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": k_steps, "warmup": w_steps, "ms_per_step": 1e3 * dt / k_steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"FADI {n}^3 PEC cavity, 1 mm cells, vacuum, CFL {args.cfl}, 8 seeded modes",
                   "grid": [n, n, n], "scheme": "fadi"},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": procs, "host_cores": cores, "kind": "oracle",
                         "sample": f"{k_steps} of the {args.steps} requested steps of the full {n}^3 "
                                   f"workload on each of {procs} concurrent processes (FP64 numpy oracle, one "
                                   f"core each; {cores} host cores; aggregate cell-steps/s over the wall time "
                                   f"from the first start to the last end)"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def suite(args):
    """Throughput of every workload recipe at its full size (one JSON line
    each; not the bench line): GPU FP32 and FP64 cell-steps/s with CUDA events
    after warm-up, and the FP64 oracle on one host core over a short sample."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2011_14043_gb300 import Simulation
    import oracle.grid as G
    import oracle.schemes as S

    def gpu(nx, ny, nz, d, scheme, prec, cfl, fields, eps=None, src=None, steps=50, warm=5, sigma=None, order=2):
        sim = Simulation(nx, ny, nz, d, scheme=scheme, precision=prec, cfl=cfl, tune=tuple(args.tune))
        if order != 2:
            sim.set_order(order)
        if eps is not None or sigma is not None:
            sim.set_material(eps, None, sigma)
        if src is not None:
            sim.set_source(*src)
        sim.set_fields(fields)
        sim.step(warm)
        sim.synchronize()
        stream = torch.cuda.ExternalStream(sim._stream.value) if sim._stream.value else torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        sim.close()
        return nx * ny * nz * steps / (ms / 1e3)

    def cpu(nx, ny, nz, d, scheme, cfl, fields, eps=None, steps=2):
        g = G.Grid(nx, ny, nz, d, d, d)
        P = S.Problem(g, cfl * g.dt_cfl(), eps_r_cell=eps)
        u = S.fadi_init(P, fields) if scheme == "fadi" else {c: fields[c].copy() for c in G.COMPS}
        step = {"fadi": S.fadi_step, "flod": S.flod_step, "fss": S.fss_step}[scheme]
        t0 = time.perf_counter()
        for k in range(steps):
            u = step(P, u, k)
        return nx * ny * nz * steps / (time.perf_counter() - t0)

    out = []
    w = W.workload_2d_gaussian()
    out.append({"workload": "2-D TM FADI 64x64, CFL 5", "f64": gpu(64, 64, 1, 1e-3, "fadi", "f64", 5.0, w.fields,
                                                                  steps=200),
                "f32": gpu(64, 64, 1, 1e-3, "fadi", "f32", 5.0, w.fields, steps=200),
                "oracle_1core": cpu(64, 64, 1, 1e-3, "fadi", 5.0, w.fields, steps=20)})
    w = W.workload_cavity_modes()
    out.append({"workload": "FADI 128^3 cavity, CFL 4, 8 modes",
                "f32": gpu(128, 128, 128, 1e-3, "fadi", "f32", 4.0, w.fields, steps=200),
                "f64": gpu(128, 128, 128, 1e-3, "fadi", "f64", 4.0, w.fields, steps=50),
                "oracle_1core": cpu(128, 128, 128, 1e-3, "fadi", 4.0, w.fields, steps=2)})
    f256 = workload_fields(256)
    out.append({"workload": "FADI 256^3 cavity, CFL 4, 8 modes (no per-launch timing)",
                "f32": gpu(256, 256, 256, 1e-3, "fadi", "f32", 4.0, f256, steps=200),
                "f64": gpu(256, 256, 256, 1e-3, "fadi", "f64", 4.0, f256, steps=20)})
    out.append({"workload": "FADI 256^3 cavity, CFL 4, 8 modes, fourth-order differences",
                "f32": gpu(256, 256, 256, 1e-3, "fadi", "f32", 4.0, f256, steps=40, order=4),
                "f64": gpu(256, 256, 256, 1e-3, "fadi", "f64", 4.0, f256, steps=10, order=4)})
    out.append({"workload": "FADI 256^3 cavity, CFL 4, 8 modes, eps_r 2.5, uniform sigma 0.05 S/m (lossy)",
                "f32": gpu(256, 256, 256, 1e-3, "fadi", "f32", 4.0, f256, steps=200,
                           eps=np.full((256, 256, 256), 2.5), sigma=np.full((256, 256, 256), 0.05))})
    del f256
    n = 256
    d = 0.5e-3
    eps = W.eps_blocks(3, n, n, n, 1.0, 10.0)
    dt = 8.0 / (299792458.0 * math.sqrt(3.0 / d ** 2))
    cur = W.dipole_current((np.arange(200) + 0.5) * dt)
    z = W.zero_fields(n, n, n)
    for scheme in ("flod", "fss"):
        out.append({"workload": f"{scheme.upper()} 256^3, eps_r blocks U[1,10], CFL 8, z dipole",
                    "f32": gpu(n, n, n, d, scheme, "f32", 8.0, z, eps, ("ez", 128, 128, 128, cur), steps=100),
                    "f64": gpu(n, n, n, d, scheme, "f64", 8.0, z, eps, ("ez", 128, 128, 128, cur), steps=20),
                    "oracle_1core": cpu(n, n, n, d, scheme, 8.0, z, eps, steps=1)})
    sig = np.where(eps > 5.0, 0.5, 0.0)
    out.append({"workload": "FLOD 256^3, eps_r blocks U[1,10] with sigma 0.5 S/m where eps_r > 5 (lossy), CFL 8, "
                            "z dipole",
                "f32": gpu(n, n, n, d, "flod", "f32", 8.0, z, eps, ("ez", 128, 128, 128, cur), steps=100,
                           sigma=sig)})
    for o in out:
        o["unit"] = "cell-steps/s"
        print(json.dumps(o), flush=True)


def main():
    args = parse()
    if args.suite:
        from paper_2011_14043_gb300 import build
        build()
        suite(args)
        return
    ws, rank, local = dist_env()
    if args.impl == "reference":
        reference_arm(args)
        return
    import torch
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2011_14043_gb300 import build
    build()
    fields = workload_fields(args.n)
    n = args.n
    cells = n ** 3

    # --- device-resident timed region (FP32 headline) -------------------------
    sampler = ClockSampler(local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.4)
    r32 = run_gpu(args, "f32", fields, keep_fields=(rank == 0 and not args.no_fp64))
    clocks = sampler.stop()
    ms, value = replica_throughput(r32["ms"], cells * args.steps, ws, "cuda")

    # dominant kernel roofline from live CUDA events in the timed region
    st = r32["stats"]
    peaks, peak_kind = measured_peaks()
    cls_names = ["y-lines", "z-lines", "x-lines"]
    dom = max(range(3), key=lambda c: st["timed_ms"][c])
    kernel_steps = st["timed_launches"][0] // 2 if st["timed_launches"][0] else 0
    avg_ms = st["timed_ms"][dom] / max(1, st["timed_launches"][dom])
    achieved = st["bytes_per_launch"][dom] / (avg_ms / 1e3) / 1e9
    per_class = {cls_names[c]: {"launches": st["timed_launches"][c],
                                "avg_ms": st["timed_ms"][c] / max(1, st["timed_launches"][c]),
                                "gbs": st["bytes_per_launch"][c] / (st["timed_ms"][c] / max(1, st["timed_launches"][c]) / 1e3) / 1e9
                                if st["timed_ms"][c] > 0 else None}
                 for c in range(3)}
    step_bytes = 96.0 * cells  # 2 procedures x 6 arrays x (4 B read + 4 B write)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": recorded_traffic(cls_names[dom], n),
                "kernel": f"proc line solve, {cls_names[dom]}", "peak_kind": peak_kind,
                "kernel_timing": f"per-launch CUDA event pairs on the handle's stream over a serialised pass of "
                                 f"{kernel_steps} steps of the same kernels right after the timed region (the "
                                 f"timed region runs the three pairs of each procedure concurrently)",
                "step_achieved": step_bytes * args.steps / (r32["ms"] / 1e3) / 1e9,
                "step_frac": step_bytes * args.steps / (r32["ms"] / 1e3) / 1e9 / peaks["hbm_gbs"],
                "per_class": per_class}

    # FP32 state: six arrays in the padded layout (rows of x rounded up to 32)
    state = 6 * ((n + 1 + 31) // 32 * 32) * (n + 1) ** 2 * 4
    l2_note = (f"state {state / 1e6:.0f} MB > 129 MB L2, no flush" if state > 129e6 else
               f"state {state / 1e6:.0f} MB fits the 129 MB L2: timings are L2-resident")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"FADI {n}^3 PEC cavity, 1 mm cells, vacuum, CFL {args.cfl}, 8 seeded modes",
                   "grid": [n, n, n], "scheme": "fadi", "parallelism": f"replicas x{ws}",
                   "l2": l2_note},
        "roofline": roofline,
        "gpu_launches": r32["launches"],
        "clocks": clocks,
    }
    if rank == 0 and not args.no_fp64:
        a = argparse.Namespace(**vars(args))
        a.steps = max(3, min(args.steps, 20))
        r64 = run_gpu(a, "f64", fields, time_kernels=False)
        v64 = cells * a.steps / (r64["ms"] / 1e3)
        ref = fp64_reference_fields(args, fields, r32["total_steps"])
        line["accuracy"] = {"fp32_vs_fp64_rel_l2": device_rel_err(r32["fields"], ref),
                            "steps": r32["total_steps"],
                            "norm": "relative L2 in the vacuum energy norm, FP32 GPU path against the FP64 GPU "
                                    "path after the same steps from the same initial field"}
        del ref
        r32["fields"] = None
        line["fp64"] = {"value": v64, "unit": UNIT, "ms_per_step": r64["ms"] / a.steps, "steps": a.steps,
                        "hbm_frac": 192.0 * cells * a.steps / (r64["ms"] / 1e3) / 1e9 / peaks["hbm_gbs"],
                        "roofline": fp64_alu_roofline(v64)}
    if not args.no_e2e:
        e = run_e2e(args, "f32", fields)
        ev = ws * cells * args.steps / e["s"]
        line["e2e"] = {"value": ev, "unit": UNIT, "h2d_bytes_per_step": e["h2d"] / args.steps,
                       "d2h_bytes_per_step": e["d2h"] / args.steps,
                       "timing": "median of 3 timed rounds after one untimed round, host clock around "
                                 "set_field x6, step(K), get_field x6 with pinned buffers",
                       "samples": [ws * cells * args.steps / t for t in e["samples_s"]]}
    if not args.no_batch:
        line["batch"] = batch_section(args)
    if not args.no_adjoint:
        line["adjoint"] = adjoint_section(args)
    if rank == 0 and not args.no_cpu_baseline:
        v1, s1 = cpu_baseline(n, steps=1)
        procs, cores = oracle_processes(n)
        va, sa = oracle_replicas(n, args.cfl, 0, 1, procs)
        line["cpu_baseline"] = {"value": va, "unit": UNIT, "cores": procs, "host_cores": cores, "kind": "oracle",
                                "sample": f"1 FADI step of the full {n}^3 workload on each of {procs} concurrent "
                                          f"processes (FP64 numpy oracle, one core each, {sa:.1f} s wall; "
                                          f"{cores} host cores)",
                                "single_core": {"value": v1, "cores": 1,
                                                "sample": f"1 FADI step of the full {n}^3 workload, one process "
                                                          f"({s1:.1f} s)"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
