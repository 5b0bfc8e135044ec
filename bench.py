#!/usr/bin/env python
"""Throughput of the GB300 pressurized phase-field fracture solver.

One benchmark step = the whole hot path on one problem, solved to
convergence by the Newton / active-set method with FGMRES + block AMG on the
device (mixed precision: FP32 V-cycles inside the FP64 outer iteration),
followed by TCV and the COD at 64 points.

Default line (the largest single-GPU configuration): the 3d penny-shaped
Sneddon crack, [-2,2]^3 graded 128^3 Q1 hexes from h_min = 4e-3 (8,586,756
DoFs), one loading step at p = 1e-3.  The same run measures the 2d graded
Sneddon ramp (1024^2 cells graded from h_min = 2e-4 on [-10,10]^2, 3,151,875
DoFs, five loading steps to p = 1e-3) the same way and reports it under
"workloads".  --workload penny3d / graded2d prints one of them alone.

value  = DoF/s = (loading steps solved x DoFs) / device time, inputs resident
         in HBM (the state is reset from device buffers each step); the timed
         region carries no instrumentation.
e2e    = the same through the C ABI with host buffers: the initial state is
         copied host -> device and the solution device -> host every step.
fp64_path = the plain FP64 GPU path (FP64 V-cycles too) on the same steps.
roofline  = the dominant kernel, timed with CUDA event pairs in a separate
         instrumented step after the timed region; the coarse AMG levels (one
         CUDA graph replay per V-cycle) are reported beside it.
cpu_baseline / --impl reference = the CPU oracle (oracle/) on a bounded sample
         of the same workload recipe, on the host cores.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
       [--workload default|penny3d|graded2d] [--cells C]   (C: the same recipe at
              C cells per axis, small cases for profiler captures)
       [--workload batched [--instances 256] [--workers 16]]
              256 independent 2d instances (32^2..512^2) through the batch executor
       [--workload served [--requests 12] [--loads 0.5,1,2,4] [--budget-gb 150]]
              a Poisson stream of mixed 2d / 3d 10-step requests through the server,
              at each arrival rate (multiples of the FP64 one-at-a-time service rate)
       [--workload adaptive [--adapt-n0 64] [--adapt-cycles 6]]
              the adaptive 2d Sneddon sequence (refine -> transfer -> solve, eps = 2h)
              next to the uniform mesh of the same finest h
Multi-GPU runs (torchrun) are independent replicas: each rank solves its own
copy of the workload; value sums the ranks' work over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Newton-Krylov solves/s & DoF/s at <=1e-8 rel err; p50/p99 latency; HBM GB/s"
UNIT = "DoF/s"
# workload recipes: index of the standard configuration, CPU-oracle sample size
# (cells per axis) and loading steps of the sample
WORKLOADS = {
    "penny3d": {"index": 2, "sample_cells": 16, "sample_steps": 1},
    "graded2d": {"index": 1, "sample_cells": 128, "sample_steps": 2},
}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def host_cpu():
    """Model name and logical core count of the host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith("model name"):
                        model = line.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    return {"model": model or platform.machine(), "arch": platform.machine(), "nproc": os.cpu_count()}


# ------------------------------------------------------------ CPU oracle ----
ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import workloads as W
from oracle import fe, model, pdas
w = W.scaled_workload(W.config({idx}), {cells})
mesh = fe.Mesh(w.coords)
prm = model.Params(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, p=w.pressures[0])
st = pdas.State.initial(mesh, prm, w.phi0())
times = []
for k in range({nsteps}):
    p = w.pressures[k % len(w.pressures)]
    if k % len(w.pressures) == 0 and k > 0:
        st = pdas.State.initial(mesh, prm, w.phi0())
    t = time.perf_counter()
    rep = pdas.loading_step(st, p)
    times.append(time.perf_counter() - t)
print(json.dumps({{"times": times, "n_dofs": w.n_dofs, "name": w.name}}))
"""


def run_oracle(kind: str, nsteps: int):
    spec = WORKLOADS[kind]
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    code = ORACLE_SNIPPET.format(root=ROOT, idx=spec["index"], cells=spec["sample_cells"],
                                 nsteps=nsteps)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                         check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def cpu_baseline(kind: str):
    spec = WORKLOADS[kind]
    r = run_oracle(kind, spec["sample_steps"])
    total = sum(r["times"])
    c = spec["sample_cells"]
    cells = f"{c}^3" if kind == "penny3d" else f"{c}^2"
    return {"value": spec["sample_steps"] * r["n_dofs"] / total, "unit": UNIT, "cores": 1,
            "kind": "oracle", "host": host_cpu(),
            "sample": f"{spec['sample_steps']} loading step(s) of the same recipe at {cells} cells "
                      f"({r['n_dofs']} DoFs), {total:.1f} s single-threaded (FP64 numpy/scipy, "
                      f"exact sparse LU solves)"}


def reference_arm(args, rank, world):
    if rank != 0:
        return 0
    kind = "penny3d" if args.workload == "default" else args.workload
    spec = WORKLOADS[kind]
    r = run_oracle(kind, args.warmup + args.steps)
    times = r["times"][args.warmup:]
    total = sum(times)
    value = len(times) * r["n_dofs"] / total
    c = spec["sample_cells"]
    cells = f"{c}^3" if kind == "penny3d" else f"{c}^2"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": r["name"], "loading_steps_per_step": 1,
                                            "n_dofs": r["n_dofs"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": 1,
                             "host": host_cpu(),
                             "sample": f"one loading step per bench step at {cells} cells "
                                       f"({r['n_dofs']} DoFs) of the {kind} recipe"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ clocks ----
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "-i", self.gpu_id,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names[1:], parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# -------------------------------------------------------------- GPU arm ----
def _source_hash(rel_path: str) -> str:
    with open(os.path.join(ROOT, rel_path), "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def _traffic_for(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu
    summary, or None when there is none or the source file of the kernel changed
    since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            e = json.load(f).get(f"{kernel}@{workload}")
        if not e or e.get("source_sha256") != _source_hash(e["source"]):
            return None
        return e.get("dram_bytes_per_launch_full_size")
    except Exception:
        return None


def _cod_points(w, fn, np):
    xs = fn.cod_points(w.l0, 64)
    if w.dim == 2:
        return xs
    return np.stack([xs, np.zeros_like(xs)], axis=1).ravel()   # lines along z through y = 0


COARSE = ("coarse_levels_graph_u", "coarse_levels_graph_phi")


def measure_problem(kind, args, rank, world, local_rank, dist, with_fp64=True):
    """Time one workload (mixed precision) as the module docstring describes and
    return the fields of its bench line."""
    import numpy as np
    import torch
    import paper_1806_09924_gb300 as pff
    import workloads as W
    from oracle import functionals as fn   # COD sample points only

    w = W.config(WORKLOADS[kind]["index"])
    if args.cells:
        w = W.scaled_workload(w, args.cells)
    dev = torch.device("cuda", local_rank)
    opts = pff.options(precision=pff.PFF_PREC_MIXED)
    # the profiled step runs the two preconditioner blocks one after the other,
    # so every kernel is timed alone (isolated efficiencies)
    opts_isolated = pff.options(precision=pff.PFF_PREC_MIXED, precond_overlap=0)
    stream = torch.cuda.Stream(device=dev)
    P = pff.problem_from_workload(w)
    P.set_stream(stream)
    n, d = P.n_nodes, w.dim
    phi0_h = w.phi0()
    u0_h = np.zeros((n, d))
    u0 = torch.zeros(n * d, dtype=torch.float64, device=dev)
    phi0 = torch.tensor(phi0_h, device=dev)
    pts = _cod_points(w, fn, np)
    pressures = list(w.pressures)

    def step_device(Q, o):
        Q.set_state_dev(u0, phi0, phi0, phi0, 0)
        reps = Q.solve_loading_steps(pressures, o)
        tcv, cod = Q.eval_tcv_cod(pts)
        return reps, tcv, cod

    def step_e2e():
        P.set_state(u0_h, phi0_h, phi0_h, phi0_h, 0)
        reps = P.solve_loading_steps(pressures, opts)
        tcv, cod = P.eval_tcv_cod(pts)
        P.get_solution()
        return reps, tcv, cod

    def timed(Q, o, steps):
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        reps = []
        for _ in range(steps):
            reps.append(step_device(Q, o))
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        if dist:
            t = torch.tensor([ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms, reps

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step_device(P, opts)
        # timed region: resident inputs, no instrumentation
        sampler = ClockSampler(_gpu_id(torch, local_rank))
        sampler.start()
        launches0 = pff.launch_count()
        ms, runs = timed(P, opts, args.steps)
        launches = pff.launch_count() - launches0
        clocks = sampler.stop()
        reps, tcv, cod = runs[-1]
        # instrumented step 1: blocks serialised, every kernel timed (isolated)
        pff.profile_select(None)
        pff.profile_enable(True)
        step_device(P, opts_isolated)
        iso = pff.profile_report()
        pff.profile_enable(False)
        kern = {k: v for k, v in iso.items() if v["bytes"] > 0 and k not in COARSE}
        top_name = max(kern.items(), key=lambda kv: kv[1]["ms"])[0] if kern else None
        # instrumented step 2: as timed (blocks concurrent), the roofline kernel and
        # the coarse-level graph replays timed with event pairs on their streams
        pff.profile_select(",".join([top_name, *COARSE]) if top_name else ",".join(COARSE))
        pff.profile_enable(True)
        step_device(P, opts)
        live = pff.profile_report()
        pff.profile_enable(False)
        pff.profile_select(None)
        # e2e through host buffers
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step_e2e()
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = max(e0.elapsed_time(e1), 1e3 * (time.perf_counter() - t0))
        if dist:
            t = torch.tensor([e2e_ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_ms = float(t.item())
        u_m, phi_m, _ = P.get_solution()
        P.close()
        # the plain FP64 GPU path on the same steps (FP64 V-cycles and Gram-Schmidt)
        fp64 = None
        if with_fp64:
            Q = pff.problem_from_workload(w)
            Q.set_stream(stream)
            o64 = pff.options(precision=pff.PFF_PREC_FP64)
            step_device(Q, o64)
            ms64, runs64 = timed(Q, o64, args.steps)
            u_f, phi_f, _ = Q.get_solution()
            Q.close()
            solves = args.steps * len(pressures) * world
            fp64 = {"value": solves * w.n_dofs / (ms64 / 1e3), "unit": UNIT,
                    "solves_per_s": solves / (ms64 / 1e3), "ms_per_step": ms64 / args.steps,
                    "newton_its": [r["newton_its"] for r in runs64[-1][0]],
                    "krylov_its": [r["krylov_its"] for r in runs64[-1][0]],
                    "mixed_speedup": ms64 / ms,
                    "rel_err_mixed_vs_fp64": {
                        "u": float(np.linalg.norm(u_m - u_f) / np.linalg.norm(u_f)),
                        "phi": float(np.linalg.norm(phi_m - phi_f) / np.linalg.norm(phi_f)),
                        "u_max_norm": float(np.max(np.abs(u_m - u_f)) / np.max(np.abs(u_f))),
                        "phi_max_norm": float(np.max(np.abs(phi_m - phi_f)) / np.max(np.abs(phi_f)))}}

    solves = args.steps * len(pressures)
    dofs = solves * w.n_dofs * world
    value = dofs / (ms / 1e3)
    h2d = n * (d + 3) * 8
    d2h = n * (d * 8 + 8 + 1) + 8 * (len(pts) // (d - 1) + 1)
    peak, peak_kind = _peaks()

    def rate(st):
        if not st or st["ms"] <= 0 or st["bytes"] <= 0:
            return None
        per = st["bytes"] / max(st["count"], 1)
        avg = st["ms"] / max(st["count"], 1)
        ach = per / (avg / 1e3) / 1e9
        return {"achieved": ach, "frac": ach / peak, "launches": st["count"],
                "avg_launch_us": 1e3 * avg, "algorithmic_bytes_per_launch": per}

    roof = None
    if top_name and top_name in live:
        r_live = rate(live[top_name])
        roof = {"bound": "hbm", "kernel": top_name, "achieved": r_live["achieved"], "peak": peak,
                "unit": "GB/s", "frac": r_live["frac"], "traffic": _traffic_for(top_name, w.name),
                "peak_source": f"{peak_kind} hbm_gbs (copy bandwidth)",
                "launches": r_live["launches"], "avg_launch_us": r_live["avg_launch_us"],
                "algorithmic_bytes_per_launch": r_live["algorithmic_bytes_per_launch"],
                "share_of_step_time": live[top_name]["ms"] / (ms / args.steps),
                "timing": "CUDA event pair around every launch of this kernel during one "
                          "instrumented step after the timed region, blocks concurrent as in the "
                          "timed steps (the kernel shares HBM with the other block's V-cycle)"}
        r_iso = rate(iso.get(top_name))
        if r_iso:
            roof["isolated"] = dict(r_iso, timing="instrumented step with the two preconditioner "
                                                  "blocks one after the other, CUDA events")
        coarse = {}
        for name in COARSE:
            r = rate(live.get(name))
            ri = rate(iso.get(name))
            if r:
                coarse[name] = dict(r, isolated=ri,
                                    note="one CUDA graph replay = every kernel of AMG levels >= 1 "
                                         "of one V-cycle; bytes = their summed algorithmic bytes")
        roof["coarse_levels"] = coarse
    last = reps
    out = {
        "value": value, "ms_per_step": ms / args.steps,
        "dtype": "f64+f32",
        "config": {"workload": w.name, "n_cells": "x".join(str(c) for c in w.n_cells),
                   "n_dofs": w.n_dofs, "loading_steps_per_step": len(pressures),
                   "precision": "mixed: FP32 AMG V-cycles (and FP32 views of the Krylov basis for "
                                "the Gram-Schmidt coefficients) inside FP64 FGMRES / Newton; "
                                "residuals, updates, active sets and TCV/COD in FP64",
                   "grading": ("geometric from h_min=4e-3, ratio solved to fill [-2,2]" if kind == "penny3d"
                               else "geometric from h_min=2e-4, ratio solved to fill [-10,10]"),
                   "l2": "no flush: the working set (state, stencils, AMG, Krylov basis) is "
                         "several GB, > L2",
                   "parallelism": f"replicas x{world}"},
        "solves_per_s": solves * world / (ms / 1e3),
        "newton_its": [r["newton_its"] for r in last],
        "krylov_its": [r["krylov_its"] for r in last],
        "krylov_its_max": [r["krylov_its_max"] for r in last],
        "locked": [r["locked"] for r in last],
        "tcv": tcv, "cod_center": float(cod[len(cod) // 2]),
        "fp64_path": fp64,
        "gpu_launches": int(launches),
        "e2e": {"value": dofs / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "roofline": roof,
        "kernels_isolated_step": {
            k: {"count": v["count"], "ms": round(v["ms"], 3),
                "GB/s": (v["bytes"] / (v["ms"] / 1e3) / 1e9) if v["ms"] > 0 and v["bytes"] > 0 else None}
            for k, v in sorted(iso.items(), key=lambda kv: -kv[1]["ms"])[:16]},
        "clocks": clocks,
    }
    return out


def gpu_arm(args, rank, world, local_rank):
    import torch
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    kinds = ["penny3d", "graded2d"] if args.workload == "default" else [args.workload]
    results = {k: measure_problem(k, args, rank, world, local_rank, dist,
                                  with_fp64=not args.no_fp64) for k in kinds}
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    main_kind = kinds[0]
    r = results[main_kind]
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": r["dtype"],
            "data": "synthetic"}
    line.update({k: v for k, v in r.items() if k not in line})
    if world == 1 and not args.no_cpu_baseline:
        for k in kinds:
            try:
                results[k]["cpu_baseline"] = cpu_baseline(k)
            except Exception as e:   # the CPU leg must not hide the GPU number
                results[k]["cpu_baseline"] = {"error": str(e)[:200]}
        line["cpu_baseline"] = results[main_kind]["cpu_baseline"]
    if len(kinds) > 1:
        line["workloads"] = {results[k]["config"]["workload"]: results[k] for k in kinds[1:]}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------ multi-rank helpers ----
def shard(items, rank: int, world: int):
    """Weak scaling over ranks: rank r takes every world-th item (no data-path exchange)."""
    return list(items)[rank::world]


def reduce_across_ranks(value: float, op: str, dist=None, device="cpu") -> float:
    """max / sum of a host scalar over the ranks of the default process group."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------- batched / served modes ----
def _gpu_id(torch, local_rank):
    try:
        return "GPU-" + str(torch.cuda.get_device_properties(local_rank).uuid)
    except Exception:
        return str(local_rank)


def batched_arm(args, rank, world, local_rank):
    """256 independent 2d instances (32^2..512^2, one loading step each) solved
    concurrently by the batch executor; the one-at-a-time solve of the same
    instances is timed beside it."""
    import torch
    import paper_1806_09924_gb300 as pff
    import workloads as W
    torch.cuda.set_device(local_rank)
    inst = shard(W.batched_instances(args.instances), rank, world)
    probs = [pff.problem_from_workload(w) for w in inst]
    opts = pff.options(precision=pff.PFF_PREC_MIXED)
    scheds = [w.pressures for w in inst]
    dofs = sum(w.n_dofs * len(w.pressures) for w in inst)

    def reset():
        for P, w in zip(probs, inst):
            P.set_crack(w.l0)
        torch.cuda.synchronize()

    def run(workers):
        reset()
        t0 = time.perf_counter()
        reports, status = pff.batch_solve(probs, scheds, opts, workers=workers)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if any(s != 0 for s in status):
            raise RuntimeError(f"batch solve failed: {status}")
        return dt, reports

    for _ in range(args.warmup):
        run(args.workers)
    sampler = ClockSampler(_gpu_id(torch, local_rank))
    sampler.start()
    launches0 = pff.launch_count()
    times = []
    for _ in range(args.steps):
        dt, reports = run(args.workers)
        times.append(dt)
    launches = pff.launch_count() - launches0
    clocks = sampler.stop()
    seq, _ = run(1)          # one at a time, same instances (untimed in value)
    dist = None
    if world > 1:
        import torch.distributed as dist
    total = reduce_across_ranks(sum(times), "max", dist, "cuda")
    dofs_all = reduce_across_ranks(dofs, "sum", dist, "cuda")
    n_all = int(reduce_across_ranks(len(inst), "sum", dist, "cuda"))
    for P in probs:
        P.close()
    if rank != 0:
        return 0
    value = dofs_all * args.steps / total
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": "batched_sneddon2d_256", "instances": n_all,
                   "cells": "32^2..512^2 (seed 1806)", "loading_steps_per_instance": 1,
                   "n_dofs_total": dofs_all, "workers": args.workers,
                   "parallelism": f"instances sharded over {world} rank(s)",
                   "l2": "instances total several GB, > L2"},
        "solves_per_s": n_all * args.steps / total,
        "one_at_a_time": {"value": dofs / seq, "unit": UNIT, "s": seq},
        "speedup_vs_one_at_a_time": seq * args.steps / total,
        "newton_its_total": sum(r[0]["newton_its"] for r in reports),
        "krylov_its_total": sum(r[0]["krylov_its"] for r in reports),
        "gpu_launches": int(launches), "clocks": clocks,
        "timing": "host wall clock around the synchronous batch call, state reset before",
    }
    print(json.dumps(line), flush=True)
    return 0


ADAPT_ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import workloads as W
from oracle import adapt, fe, model, pdas
w, sched = W.adaptive_sneddon2d({n0}, {cycles})
coords, dofs = w.coords, 0
t0 = time.perf_counter()
for hk, eps in sched:
    mesh = fe.Mesh(coords)
    prm = model.Params(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=eps, p=w.pressures[0])
    st = pdas.State.initial(mesh, prm, W.crack_phi(coords, w.l0))
    pdas.solve_loading_steps(st, w.pressures)
    dofs += 3 * mesh.n_nodes
    coords, _ = adapt.refine(mesh, st.u, st.phi, W.ADAPT_THETA, hk / 2.0, W.ADAPT_PHI_BAND)
print(json.dumps({{"dofs": dofs, "s": time.perf_counter() - t0}}))
"""


def adaptive_arm(args, rank, world, local_rank):
    """The adaptive 2d Sneddon sequence (Section 3 refinement strategy, Section
    4.4 study): from a uniform 64^2 mesh, six cycles of solve (eps = 2 h_k,
    from u = 0 with the crack set on the new mesh) -> indicator / marking /
    refinement, down to h = 1/512 in the crack region; next to it the uniform
    mesh with the same finest h (global refinement) solved once."""
    import numpy as np
    import torch
    import paper_1806_09924_gb300 as pff
    import workloads as W
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w, sched = W.adaptive_sneddon2d(args.adapt_n0, args.adapt_cycles)
    opts = pff.options(precision=pff.PFF_PREC_MIXED)
    stream = torch.cuda.Stream(device=dev)

    def sequence():
        coords, prev, out = w.coords, None, []
        for hk, eps in sched:
            Q = pff.Problem(coords)
            Q.set_stream(stream)
            Q.set_material(w.E, w.nu, w.Gc, w.kappa, eps)
            Q.set_crack(w.l0)
            if prev is not None:
                prev.close()
            reps = Q.solve_loading_steps(w.pressures, opts)
            coords_next = Q.refine_axes(W.ADAPT_THETA, hk / 2.0, W.ADAPT_PHI_BAND)
            out.append((Q.n_dofs, [len(c) - 1 for c in coords], reps[0]))
            coords, prev = coords_next, Q
        tcv, cod = prev.eval_tcv_cod([0.0])
        prev.close()
        return out, tcv, cod[0]

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            sequence()
        sampler = ClockSampler(_gpu_id(torch, local_rank))
        sampler.start()
        launches0 = pff.launch_count()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            cycles, tcv, cod0 = sequence()
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / args.steps
        launches = pff.launch_count() - launches0
        clocks = sampler.stop()
        # roofline: one instrumented sequence after the timed region
        pff.profile_select(None)
        pff.profile_enable(True)
        sequence()
        prof = pff.profile_report()
        pff.profile_enable(False)
        # global refinement at the same finest h, solved once
        h_fin, eps_fin = sched[-1]
        n_uni = int(round(4.0 / h_fin))
        ax = W.uniform_axis(n_uni, -2.0, 2.0)
        U = pff.Problem([ax, ax.copy()])
        U.set_stream(stream)
        U.set_material(w.E, w.nu, w.Gc, w.kappa, eps_fin)
        U.set_crack(w.l0)
        torch.cuda.synchronize()
        tu = time.perf_counter()
        U.solve_loading_steps(w.pressures, opts)
        tcv_u, cod_u = U.eval_tcv_cod([0.0])
        torch.cuda.synchronize()
        tu = time.perf_counter() - tu
        n_uni_dofs = U.n_dofs
        U.close()
    if rank != 0:
        return 0
    dofs = sum(c[0] for c in cycles)
    peak, peak_kind = _peaks()
    kern = {k: v for k, v in prof.items() if v["bytes"] > 0 and k not in COARSE}
    roof = None
    if kern:
        name, st = max(kern.items(), key=lambda kv: kv[1]["ms"])
        per = st["bytes"] / max(st["count"], 1)
        avg = st["ms"] / max(st["count"], 1) / 1e3
        ach = per / avg / 1e9
        ind = prof.get("jump_indicator")
        roof = {"bound": "hbm", "kernel": name, "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "traffic": None, "peak_source": f"{peak_kind} hbm_gbs",
                "launches": st["count"], "avg_launch_us": 1e6 * avg,
                "algorithmic_bytes_per_launch": per,
                "note": "meshes of 13k-60k DoFs: every kernel is latency- and launch-bound",
                "jump_indicator": None if not ind else {
                    "launches": ind["count"], "avg_launch_us": 1e3 * ind["ms"] / max(ind["count"], 1),
                    "GB/s": ind["bytes"] / (ind["ms"] / 1e3) / 1e9 if ind["ms"] > 0 else None}}
    cpu = None
    if not args.no_cpu_baseline:
        env = dict(os.environ)
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            env[k] = "1"
        code = ADAPT_ORACLE_SNIPPET.format(root=ROOT, n0=32, cycles=4)
        r = json.loads(subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                                      env=env, check=True).stdout.strip().splitlines()[-1])
        cpu = {"value": r["dofs"] / r["s"], "unit": UNIT, "cores": 1, "kind": "oracle",
               "host": host_cpu(),
               "sample": f"the same sequence from a uniform 32^2 mesh, 4 cycles ({r['dofs']} DoFs "
                         f"solved), {r['s']:.1f} s single-threaded"}
    line = {
        "metric": METRIC, "value": dofs / dt, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dt, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": w.name, "cycles": len(sched),
                   "h": [h for h, _ in sched], "eps": [e for _, e in sched],
                   "theta": W.ADAPT_THETA, "phi_band": W.ADAPT_PHI_BAND,
                   "l2": "small meshes (< L2); each cycle allocates a new problem",
                   "parallelism": "one GPU"},
        "cycles": [{"dofs": c[0], "cells": c[1], "newton_its": c[2]["newton_its"],
                    "krylov_its": c[2]["krylov_its"]} for c in cycles],
        "tcv": tcv, "cod0": cod0,
        "uniform_same_h": {"dofs": n_uni_dofs, "s": tu, "tcv": tcv_u, "cod0": float(cod_u[0]),
                           "rel_diff_tcv": (tcv - tcv_u) / tcv_u,
                           "rel_diff_cod0": (cod0 - float(cod_u[0])) / float(cod_u[0]),
                           "adaptive_speedup": tu / dt},
        "gpu_launches": int(launches),
        "e2e": {"value": dofs / dt, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 16,
                "note": "host wall clock around the whole sequence, meshes and crack set from the "
                        "host each cycle"},
        "roofline": roof, "cpu_baseline": cpu, "clocks": clocks,
        "timing": "host wall clock around each adaptive sequence (problem creation, solves, "
                  "refinement, transfer), synchronized",
    }
    print(json.dumps(line), flush=True)
    return 0


def served_arm(args, rank, world, local_rank):
    """Poisson stream of mixed 2d / 3d requests (10-step ramps) through the
    request server under a device-memory budget; p50 / p99 latency and
    throughput, next to the plain FP64 one-at-a-time GPU path on the same
    requests (which also sets the arrival rate)."""
    import numpy as np
    import torch
    import paper_1806_09924_gb300 as pff
    import workloads as W
    torch.cuda.set_device(local_rank)
    if rank != 0:
        return 0
    reqs = W.served_requests(args.requests, steps=10)
    budget = int(args.budget_gb * (1 << 30))
    cod_x = [0.0]

    def closed_loop(opts, workers):
        S = pff.Server(budget, workers, opts)
        t0 = time.perf_counter()
        ids = [S.submit(w, cod_x=cod_x) for w, _ in reqs]
        res = [S.wait(i) for i in ids]
        dt = time.perf_counter() - t0
        S.close()
        if any(r["status"] != 0 for r in res):
            raise RuntimeError("a request failed")
        return dt, res

    # plain FP64 one-at-a-time GPU path: service rate mu
    base_s, base = closed_loop(pff.options(precision=pff.PFF_PREC_FP64), 1)
    # the served form with every request queued at once (throughput bound)
    mixed_s, _ = closed_loop(pff.options(precision=pff.PFF_PREC_MIXED), args.workers)
    mu = len(reqs) / base_s
    loads = [float(x) for x in args.loads.split(",") if x.strip()]
    steps = sum(len(w.pressures) for w, _ in reqs)
    dofs = sum(w.n_dofs * len(w.pressures) for w, _ in reqs)

    def open_loop(load):
        """Requests arrive at Poisson times (unit-rate gaps / lambda) while others run."""
        lam = load * mu
        S = pff.Server(budget, args.workers, pff.options(precision=pff.PFF_PREC_MIXED))
        arrivals = np.cumsum([g for _, g in reqs]) / lam
        t0 = time.perf_counter()
        ids = []
        for (w, _), ta in zip(reqs, arrivals):
            delay = ta - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            ids.append(S.submit(w, cod_x=cod_x))
        res = [S.wait(i) for i in ids]
        makespan = time.perf_counter() - t0
        stats = S.stats()
        S.close()
        if any(r["status"] != 0 for r in res):
            raise RuntimeError("a request failed")
        lat = np.array([r["t_finish"] - r["t_submit"] for r in res])
        return {"load_vs_fp64_service_rate": load, "rate_per_s": lam, "makespan_s": makespan,
                "solves_per_s": steps / makespan, "dof_per_s": dofs / makespan,
                "latency_s": {"p50": float(np.percentile(lat, 50)),
                              "p99": float(np.percentile(lat, 99)), "mean": float(lat.mean())},
                "server": stats}

    sampler = ClockSampler(_gpu_id(torch, local_rank))
    sampler.start()
    launches0 = pff.launch_count()
    sweep = [open_loop(x) for x in loads]
    launches = pff.launch_count() - launches0
    clocks = sampler.stop()
    head = sweep[min(range(len(sweep)), key=lambda i: abs(loads[i] - 1.0))]
    base_lat = np.array([r["t_finish"] - r["t_submit"] for r in base])
    line = {
        "metric": METRIC, "value": head["dof_per_s"], "unit": UNIT, "n_gpus": 1, "steps": 1,
        "warmup": 0, "ms_per_step": 1e3 * head["makespan_s"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": "served_mixed_2d3d", "requests": len(reqs),
                   "mix": f"{sum(1 for w, _ in reqs if w.dim == 2)} 2d (64^2..1024^2 graded), "
                          f"{sum(1 for w, _ in reqs if w.dim == 3)} 3d (32^3..128^3 graded), seed 1807",
                   "loading_steps_per_request": 10, "arrivals": "Poisson",
                   "loads_vs_fp64_service_rate": loads, "headline_load": head["load_vs_fp64_service_rate"],
                   "budget_gb": args.budget_gb, "workers": args.workers},
        "solves_per_s": head["solves_per_s"],
        "latency_s": head["latency_s"],
        "sweep": sweep,
        "closed_loop_mixed": {"value": dofs / mixed_s, "unit": UNIT, "solves_per_s": steps / mixed_s,
                              "note": "all requests queued at t = 0, same server"},
        "fp64_one_at_a_time": {"value": dofs / base_s, "unit": UNIT, "solves_per_s": steps / base_s,
                               "service_rate_per_s": mu,
                               "latency_s_closed_loop": {"p50": float(np.percentile(base_lat, 50)),
                                                         "p99": float(np.percentile(base_lat, 99))}},
        "gpu_launches": int(launches), "clocks": clocks,
        "timing": "host wall clock from the first arrival to the last completion, per load",
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 GPU path")
    ap.add_argument("--cells", type=int, default=0,
                    help="run the same recipe at this many cells per axis (profiling captures)")
    ap.add_argument("--workload", default="default",
                    choices=["default", "penny3d", "graded2d", "batched", "served", "adaptive"],
                    help="default: the 3d penny 128^3 line with the graded 2d 1024^2 ramp measured "
                         "beside it; penny3d / graded2d: one of them; batched: 256 independent "
                         "instances; served: a Poisson request stream")
    ap.add_argument("--instances", type=int, default=256)
    ap.add_argument("--workers", type=int, default=16)
    ap.add_argument("--requests", type=int, default=12)
    ap.add_argument("--loads", default="0.5,1,2,4",
                    help="served: arrival rates as multiples of the FP64 one-at-a-time service rate")
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--adapt-n0", type=int, default=64,
                    help="adaptive: cells per axis of the uniform start mesh")
    ap.add_argument("--adapt-cycles", type=int, default=6)
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if args.workload not in ("default", "penny3d", "graded2d"):
            if rank == 0:
                print(json.dumps({"impl": "reference", "unavailable":
                                  "the reference arm times the oracle on single-problem workloads only"}))
            return 0
        return reference_arm(args, rank, world)
    if args.workload == "batched":
        if world > 1:
            import torch
            import torch.distributed as dist
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
        return batched_arm(args, rank, world, local_rank)
    if args.workload == "served":
        return served_arm(args, rank, world, local_rank)
    if args.workload == "adaptive":
        return adaptive_arm(args, rank, world, local_rank)
    return gpu_arm(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
