#!/usr/bin/env python3
"""Benchmark of the cue-field + growth-cone hot path on one GB300 per rank.

Default workload: 2D 2048^2 grid, D = 1, lambda = 0.005, dt = 0.2, no-flux
walls, 64 sources (emission ~ U[0.5, 2]), 16,384 cones that stop within
radius 2 of a source or at the walls, 5,000 coupled steps.  One benchmark
step is one whole simulation of that workload from its initial state (all
field and cone rows of every time step); the state reset and an L2 flush
(a 512 MiB write) sit between timed steps, outside the timed events.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cue cell-updates/s + axon-steps/s, %HBM roofline; adjoint & batched vs plain"
UNIT = "cell-updates/s"
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["cue", "reference"], default="cue")
    ap.add_argument("--workload", default="c2", choices=["c1", "c2", "c2x", "c3", "c4", "c5", "graph"])
    ap.add_argument("--path", default="auto", choices=list(PATHS))
    ap.add_argument("--batch-mode", default="auto", choices=["auto", "persist", "step", "blocked"],
                    help="batched workload: run mode (auto = the autotuner's choice)")
    ap.add_argument("--batch-rows", type=int, default=0,
                    help="with a fixed --batch-mode: rows per field tile (0 = library choice)")
    ap.add_argument("--batch-blocks", type=int, default=0,
                    help="with --batch-mode persist: blocks per SM (0 = library choice)")
    ap.add_argument("--depth", type=int, default=0,
                    help="temporal depth on the fused path, or of the blocked batch mode with --workload c4 "
                         "(0 = auto / autotuned)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-probe", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="CPU-baseline sample budget")
    ap.add_argument("--run-steps", type=int, default=0,
                    help="time steps per benchmark step (0 = the workload's own count); for profiling")
    ap.add_argument("--subs", default="clustered,c3,batched,adjoint,whole_run",
                    help="with the default workload: sub-figures added to its line (comma list of clustered, c3, "
                         "batched, adjoint, whole_run; empty for none)")
    ap.add_argument("--whole-run-cones", type=int, default=2048,
                    help="cones the oracle follows over a whole run (the first ones)")
    # internal: time the oracle with its field rows over threads, in a process of its own
    # (no CUDA context, no second OpenMP runtime next to PyTorch's): WORKLOAD:NSTEPS:THREADS
    ap.add_argument("--oracle-threads-sample", default="", help=argparse.SUPPRESS)
    # internal: the oracle over a whole run in a process of its own: WORKLOAD:NCONES:OUT
    ap.add_argument("--oracle-whole-run", default="", help=argparse.SUPPRESS)
    return ap.parse_args()


def workload(name, rank=0):
    from paper_1405_3331_gb300 import workloads as W
    if name == "c1":
        return W.config_c1(seed=0 + 100 * rank)
    if name == "c2":
        return W.config_c2(seed=1 + 100 * rank)
    if name == "c2x":
        return W.config_c2_clustered(seed=8 + 100 * rank)
    if name == "c3":
        return W.config_c3(seed=2 + 100 * rank)
    if name == "c5":
        return W.config_c5(seed=4 + 100 * rank)
    raise KeyError(name)


def describe(w):
    dims = f"{w.nx}x{w.ny}" + (f"x{w.nz}" if w.dim == 3 else "")
    return {
        "workload": f"{w.dim}D {dims} cue field + {w.n_axons} growth cones, {w.nsteps} steps",
        "grid": dims, "n_src": w.n_src, "n_axons": w.n_axons, "steps_per_run": w.nsteps,
        "D": w.D, "lambda": w.lam, "dt": w.dt, "stop_radius": w.stop_radius,
        "wall_mode": "clamp" if w.wall_mode else "stop", "source_map": w.src_map is not None,
        "l2": "flushed between timed steps (512 MiB write)",
    }


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.out = None

    def start(self):
        try:
            self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if self.gpu_id is not None:
                cmd += ["-i", str(self.gpu_id)]
            self.proc = subprocess.Popen(cmd, stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.flush()
        self.out.seek(0)
        rows = [r.split(",") for r in self.out.read().splitlines() if r.strip()]
        os.unlink(self.out.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for name, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_id_for(device_index):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",")]
        if device_index < len(ids):
            return ids[device_index]
    return device_index


# ------------------------------------------------------------------ traffic
def source_digest():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1405_3331_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel, work):
    """DRAM bytes per launch from the committed ncu summary, if taken on this source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d[f"{kernel}@{work}"]
        if e.get("source_digest") != source_digest():
            return None
        return float(e["dram_bytes_per_launch"])
    except Exception:
        return None


# ------------------------------------------------------------------ CPU oracle
def oracle_sample(w, budget_s):
    """Time the FP64 oracle (single thread, as it stands) on the first steps of the workload."""
    import numpy as np
    import oracle
    g = oracle.Grid(w.dim, w.nx, w.ny, w.nz if w.dim == 3 else 1, h=w.h, D=w.D, lam=w.lam, dt=w.dt)
    c = oracle.Cone(w.w_prev, w.w_grad, w.w_noise, w.step_len, w.stop_radius, w.grad_eps, w.wall_mode,
                    w.seed)
    C = w.field0().astype(np.float64)
    t0 = time.perf_counter()
    oracle.run(g, c, C, 0, 1, w.src_cell, w.src_emit, w.src_map, w.pos, w.dir, w.active)
    one = time.perf_counter() - t0
    nsteps = max(1, min(w.nsteps, int(budget_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    _, _, _, act = oracle.run(g, c, C, 0, nsteps, w.src_cell, w.src_emit, w.src_map, w.pos, w.dir,
                              w.active)
    dt = time.perf_counter() - t0
    return nsteps, dt


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform string)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_threads_child(spec):
    """Child process: the oracle on the first NSTEPS steps of WORKLOAD with the field's node
    loop over THREADS threads; prints {"seconds", "threads", "nsteps"}."""
    name, nsteps, threads = spec.split(":")
    if name.startswith("c4"):
        from paper_1405_3331_gb300 import workloads as W
        w = W.config_c4(seed=3)[0]
    else:
        w = workload(name)
    import numpy as np
    import oracle
    used = oracle.set_threads(int(threads))
    g = oracle.Grid(w.dim, w.nx, w.ny, w.nz if w.dim == 3 else 1, h=w.h, D=w.D, lam=w.lam, dt=w.dt)
    c = oracle.Cone(w.w_prev, w.w_grad, w.w_noise, w.step_len, w.stop_radius, w.grad_eps, w.wall_mode,
                    w.seed)
    C = w.field0().astype(np.float64)
    oracle.run(g, c, C, 0, 1, w.src_cell, w.src_emit, w.src_map, w.pos, w.dir, w.active)
    t0 = time.perf_counter()
    oracle.run(g, c, C, 0, int(nsteps), w.src_cell, w.src_emit, w.src_map, w.pos, w.dir, w.active)
    print(json.dumps({"seconds": time.perf_counter() - t0, "threads": used, "nsteps": int(nsteps)}), flush=True)
    return 0


def oracle_threads_sample(name, n_cells, nsteps, sample):
    """The same bounded sample as the single-threaded baseline, the field's node loop over
    every host core (rows are independent; the cone loop stays serial)."""
    threads = os.cpu_count() or 1
    try:
        out = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-threads-sample",
                              f"{name}:{nsteps}:{threads}"], capture_output=True, text=True, timeout=300)
        d = json.loads(out.stdout.strip().splitlines()[-1])
    except Exception as e:                      # the baseline is context, not a result
        return {"unavailable": f"{type(e).__name__}"}
    return {"value": n_cells * d["nsteps"] / d["seconds"], "unit": UNIT, "cores": d["threads"],
            "kind": "oracle, field rows over OpenMP threads", "sample": sample, "seconds": d["seconds"]}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if args.workload == "graph":
        return run_reference_graph(args)
    w = workload(args.workload)
    import numpy as np
    import oracle
    g = oracle.Grid(w.dim, w.nx, w.ny, w.nz if w.dim == 3 else 1, h=w.h, D=w.D, lam=w.lam, dt=w.dt)
    c = oracle.Cone(w.w_prev, w.w_grad, w.w_noise, w.step_len, w.stop_radius, w.grad_eps, w.wall_mode,
                    w.seed)
    C0 = w.field0().astype(np.float64)
    # each reference step: a bounded sample (the first S time steps) of the workload
    t0 = time.perf_counter()
    oracle.run(g, c, C0, 0, 1, w.src_cell, w.src_emit, w.src_map, w.pos, w.dir, w.active)
    one = time.perf_counter() - t0
    total_budget = 150.0
    S = max(1, min(w.nsteps, int(total_budget / max(1, args.steps + args.warmup) / max(one, 1e-6))))
    for _ in range(args.warmup):
        oracle.run(g, c, C0, 0, S, w.src_cell, w.src_emit, w.src_map, w.pos, w.dir, w.active)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.run(g, c, C0, 0, S, w.src_cell, w.src_emit, w.src_map, w.pos, w.dir, w.active)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = w.n_cells * S * args.steps / total
    sample = f"first {S} of {w.nsteps} time steps of the workload per step (field + cones), from C0"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": describe(w),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                         "host_cores": os.cpu_count(), "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ ranks
def aggregate(local_ms, units_per_step, steps, world, dist=None, device=None):
    """Whole-job figures: the slowest rank's time, and the units all ranks processed per second.

    Each rank runs its own replica (no data-path collective); `local_ms` is this rank's summed
    device time for `steps` steps.  Returns (max_ms, value)."""
    t = float(local_ms)
    if dist is not None and world > 1:
        import torch
        x = torch.tensor([t], dtype=torch.float64, device=device)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        t = float(x.item())
    return t, world * units_per_step * steps / (t / 1e3)


# ------------------------------------------------------------------ GPU arm
PATHS = ("auto", "plain", "fused", "persist", "resident", "cluster")


def path_code(cue, name):
    return {"auto": cue.CUE_PATH_AUTO, "plain": cue.CUE_PATH_PLAIN, "fused": cue.CUE_PATH_FUSED,
            "persist": cue.CUE_PATH_PERSIST, "resident": cue.CUE_PATH_RESIDENT, "cluster": cue.CUE_PATH_CLUSTER}[name]


class Runner:
    """One simulation handle over a workload, with its initial state kept on the device so that
    every benchmark step restarts from it (reset and L2 flush outside the timed events)."""

    def __init__(self, cue, torch, dev, w, path="auto", depth=0, flush=None):
        self.cue, self.torch, self.w = cue, torch, w
        self.sim = cue.Simulation(w, device=dev, path=path_code(cue, path))
        if depth:
            self.sim.set_option(cue.CUE_OPT_TEMPORAL_DEPTH, depth)
        self.stream = self.sim.stream
        s = self.sim
        self.init = (s.fields[0].clone(), s.pos.clone(), s.dir.clone(), s.active.clone())
        self.flush = flush

    def reset(self):
        s, torch = self.sim, self.torch
        with torch.cuda.stream(self.stream):
            for dst, src in zip((s.fields[0], s.pos, s.dir, s.active), self.init):
                dst.copy_(src)
        self.cue._check(self.cue.cue_set_state(s.h, 0, 0, 0), "cue_set_state")

    def timed_runs(self, steps, warmup, barrier, sampler=None, sample_period=16):
        """``warmup`` untimed runs, then ``steps`` timed whole runs.  Returns a dict with the
        per-run device times, the launches of the timed region, the cone updates of one run and
        the CUDA-event times of every ``sample_period``-th launch of the dominant kernel."""
        torch, sim, w = self.torch, self.sim, self.w
        for i in range(max(warmup, 3)):
            self.reset()
            if i == max(warmup, 3) - 1:
                sim.cone_updates()
            sim.sim_run(w.nsteps)
        sim.check()
        cone_updates = sim.cone_updates()
        path = sim_path_used(sim)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        sim.set_option(self.cue.CUE_OPT_TIME_KERNEL, 1 if path in ("persist", "resident", "cluster")
                       else sample_period)
        sim.kernel_time()
        barrier()
        if sampler is not None:
            sampler.start()
        launches0 = sim.launches()
        for k in range(steps):
            with torch.cuda.stream(self.stream):
                self.flush.zero_()
            self.reset()
            evs[k][0].record(self.stream)
            sim.sim_run(w.nsteps)
            evs[k][1].record(self.stream)
        barrier()
        clocks = sampler.stop() if sampler is not None else None
        launches = sim.launches() - launches0
        kern_ms, kern_n = sim.kernel_time()
        sim.set_option(self.cue.CUE_OPT_TIME_KERNEL, 0)
        sim.check()
        return {"run_ms": [a.elapsed_time(b) for a, b in evs], "launches": launches, "cone_updates": cone_updates,
                "sampled_ms": kern_ms, "sampled_n": kern_n, "clocks": clocks, "path": path}

    def close(self):
        self.sim.close()


def dominant_kernel(sim, w):
    """(name, launches of the dominant kernel in one run, steps one launch covers)."""
    path = sim_path_used(sim)
    if path == "fused":
        K = sim.get_option(sim_cue().CUE_INFO_DEPTH)
        if w.dim == 3:          # an odd last step runs on the one-step kernel
            return "fused3d", w.nsteps // K, K
        return "fused", (w.nsteps + K - 1) // K, K
    if path in ("persist", "resident", "cluster"):
        return path, 1, w.nsteps
    return ("step3d" if w.dim == 3 else "field"), w.nsteps, 1


def sim_cue():
    from paper_1405_3331_gb300 import cue
    return cue


def roofline_single(sim, w, rec, ms_per_run, hbm, peak_kind, work):
    """Roofline of the dominant kernel.  achieved = 8 B per node update (12 B with a rate map;
    the 3D step launch also moves its cones' state) x the node updates one launch makes, over
    the launch's time.  The launch time is the timed runs' device time over the dominant
    kernel's launches in them: on these paths the dominant kernel is all but all of a run (the
    committed launch lists), so launches x time never exceeds the run.  The CUDA-event figure of
    sampled launches is kept beside it (events between back-to-back launches inflate it)."""
    name, per_run, K = dominant_kernel(sim, w)
    bpc = 12 if w.src_map is not None else 8
    units = w.n_cells * K
    alg = bpc * units
    if name == "step3d":
        alg += w.n_axons * (4 * w.dim * 4 + 1)
    avg_s = ms_per_run / per_run / 1e3
    achieved = alg / avg_s / 1e9
    # compulsory traffic: a launch reads and writes its field once however many steps it covers
    one_pass = bpc * w.n_cells * (1 if name in ("fused", "fused3d") else K)
    r = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
         "traffic": recorded_traffic({"step3d": "field"}.get(name, name), work), "kernel": name,
         "peak_kind": peak_kind, "launches_per_run": per_run, "steps_per_launch": K,
         "node_updates_per_launch": units, "algorithmic_bytes_per_launch": alg,
         "avg_launch_us": avg_s * 1e6,
         "launch_time": "device time of the timed runs / launches of the dominant kernel in them",
         "compulsory_bytes_per_launch": one_pass, "compulsory_gbs": one_pass / avg_s / 1e9,
         "compulsory_frac": one_pass / avg_s / 1e9 / hbm}
    if rec["sampled_n"]:
        r["sampled_launch_us"] = rec["sampled_ms"] / rec["sampled_n"] * 1e3
    if name == "resident":
        r["note"] = ("one block holds the grid in shared memory for the whole run: HBM is read and "
                     "written once per launch; a step is bound by one SM's shared-memory and issue rate")
    return r


def single_summary(runner, rec, hbm, peak_kind, work, world=1):
    w = runner.w
    ms = statistics.median(rec["run_ms"])
    return {"workload": describe(w)["workload"], "path": rec["path"], "value": world * w.n_cells * w.nsteps / (ms / 1e3),
            "unit": UNIT, "ms_per_run": ms, "runs": len(rec["run_ms"]),
            "axon_steps_per_s": world * rec["cone_updates"] / (ms / 1e3),
            "roofline": roofline_single(runner.sim, w, rec, ms, hbm, peak_kind, work),
            "gpu_launches_per_run": rec["launches"] / max(1, len(rec["run_ms"])),
            **({"helper_blocks": runner.sim.get_option(sim_cue().CUE_INFO_HELPERS)}
               if rec["path"] == "fused" and w.dim == 2 else {})}


def main():
    args = parse_args()
    if args.oracle_threads_sample:
        return oracle_threads_child(args.oracle_threads_sample)
    if args.oracle_whole_run:
        return oracle_whole_run_child(args.oracle_whole_run)
    if args.impl == "reference":
        return run_reference(args)
    import torch
    from paper_1405_3331_gb300 import build as cue_build
    cue_build.build()
    from paper_1405_3331_gb300 import cue

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    if args.workload == "c4":
        return main_batch(args, torch, cue, dev, rank, world, dist, barrier)
    if args.workload == "graph":
        return main_graph(args, torch, dev, rank, world, dist, barrier)
    w = workload(args.workload, rank)
    if args.run_steps:
        w.nsteps = args.run_steps
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    hbm, peak_kind = peaks()
    run = Runner(cue, torch, dev, w, args.path, args.depth, flush)
    rec = run.timed_runs(args.steps, args.warmup, barrier, ClockSampler(gpu_id_for(local)))
    local_ms = sum(rec["run_ms"])
    cells_per_run = w.n_cells * w.nsteps
    total_ms, value = aggregate(local_ms, cells_per_run, args.steps, world, dist, dev)
    ms_run = total_ms / args.steps
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_run, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": describe(w),
        "parallelism": f"replicas x{world}" if world > 1 else "single GPU", "path": rec["path"],
        "axon_steps_per_s": world * rec["cone_updates"] * args.steps / (total_ms / 1e3),
        "cone_updates_per_run": rec["cone_updates"],
        "roofline": roofline_single(run.sim, w, rec, ms_run, hbm, peak_kind, args.workload),
        "clocks": rec["clocks"], "gpu_launches": rec["launches"],
    }
    if rec["path"] == "fused" and w.dim == 2:
        line["helper_blocks"] = run.sim.get_option(cue.CUE_INFO_HELPERS)

    # end to end through the public API from pinned host buffers
    if not args.no_e2e:
        line["e2e"] = e2e_single(torch, run, args.steps, barrier, world)

    subs = [s for s in args.subs.split(",") if s] if (args.workload == "c2" and not args.run_steps) else []
    if rank == 0 and "whole_run" in subs:
        final_c2 = final_state(run)
    run.close()
    if rank == 0:
        # the rest of the metric on the same GPU: the same grid with its cones clustered, the 3D
        # workload, the batch against the one-instance-per-launch solver, the adjoint against
        # the forward solvers
        if "clustered" in subs:
            wx = workload("c2x")
            rx = Runner(cue, torch, dev, wx, flush=flush)
            recx = rx.timed_runs(3, 2, barrier)
            line["clustered"] = single_summary(rx, recx, hbm, peak_kind, "c2x")
            line["clustered"]["ms_per_run_vs_uniform"] = line["clustered"]["ms_per_run"] / ms_run
            rx.close()
        if "c3" in subs:
            w3 = workload("c3")
            r3 = Runner(cue, torch, dev, w3, flush=flush)
            rec3 = r3.timed_runs(3, 2, barrier)
            line["c3"] = single_summary(r3, rec3, hbm, peak_kind, "c3")
            if "whole_run" in subs:
                final_c3 = final_state(r3)
            r3.close()
            # the opt-in temporally blocked 3D path (two steps per launch) on the same workload
            r3b = Runner(cue, torch, dev, w3, path="fused", flush=flush)
            rec3b = r3b.timed_runs(2, 1, barrier)
            ms3b = statistics.median(rec3b["run_ms"])
            line["c3"]["blocked_path"] = {
                "path": rec3b["path"], "ms_per_run": ms3b, "value": w3.n_cells * w3.nsteps / (ms3b / 1e3),
                "unit": UNIT, "vs_default_path": line["c3"]["ms_per_run"] / ms3b,
                "roofline": roofline_single(r3b.sim, w3, rec3b, ms3b, hbm, peak_kind, "c3")}
            r3b.close()
        if "batched" in subs:
            line["batched"] = batch_summary(args, torch, cue, dev, rank, barrier, flush, hbm, peak_kind)
        if "adjoint" in subs:
            line["adjoint"] = adjoint_summary(cue, torch, dev, flush, barrier, hbm, peak_kind)
    if w.targets is not None and w.wall_mode == 1 and rank == 0 and args.workload == "c5":
        r5 = Runner(cue, torch, dev, w, flush=flush)
        line["adjoint"] = adjoint_timing(cue, torch, r5, w, ms_run)
        r5.close()

    # HBM probes: the unblocked field kernels on grids that cannot stay in L2
    if not args.no_probe and rank == 0:
        line["hbm_probe"] = hbm_probe(cue, torch, dev, hbm)
        if w.dim == 3 or "c3" in subs:
            line["hbm_probe_3d"] = hbm_probe(cue, torch, dev, hbm, dim=3)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        nsteps, secs = oracle_sample(w, args.cpu_seconds)
        sample = f"first {nsteps} of {w.nsteps} time steps of the same workload (FP64)"
        line["cpu_baseline"] = {
            "value": w.n_cells * nsteps / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": sample + ", one thread", "seconds": secs, "host_cores": os.cpu_count(),
            "cpu_model": cpu_model()}
        line["cpu_baseline_threads"] = oracle_threads_sample(args.workload, w.n_cells, nsteps, sample)
    if rank == 0 and "whole_run" in subs:
        # FP32-vs-FP64 after the full runs (oracle in a child process over every host core)
        line["whole_run"] = {"c2": whole_run_report("c2", final_c2, args.whole_run_cones)}
        if "c3" in subs:
            line["whole_run"]["c3"] = whole_run_report("c3", final_c3, args.whole_run_cones)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def e2e_single(torch, run, steps, barrier, world):
    """The same runs through Simulation.run_host: state from pinned host buffers, field and
    cones back into pinned host buffers, copies inside the timed events."""
    w, sim = run.w, run.sim
    host = [torch.from_numpy(a).pin_memory() for a in (w.field0(), w.pos, w.dir, w.active)]
    out = tuple(torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in host)
    sim.run_host(*host, w.nsteps, out=out)     # warm
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(1, min(steps, 3))
    barrier()
    tot = 0.0
    for _ in range(reps):
        with torch.cuda.stream(run.stream):
            run.flush.zero_()
        e0.record(run.stream)
        sim.run_host(*host, w.nsteps, out=out)
        e1.record(run.stream)
        e1.synchronize()
        tot += e0.elapsed_time(e1)
    return {"value": world * w.n_cells * w.nsteps * reps / (tot / 1e3), "unit": UNIT,
            "h2d_bytes_per_step": sum(t.numel() * t.element_size() for t in host),
            "d2h_bytes_per_step": sum(t.numel() * t.element_size() for t in out), "ms_per_step": tot / reps}


def final_state(run):
    """State after the last timed full run (numpy): field, initial and final cone positions, active."""
    C, pos, dirs, act, fs, cs = run.sim.snapshot()
    assert fs == run.w.nsteps
    return {"C": C, "pos": pos, "act": act}


# ------------------------------------------------------------------ batched workload
def build_batch(torch, dev, ws):
    from paper_1405_3331_gb300 import batch as B
    b = B.Batch(ws, device=dev)
    init = [(b.fields[i][0].clone(), b.pos[i].clone(), b.dir[i].clone(), b.active[i].clone())
            for i in range(len(ws))]

    def reset():
        with torch.cuda.stream(b.stream):
            for i, (C, p, d, a) in enumerate(init):
                b.fields[i][0].copy_(C)
                b.pos[i].copy_(p)
                b.dir[i].copy_(d)
                b.active[i].copy_(a)
        b.reset_state(0, 0)
    return b, init, reset


def batch_timed(torch, b, reset, T, steps, warmup, barrier, flush, sampler=None):
    for _ in range(max(warmup, 3)):
        reset()
        b.run(T)
    b.check()
    b.cone_updates()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    barrier()
    if sampler is not None:
        sampler.start()
    for k in range(steps):
        with torch.cuda.stream(b.stream):
            flush.zero_()
        reset()
        evs[k][0].record(b.stream)
        b.run(T)
        evs[k][1].record(b.stream)
    barrier()
    clocks = sampler.stop() if sampler is not None else None
    b.check()
    return [x.elapsed_time(y) for x, y in evs], b.cone_updates() / steps, clocks


def batch_mode_name(B, b):
    mode = b.get_option(B.CUE_BOPT_MODE)
    rows = b.get_option(B.CUE_BOPT_ROWS)
    depth = b.get_option(B.CUE_BOPT_DEPTH)
    if mode == 1:
        return "persist", "one persistent launch per run", 1
    if mode == 3:
        return "blocked", f"one temporally blocked launch per {depth} steps", depth
    return "step", ("per time step one launch over every instance's cone chunks and streamed field tiles"
                    if rows > 4 else "per time step one launch over the cone chunks and one over the field tiles"), 1


def batch_roofline(B, b, cells, T, ms_run, hbm, peak_kind):
    name, _, K = batch_mode_name(B, b)
    per_run = 1 if name == "persist" else (T + K - 1) // K
    avg_s = ms_run / per_run / 1e3
    alg = 8.0 * cells * (T if name == "persist" else K)
    one_pass = 8.0 * cells * (T if name == "persist" else 1)
    return {"bound": "hbm", "achieved": alg / avg_s / 1e9, "peak": hbm, "unit": "GB/s",
            "frac": alg / avg_s / 1e9 / hbm, "traffic": recorded_traffic(name, "c4"), "kernel": name,
            "peak_kind": peak_kind, "launches_per_run": per_run, "steps_per_launch": T if name == "persist" else K,
            "algorithmic_bytes_per_launch": alg, "avg_launch_us": avg_s * 1e6,
            "launch_time": "device time of the timed runs / launches of the dominant kernel in them",
            "compulsory_bytes_per_launch": one_pass, "compulsory_frac": one_pass / avg_s / 1e9 / hbm}


def sequential_rate(torch, cue, dev, ws, path, Tb=100):
    """Every instance alone, one after another, ``Tb`` steps each (a rate, so runs of other
    lengths compare directly); each Simulation has its own stream, so instances may overlap on
    the GPU, which only favours this baseline."""
    sims = [cue.Simulation(w, device=dev, path=path) for w in ws]
    for sm in sims:
        sm.sim_run(2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for sm in sims:
        sm.sim_run(Tb)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    for sm in sims:
        sm.check()
        sm.close()
    return sum(w.n_cells for w in ws) * Tb / dt


def batch_summary(args, torch, cue, dev, rank, barrier, flush, hbm, peak_kind):
    """The 512-instance workload (sub-figure of the default line): autotuned, graph-replayed,
    against the one-instance-per-launch plain solver and one sim_run per instance."""
    from paper_1405_3331_gb300 import batch as B
    from paper_1405_3331_gb300 import workloads as W
    ws = W.config_c4(seed=3 + 100 * rank)
    T = ws[0].nsteps
    cells = sum(w.n_cells for w in ws)
    b, init, reset = build_batch(torch, dev, ws)
    tuned = b.autotune(16)
    b.set_option(B.CUE_BOPT_GRAPH, 1)
    run_ms, cone_updates, _ = batch_timed(torch, b, reset, T, 3, 2, barrier, flush)
    ms = statistics.median(run_ms)
    value = cells * T / (ms / 1e3)
    plain = sequential_rate(torch, cue, dev, ws, cue.CUE_PATH_PLAIN)
    auto = sequential_rate(torch, cue, dev, ws, cue.CUE_PATH_AUTO)
    name, launch, K = batch_mode_name(B, b)
    out = {"workload": f"batched: {len(ws)} independent 2D instances (sides U{{64..1024}}, {cells / 1e6:.1f} M "
                       f"cells, {sum(w.n_axons for w in ws)} cones), {T} steps",
           "value": value, "unit": UNIT, "ms_per_run": ms, "runs": len(run_ms),
           "axon_steps_per_s": cone_updates / (ms / 1e3),
           "launch": launch + ", replayed from a CUDA graph", "autotuned": autotune_record(B, b, tuned),
           "roofline": batch_roofline(B, b, cells, T, ms, hbm, peak_kind),
           "vs_plain_per_instance": {"value": plain, "unit": UNIT, "speedup": value / plain,
                                     "sample": f"all {len(ws)} instances x 100 steps, each instance its own "
                                               "cone and field launches per step"},
           "vs_sequential_sim_run": {"value": auto, "unit": UNIT, "speedup": value / auto,
                                     "sample": f"all {len(ws)} instances x 100 steps, one sim_run per instance "
                                               "in turn (the library's own path choice)"}}
    b.close()
    return out


def autotune_record(B, b, tuned):
    rows, bpsm, ms = tuned[:3]
    name, _, depth = batch_mode_name(B, b)
    return {"mode": name, "rows": rows, "blocks_per_sm": bpsm, "depth": depth, "probe_ms_per_step": ms,
            "candidates": "persistent (rows 1, 2, 4 x blocks per SM 1..3), one launch per step (rows 2..16), "
                          "temporally blocked (depth 2, 4, 8)"}


def main_batch(args, torch, cue, dev, rank, world, dist, barrier):
    """512 independent 2D instances of uneven sizes and physics, 1,000 coupled steps, replayed
    from a captured CUDA graph, run mode, tile shape and temporal depth chosen by the
    autotuner.  One benchmark step = the whole batch from its initial state."""
    from paper_1405_3331_gb300 import batch as B
    from paper_1405_3331_gb300 import workloads as W
    ws = W.config_c4(seed=3 + 100 * rank)
    T = args.run_steps or ws[0].nsteps
    cells = sum(w.n_cells for w in ws)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    b, init, reset = build_batch(torch, dev, ws)
    if args.depth:                       # a fixed blocked depth (profiling): no autotuner
        b.set_option(B.CUE_BOPT_MODE, 3)
        b.set_option(B.CUE_BOPT_DEPTH, args.depth)
        tuned = (0, 0, 0.0)
    elif args.batch_mode in ("persist", "step"):     # a fixed mode (profiling): no autotuner
        b.set_option(B.CUE_BOPT_MODE, 1 if args.batch_mode == "persist" else 2)
        b.set_option(B.CUE_BOPT_ROWS, args.batch_rows)
        b.set_option(B.CUE_BOPT_BLOCKS, args.batch_blocks)
        tuned = (0, 0, 0.0)
    else:
        tuned = b.autotune(16)
    b.set_option(B.CUE_BOPT_GRAPH, 1)
    run_ms, cone_updates, clocks = batch_timed(torch, b, reset, T, args.steps, args.warmup, barrier, flush,
                                               ClockSampler(gpu_id_for(dev.index or 0)))
    local_ms = sum(run_ms)
    total_ms, value = aggregate(local_ms, cells * T, args.steps, world, dist, dev)
    hbm, peak_kind = peaks()
    name, launch, K = batch_mode_name(B, b)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batched: {len(ws)} independent 2D instances (sides U{{64..1024}}, "
                               f"{cells / 1e6:.1f} M cells, {sum(w.n_axons for w in ws)} cones), {T} steps",
                   "instances": len(ws), "cells": cells, "steps_per_run": T,
                   "l2": "flushed between timed steps (512 MiB write); 1.2 GB working set"},
        "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
        "launch": launch + ", replayed from a CUDA graph", "autotuned": autotune_record(B, b, tuned),
        "axon_steps_per_s": world * cone_updates * args.steps / (total_ms / 1e3),
        "roofline": batch_roofline(B, b, cells, T, total_ms / args.steps, hbm, peak_kind),
        "clocks": clocks,
        "gpu_launches": args.steps * (2 if name == "persist" else
                                      ((T + K - 1) // K if name == "blocked" else
                                       (T if b.get_option(B.CUE_BOPT_ROWS) > 4 else 2 * T)) + 1),
    }
    plain = sequential_rate(torch, cue, dev, ws, cue.CUE_PATH_PLAIN)
    auto = sequential_rate(torch, cue, dev, ws, cue.CUE_PATH_AUTO)
    line["baseline_plain_per_instance"] = {
        "value": plain, "unit": UNIT, "speedup": value / world / plain,
        "sample": f"all {len(ws)} instances x 100 steps, each instance its own cone and field launches per step"}
    line["baseline_sequential_sim_run"] = {
        "value": auto, "unit": UNIT, "speedup": value / world / auto,
        "sample": f"all {len(ws)} instances x 100 steps, one sim_run per instance in turn (the library's own "
                  "path choice)"}
    if not args.no_e2e:
        # end to end: every instance's state from pinned host memory, the run, the fields back
        host = [tuple(t.cpu().pin_memory() for t in st) for st in init]
        outs = [torch.empty_like(h[0]).pin_memory() for h in host]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(b.stream)
        with torch.cuda.stream(b.stream):
            for i, (C, p, d, a) in enumerate(host):
                b.fields[i][0].copy_(C, non_blocking=True)
                b.pos[i].copy_(p, non_blocking=True)
                b.dir[i].copy_(d, non_blocking=True)
                b.active[i].copy_(a, non_blocking=True)
        b.reset_state()
        b.run(T)
        cur = b.get_option(B.CUE_BINFO_CUR)
        with torch.cuda.stream(b.stream):
            for i in range(len(ws)):
                outs[i].copy_(b.fields[i][cur], non_blocking=True)
        e1.record(b.stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        line["e2e"] = {"value": cells * T / (ms / 1e3), "unit": UNIT,
                       "h2d_bytes_per_step": sum(sum(t.numel() * t.element_size() for t in h) for h in host),
                       "d2h_bytes_per_step": sum(o.numel() * o.element_size() for o in outs), "ms_per_step": ms}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        nsteps, secs = oracle_sample(ws[0], args.cpu_seconds)
        sample = f"instance 0 ({ws[0].nx}x{ws[0].ny}), first {nsteps} of {T} steps (FP64)"
        line["cpu_baseline"] = {
            "value": ws[0].n_cells * nsteps / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": sample + ", one thread", "seconds": secs, "host_cores": os.cpu_count(),
            "cpu_model": cpu_model()}
        line["cpu_baseline_threads"] = oracle_threads_sample("c4", ws[0].n_cells, nsteps, sample)
    b.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------ adjoint workload
def adjoint_summary(cue, torch, dev, flush, barrier, hbm, peak_kind):
    """The adjoint workload (1024^2, 32 sources, 4,096 cones, 2,000 steps, checkpoint every 64):
    sim_adjoint against the fastest forward run (the library's own path) and the plain forward
    solver (one cone and one field launch per step) of the same workload."""
    from paper_1405_3331_gb300 import workloads as W
    w = W.config_c5()
    fwd = Runner(cue, torch, dev, w, flush=flush)
    frec = fwd.timed_runs(3, 2, barrier)
    plain = Runner(cue, torch, dev, w, path="plain", flush=flush)
    prec = plain.timed_runs(3, 2, barrier)
    plain.close()
    out = adjoint_timing(cue, torch, fwd, w, statistics.median(frec["run_ms"]))
    # the same gradients with the whole run stored once (ckpt_every >= nsteps: no recompute,
    # nsteps + 1 states of workspace)
    stored = adjoint_timing(cue, torch, fwd, w, out["forward_ms_per_run"], k=w.nsteps)
    out["stored_run"] = {k: stored[k] for k in ("ms_per_run", "ratio_to_forward", "ckpt_every")}
    out["stored_run"]["workspace_bytes"] = cue.cue_adjoint_workspace_bytes(fwd.sim.params, fwd.sim.n_src,
                                                                           fwd.sim.n_axons, w.nsteps, w.nsteps)
    out["forward_path"] = frec["path"]
    out["plain_forward_ms_per_run"] = statistics.median(prec["run_ms"])
    out["ratio_to_plain_forward"] = out["ms_per_run"] / out["plain_forward_ms_per_run"]
    out["stored_run"]["ratio_to_plain_forward"] = out["stored_run"]["ms_per_run"] / out["plain_forward_ms_per_run"]
    out["forward_roofline"] = roofline_single(fwd.sim, w, frec, out["forward_ms_per_run"], hbm, peak_kind, "c5")
    fwd.close()
    return out


def adjoint_timing(cue, torch, run, w, forward_ms, k=64, reps=3):
    """Time sim_adjoint (forward with checkpoints every k steps, recompute, backward) on the
    runner's workload from its initial state; the ratio divides by the timed forward run."""
    sim = run.sim
    run.reset()
    sim.adjoint(w.targets, w.nsteps, k)          # warm (and the workspace)
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        with torch.cuda.stream(run.stream):
            run.flush.zero_()
        run.reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(run.stream)
        g = sim.adjoint(w.targets, w.nsteps, k)
        e1.record(run.stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    sim.check()
    ms = statistics.median(times)
    return {"workload": describe(w)["workload"] + ", gradients of the endpoint loss",
            "ms_per_run": ms, "runs": reps, "forward_ms_per_run": forward_ms, "ratio_to_forward": ms / forward_ms,
            "ckpt_every": k, "loss": float(g["loss"]), "dL_dD": float(g["dD"]),
            "dL_dlambda": float(g["dlambda"]), "dL_de_max": float(g["dsrc"].abs().max()),
            "dL_dM_max": float(g["dmap"].abs().max())}


# ------------------------------------------------------------------ whole runs against the oracle
def oracle_whole_run_child(spec):
    """Child process: the oracle over the whole run of WORKLOAD (field on every host core, the
    first NCONES cones; cones never interact, so a prefix of them follows exactly the paths it
    follows among all of them, its Philox counters being the cone indices); saves the final
    field and cone state to OUT (.npz) and prints {"seconds", "threads"}."""
    name, ncones, out = spec.split(":", 2)
    import numpy as np
    import oracle
    w = workload(name)
    n = min(int(ncones), w.n_axons)
    used = oracle.set_threads(os.cpu_count() or 1)
    g = oracle.Grid(w.dim, w.nx, w.ny, w.nz if w.dim == 3 else 1, h=w.h, D=w.D, lam=w.lam, dt=w.dt)
    c = oracle.Cone(w.w_prev, w.w_grad, w.w_noise, w.step_len, w.stop_radius, w.grad_eps, w.wall_mode, w.seed)
    t0 = time.perf_counter()
    C, pos, dirs, act = oracle.run(g, c, w.field0().astype(np.float64), 0, w.nsteps, w.src_cell, w.src_emit,
                                   w.src_map, w.pos[:, :n], w.dir[:, :n], w.active[:n])
    secs = time.perf_counter() - t0
    np.savez(out, C=C, pos=pos, act=act)
    print(json.dumps({"seconds": secs, "threads": used, "cones": n}), flush=True)
    return 0


def whole_run_report(name, gpu, ncones):
    """FP32 GPU run against the FP64 oracle after the workload's full run: the field error (the
    field does not depend on the cones), and the cones' endpoint distributions (displacement
    from the start) -- quantiles and a two-sample Kolmogorov-Smirnov test -- plus how many of the
    same cones end within 1e-3 of the oracle's endpoint.  Whole-run trajectories are chaotic in
    rounding, so the endpoint figures are a report, not a pass criterion."""
    import numpy as np
    w = workload(name)
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "orc.npz")
        t0 = time.perf_counter()
        try:
            r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-whole-run",
                                f"{name}:{ncones}:{out}"], capture_output=True, text=True, timeout=1200)
            meta = json.loads(r.stdout.strip().splitlines()[-1])
            ref = dict(np.load(out))
        except Exception as e:
            return {"unavailable": f"oracle whole run failed: {type(e).__name__}"}
        wall = time.perf_counter() - t0
    n = meta["cones"]
    Cg, Cr = gpu["C"].astype(np.float64), ref["C"]
    scale = np.abs(Cr).max()
    rel = np.abs(Cg - Cr) / np.maximum(np.abs(Cr), 1e-6 * scale)
    p0 = w.pos[:, :n].astype(np.float64)
    dg = np.linalg.norm(gpu["pos"][:, :n].astype(np.float64) - p0, axis=0)
    dr = np.linalg.norm(ref["pos"] - p0, axis=0)
    gap = np.linalg.norm(gpu["pos"][:, :n].astype(np.float64) - ref["pos"], axis=0)
    q = [0.1, 0.5, 0.9]
    try:
        from scipy.stats import ks_2samp
        ks = ks_2samp(dg, dr)
        ks_rec = {"statistic": float(ks.statistic), "pvalue": float(ks.pvalue)}
    except Exception as e:
        ks_rec = {"unavailable": type(e).__name__}
    return {"workload": describe(w)["workload"],
            "field": {"max_rel_err": float(rel.max()),
                      "rel_l2_err": float(np.linalg.norm(Cg - Cr) / max(np.linalg.norm(Cr), 1e-300)),
                      "denominator": "max(|C64|, 1e-6 max|C64|)"},
            "endpoints": {"cones": n, "of": w.n_axons,
                          "displacement_quantiles_gpu": [float(x) for x in np.quantile(dg, q)],
                          "displacement_quantiles_oracle": [float(x) for x in np.quantile(dr, q)],
                          "quantiles": q, "ks_2samp": ks_rec,
                          "same_endpoint_within_1e-3": float((gap <= 1e-3).mean()),
                          "median_endpoint_gap": float(np.median(gap)),
                          "stopped_gpu": float(1 - gpu["act"][:n].mean()),
                          "stopped_oracle": float(1 - ref["act"].mean())},
            "oracle": {"seconds": meta["seconds"], "threads": meta["threads"], "wall_s": wall,
                       "kind": "FP64 oracle, field rows over every host core, the first cones"}}


# ------------------------------------------------------------------ connectivity
GRAPH_METRIC = "cue connectivity pipeline: cones/s (bin neurons + connect cones + adjacency list + BFS)"
GRAPH_UNIT = "cones/s"
GRAPH_LAUNCHES = 7 + 1 + 10 + 1        # kernels per pipeline: binning, connections, adjacency list, BFS


def graph_describe(gw):
    return {"workload": f"connectivity: {gw.n_neurons} neurons uniform on 2048x2048, {gw.n_cones} cones "
                        f"grown up to 48 from them (95% active), radius {gw.radius}, "
                        f"{gw.grid[0]}x{gw.grid[1]} cells",
            "neurons": gw.n_neurons, "cones": gw.n_cones, "radius": gw.radius, "cell": gw.cell,
            "grid": list(gw.grid)}


def graph_oracle_sample(gw, budget_s):
    """The FP64 oracle's connectivity on the first S cones (S sized to the budget): binning of
    every neuron, the brute-force pair test of the S cones, the adjacency list, BFS.
    Returns (S, seconds, pairs)."""
    import oracle
    probe = 256
    t0 = time.perf_counter()
    oracle.connect(gw.pos[:, :probe], gw.owner[:probe], gw.active[:probe], gw.npos, gw.radius, cap=1 << 16)
    per_cone = (time.perf_counter() - t0) / probe
    S = int(max(probe, min(gw.n_cones, budget_s / max(per_cone, 1e-9))))
    t0 = time.perf_counter()
    oracle.bin_points(gw.npos, gw.cell, gw.grid)
    src, dst = oracle.connect(gw.pos[:, :S], gw.owner[:S], gw.active[:S], gw.npos, gw.radius, cap=8 * S + 1024)
    row, col = oracle.csr(gw.n_neurons, src, dst)
    oracle.bfs(row, col, gw.source)
    return S, time.perf_counter() - t0, int(src.size)


def run_reference_graph(args):
    from paper_1405_3331_gb300 import workloads as W
    gw = W.config_graph()
    budget = 120.0 / max(1, args.steps + args.warmup)
    S, secs, pairs = graph_oracle_sample(gw, budget)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        graph_oracle_sample(gw, budget)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = S * args.steps / total
    sample = (f"first {S} of {gw.n_cones} cones per step (all {gw.n_neurons} neurons binned; pair test "
              f"against every neuron; adjacency list and BFS of their edges), FP64")
    line = {
        "impl": "reference", "metric": GRAPH_METRIC, "value": value, "unit": GRAPH_UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": graph_describe(gw),
        "cpu_baseline": {"value": value, "unit": GRAPH_UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                         "host_cores": os.cpu_count(), "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": GRAPH_UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main_graph(args, torch, dev, rank, world, dist, barrier):
    """The connectivity stage (cue_graph.h) as one step: bin the neurons, connect the cones to
    them, build the adjacency list of the connection graph, BFS from neuron 0; every call on one
    stream with preallocated workspaces, each stage bracketed by CUDA events."""
    import ctypes as ct

    import numpy as np

    from paper_1405_3331_gb300 import cue
    from paper_1405_3331_gb300 import graph as G
    from paper_1405_3331_gb300 import workloads as W
    gw = W.config_graph(seed=7 + 100 * rank)
    L = G._lib()
    m, n = gw.n_neurons, gw.n_cones
    ncell = gw.grid[0] * gw.grid[1]
    cap = 4 * n                                     # ~0.8 connections per cone expected
    t = lambda a, dt: torch.as_tensor(a, dtype=dt).to(dev)
    npos, pos = t(gw.npos, torch.float32), t(gw.pos, torch.float32)
    owner, active = t(gw.owner, torch.int32), t(gw.active, torch.uint8)
    i32 = lambda k: torch.empty(k, dtype=torch.int32, device=dev)
    cell_of, sid, start, end = i32(m), i32(m), i32(ncell), i32(ncell)
    src, dst, cnt = i32(cap), i32(cap), i32(1)
    row, col, medges, level = i32(m + 1), i32(cap), i32(1), i32(m)
    nb_bin, nb_csr, nb_bfs = (int(L.cue_bin_workspace_bytes(m, ncell)), int(L.cue_csr_workspace_bytes(m, cap)),
                              int(L.cue_bfs_workspace_bytes(m)))
    ws = [torch.empty(nb + 256, dtype=torch.uint8, device=dev) for nb in (nb_bin, nb_csr, nb_bfs)]
    wp = [(b.data_ptr() + 255) & ~255 for b in ws]
    grid3 = (ct.c_int32 * 3)(gw.grid[0], gw.grid[1], 1)
    stream = torch.cuda.Stream(dev)
    st = stream.cuda_stream
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def stages(ev=None):
        calls = [
            lambda: L.cue_bin_points(2, m, npos.data_ptr(), gw.cell, grid3, cell_of.data_ptr(), sid.data_ptr(),
                                     start.data_ptr(), end.data_ptr(), wp[0], nb_bin, st),
            lambda: L.cue_connect(2, n, pos.data_ptr(), owner.data_ptr(), active.data_ptr(), m, npos.data_ptr(),
                                  gw.radius, gw.cell, grid3, sid.data_ptr(), start.data_ptr(), end.data_ptr(), cap,
                                  src.data_ptr(), dst.data_ptr(), cnt.data_ptr(), st),
            lambda: L.cue_csr_build(m, cap, cnt.data_ptr(), src.data_ptr(), dst.data_ptr(), row.data_ptr(),
                                    col.data_ptr(), medges.data_ptr(), wp[1], nb_csr, st),
            lambda: L.cue_bfs(m, row.data_ptr(), col.data_ptr(), gw.source, level.data_ptr(), wp[2], nb_bfs, st),
        ]
        for i, f in enumerate(calls):
            if ev is not None:
                ev[i].record(stream)
            cue._check(f(), ("cue_bin_points", "cue_connect", "cue_csr_build", "cue_bfs")[i])
        if ev is not None:
            ev[4].record(stream)

    for _ in range(max(args.warmup, 3)):
        stages()
    cue._check(L.cue_graph_status(wp[2], st), "cue_graph_status")
    pairs, edges = int(cnt.item()), int(medges.item())
    if pairs > cap:
        raise RuntimeError(f"{pairs} connections exceed the preallocated {cap}")
    lv = level.cpu().numpy()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    sampler = ClockSampler(gpu_id_for(dev.index or 0))
    barrier()
    sampler.start()
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        stages(evs[k])
    barrier()
    clocks = sampler.stop()
    cue._check(L.cue_graph_status(wp[2], st), "cue_graph_status")
    stage_ms = [sum(e[i].elapsed_time(e[i + 1]) for e in evs) / args.steps for i in range(4)]
    local_ms = sum(e[0].elapsed_time(e[4]) for e in evs)
    total_ms, value = aggregate(local_ms, n, args.steps, world, dist, dev)
    hbm, peak_kind = peaks()
    # compulsory bytes of each stage: every input read once, every output written once
    alg = [16 * m + 8 * ncell,                                    # neurons in; cell, order, cell ranges out
           13 * n + 8 * ncell + 12 * m + 8 * pairs,               # cones + the binned neurons in; pairs out
           8 * pairs + 4 * (m + 1) + 4 * edges,                   # pairs in; adjacency list out
           4 * (m + 1) + 4 * edges + 4 * m]                       # adjacency list in; levels out
    names = ["bin_points", "connect", "csr_build", "bfs"]
    top = max(range(4), key=lambda i: stage_ms[i])
    achieved = alg[top] / (stage_ms[top] / 1e3) / 1e9
    line = {
        "metric": GRAPH_METRIC, "value": value, "unit": GRAPH_UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 positions, f64 distances, int32 graph", "data": "synthetic",
        "config": dict(graph_describe(gw), l2="flushed between timed steps (512 MiB write)",
                       parallelism=f"replicas x{world}" if world > 1 else "single GPU"),
        "stages_ms": dict(zip(names, stage_ms)),
        "connections": pairs, "edges": edges, "bfs_reached": int((lv >= 0).sum()), "bfs_levels": int(lv.max()) + 1,
        "bfs_edges_per_s": edges / (stage_ms[3] / 1e3),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": None, "kernel": names[top], "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": alg[top], "avg_launch_us": stage_ms[top] * 1e3,
                     "note": "compulsory bytes of the slowest stage; the working set (about 60 MB) stays in L2 "
                             "and the stages are latency-bound (atomics, scans, a barrier per BFS level)"},
        "clocks": clocks, "gpu_launches": GRAPH_LAUNCHES * args.steps,
    }
    if not args.no_e2e:
        host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
                for a in (gw.npos, gw.pos, gw.owner, gw.active)]
        lv_host = torch.empty(m, dtype=torch.int32).pin_memory()
        reps = max(1, min(args.steps, 3))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tot = 0.0
        for _ in range(reps):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0.record(stream)
            with torch.cuda.stream(stream):
                for d, h in zip((npos, pos, owner, active), host):
                    d.copy_(h, non_blocking=True)
            stages()
            with torch.cuda.stream(stream):
                lv_host.copy_(level, non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        line["e2e"] = {"value": world * n * reps / (tot / 1e3), "unit": GRAPH_UNIT,
                       "h2d_bytes_per_step": sum(h.numel() * h.element_size() for h in host),
                       "d2h_bytes_per_step": m * 4, "ms_per_step": tot / reps}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        S, secs, _ = graph_oracle_sample(gw, args.cpu_seconds)
        line["cpu_baseline"] = {
            "value": S / secs, "unit": GRAPH_UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {S} of {n} cones (all {m} neurons binned; pair test against every neuron; "
                      f"adjacency list and BFS of their edges), FP64, one thread",
            "seconds": secs, "host_cores": os.cpu_count(), "cpu_model": cpu_model()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def sim_path_used(sim):
    from paper_1405_3331_gb300 import cue
    return {cue.CUE_PATH_FUSED: "fused", cue.CUE_PATH_PERSIST: "persist", cue.CUE_PATH_RESIDENT: "resident",
            cue.CUE_PATH_CLUSTER: "cluster"}.get(sim.last_path(), "plain")


def hbm_probe(cue, torch, dev, hbm, dim=2):
    """The unblocked field step (field + sources, no cones) on a grid that cannot stay in L2:
    2D 8192^2 (plain float4 kernel) or 3D 512^3 (the TMA step kernel)."""
    from paper_1405_3331_gb300 import workloads as W
    w = W.hbm_probe_2d() if dim == 2 else W.hbm_probe_3d()
    sim = cue.Simulation(w, device=dev, path=cue.CUE_PATH_PLAIN)
    sim.cue_step(5)
    sim.set_option(cue.CUE_OPT_TIME_KERNEL, 1)
    sim.kernel_time()
    n = 20
    sim.cue_step(n)
    ms, k = sim.kernel_time()
    sim.check()
    sim.close()
    gbs = 8 * w.n_cells * k / (ms / 1e3) / 1e9
    what = ("2D 8192x8192 field only (256 MiB per buffer), plain field kernel" if dim == 2 else
            "3D 512x512x512 field only (512 MiB per buffer), TMA step kernel")
    return {"workload": what,
            "cell_updates_per_s": w.n_cells * k / (ms / 1e3), "achieved_gbs": gbs, "peak_gbs": hbm,
            "frac": gbs / hbm, "launches": k, "avg_launch_us": ms / k * 1e3}


if __name__ == "__main__":
    sys.exit(main())
