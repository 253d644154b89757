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
    ap.add_argument("--workload", default="c2", choices=["c1", "c2", "c3", "c4", "c5", "graph"])
    ap.add_argument("--path", default="auto", choices=["auto", "plain", "fused", "persist", "resident"])
    ap.add_argument("--depth", type=int, default=0, help="temporal depth on the fused path (0 = auto)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-probe", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="CPU-baseline sample budget")
    ap.add_argument("--run-steps", type=int, default=0,
                    help="time steps per benchmark step (0 = the workload's own count); for profiling")
    # internal: time the oracle with its field rows over threads, in a process of its own
    # (no CUDA context, no second OpenMP runtime next to PyTorch's): WORKLOAD:NSTEPS:THREADS
    ap.add_argument("--oracle-threads-sample", default="", help=argparse.SUPPRESS)
    return ap.parse_args()


def workload(name, rank=0):
    from paper_1405_3331_gb300 import workloads as W
    if name == "c1":
        return W.config_c1(seed=0 + 100 * rank)
    if name == "c2":
        return W.config_c2(seed=1 + 100 * rank)
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
def main():
    args = parse_args()
    if args.oracle_threads_sample:
        return oracle_threads_child(args.oracle_threads_sample)
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
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
    path = {"auto": cue.CUE_PATH_AUTO, "plain": cue.CUE_PATH_PLAIN, "fused": cue.CUE_PATH_FUSED,
            "persist": cue.CUE_PATH_PERSIST, "resident": cue.CUE_PATH_RESIDENT}[args.path]
    sim = cue.Simulation(w, device=dev, path=path)
    if args.depth:
        sim.set_option(cue.CUE_OPT_TEMPORAL_DEPTH, args.depth)
    stream = sim.stream
    C0 = sim.fields[0].clone()
    pos0, dir0, act0 = sim.pos.clone(), sim.dir.clone(), sim.active.clone()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def reset():
        with torch.cuda.stream(stream):
            sim.fields[0].copy_(C0)
            sim.pos.copy_(pos0)
            sim.dir.copy_(dir0)
            sim.active.copy_(act0)
        cue._check(cue.cue_set_state(sim.h, 0, 0, 0), "cue_set_state")

    # warm-up (also counts the cone updates of one run: every run is identical)
    for i in range(max(args.warmup, 3)):
        reset()
        if i == max(args.warmup, 3) - 1:
            sim.cone_updates()
        sim.sim_run(w.nsteps)
    sim.check()
    cone_updates_per_run = sim.cone_updates()

    # timed region
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    sampler = ClockSampler(gpu_id_for(local))
    # events around every 16th launch of the dominant kernel (every launch on the persistent
    # and resident paths, where one launch is a whole run)
    sim.set_option(cue.CUE_OPT_TIME_KERNEL, 1 if sim_path_used(sim) in ("persist", "resident") else 16)
    sim.kernel_time()
    barrier()
    sampler.start()
    launches0 = sim.launches()
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        reset()
        evs[k][0].record(stream)
        sim.sim_run(w.nsteps)
        evs[k][1].record(stream)
    barrier()
    clocks = sampler.stop()
    launches = sim.launches() - launches0
    kern_ms, kern_n = sim.kernel_time()
    sim.set_option(cue.CUE_OPT_TIME_KERNEL, 0)
    sim.check()
    local_ms = sum(a.elapsed_time(b) for a, b in evs)
    cells_per_run = w.n_cells * w.nsteps
    total_ms, value = aggregate(local_ms, cells_per_run, args.steps, world, dist, dev)
    axon_steps = world * cone_updates_per_run * args.steps / (total_ms / 1e3)

    # roofline of the dominant kernel
    hbm, peak_kind = peaks()
    fused = kern_n > 0 and sim_path_used(sim) == "fused"
    bytes_per_cell = 12 if w.src_map is not None else 8
    if kern_n:
        steps_per_launch = (w.nsteps / (launches_per_run(sim, w)))
        # compulsory field traffic of one launch: the fused kernel reads and writes the field once
        # for its K steps; the plain kernel once per step; the persistent and resident kernels
        # once per step of the whole run they cover
        per_launch_passes = steps_per_launch if sim_path_used(sim) in ("persist", "resident") else 1
        alg_bytes = bytes_per_cell * w.n_cells * per_launch_passes
        if w.dim == 3 and sim_path_used(sim) == "plain":
            # the 3D step launch also moves the cones: position and direction read and
            # written, the active flag read (the sampled field nodes are counted in the field)
            alg_bytes += w.n_axons * (4 * w.dim * 4 + 1)
        avg_s = kern_ms / kern_n / 1e3
        achieved = alg_bytes / avg_s / 1e9
    else:
        steps_per_launch, alg_bytes, avg_s, achieved = 0, 0, 0, 0.0
    kname = {"fused": "fused", "persist": "persist", "resident": "resident"}.get(sim_path_used(sim), "field")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm if hbm else None,
                "traffic": recorded_traffic(kname, args.workload),
                "kernel": kname, "peak_kind": peak_kind, "launches": kern_n,
                "avg_launch_us": avg_s * 1e6, "steps_per_launch": steps_per_launch,
                "algorithmic_bytes_per_launch": alg_bytes,
                "effective_gbs": bytes_per_cell * w.n_cells * steps_per_launch / avg_s / 1e9 if avg_s else 0}
    # a temporally blocked launch moves its field through HBM once for K steps: the bytes an
    # unblocked kernel would move for the same node updates, against the same peak
    roofline["effective_frac"] = roofline["effective_gbs"] / hbm if hbm else None
    if kname == "resident":
        roofline["note"] = ("one block holds the grid in shared memory for the whole run: HBM is read "
                            "and written once per launch, and a step is bound by one SM's shared-memory "
                            "and issue rate; achieved counts 8 B per node update as for the other kernels")

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(describe(w), parallelism=f"replicas x{world}" if world > 1 else "single GPU",
                       path=sim_path_used(sim)),
        "axon_steps_per_s": axon_steps, "cone_updates_per_run": cone_updates_per_run,
        "roofline": roofline, "clocks": clocks, "gpu_launches": launches,
    }

    # end to end through the public API from pinned host buffers
    if not args.no_e2e:
        Ch = w.field0()
        host = [torch.from_numpy(a).pin_memory() for a in (Ch, w.pos, w.dir, w.active)]
        out = tuple(torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in host)
        sim.run_host(*host, w.nsteps, out=out)     # warm
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = max(1, min(args.steps, 3))
        barrier()
        tot = 0.0
        for _ in range(reps):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0.record(stream)
            sim.run_host(*host, w.nsteps, out=out)
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        h2d = sum(t.numel() * t.element_size() for t in host)
        d2h = sum(t.numel() * t.element_size() for t in out)
        line["e2e"] = {"value": world * cells_per_run * reps / (tot / 1e3), "unit": UNIT,
                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                       "ms_per_step": tot / reps}

    # adjoint workload: gradients of the endpoint loss against the forward run's own time
    if w.targets is not None and w.wall_mode == 1 and rank == 0:
        line["adjoint"] = adjoint_timing(cue, torch, sim, w, reset, stream, flush, total_ms / args.steps)

    # HBM probe: plain field kernel on 2D 8192^2 (256 MiB per buffer), never L2-resident
    if not args.no_probe and rank == 0:
        line["hbm_probe"] = hbm_probe(cue, torch, dev, hbm)
        if w.dim == 3:
            line["hbm_probe_3d"] = hbm_probe(cue, torch, dev, hbm, dim=3)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        nsteps, secs = oracle_sample(w, args.cpu_seconds)
        sample = f"first {nsteps} of {w.nsteps} time steps of the same workload (FP64)"
        line["cpu_baseline"] = {
            "value": w.n_cells * nsteps / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": sample + ", one thread", "seconds": secs, "host_cores": os.cpu_count(),
            "cpu_model": cpu_model()}
        line["cpu_baseline_threads"] = oracle_threads_sample(args.workload, w.n_cells, nsteps, sample)
    sim.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main_batch(args, torch, cue, dev, rank, world, dist, barrier):
    """512 independent 2D instances of uneven sizes and physics, 1,000 coupled steps, in one
    persistent launch replayed from a captured CUDA graph, launch shape chosen by the autotuner.
    One benchmark step = the whole batch from its initial state."""
    from paper_1405_3331_gb300 import batch as B
    from paper_1405_3331_gb300 import workloads as W
    ws = W.config_c4(seed=3 + 100 * rank)
    T = args.run_steps or ws[0].nsteps
    cells = sum(w.n_cells for w in ws)
    b = B.Batch(ws, device=dev)
    stream = b.stream
    init = [(b.fields[i][0].clone(), b.pos[i].clone(), b.dir[i].clone(), b.active[i].clone())
            for i in range(len(ws))]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def reset():
        with torch.cuda.stream(stream):
            for i, (C, p, d, a) in enumerate(init):
                b.fields[i][0].copy_(C)
                b.pos[i].copy_(p)
                b.dir[i].copy_(d)
                b.active[i].copy_(a)
        b.reset_state(0, 0)

    rows, bpsm, tuned_ms = b.autotune(10)
    mode = b.get_option(B.CUE_BOPT_MODE)
    b.set_option(B.CUE_BOPT_GRAPH, 1)
    for _ in range(max(args.warmup, 3)):
        reset()
        b.run(T)
    b.check()
    b.cone_updates()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(gpu_id_for(dev.index or 0))
    barrier()
    sampler.start()
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        reset()
        evs[k][0].record(stream)
        b.run(T)
        evs[k][1].record(stream)
    barrier()
    clocks = sampler.stop()
    b.check()
    cone_updates = b.cone_updates() / args.steps
    local_ms = sum(x.elapsed_time(y) for x, y in evs)
    total_ms, value = aggregate(local_ms, cells * T, args.steps, world, dist, dev)
    hbm, peak_kind = peaks()
    per_launch_s = total_ms / args.steps / 1e3
    achieved = 8.0 * cells * T / per_launch_s / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batched: {len(ws)} independent 2D instances (sides U{{64..1024}}, "
                               f"{cells / 1e6:.1f} M cells, {sum(w.n_axons for w in ws)} cones), {T} steps",
                   "instances": len(ws), "cells": cells, "steps_per_run": T,
                   "launch": ("one persistent launch per run" if mode == 1 else
                              ("per time step one launch over every instance's cone chunks and streamed field "
                               "tiles" if rows > 4 else
                               "per time step one launch over the cone chunks and one over the field tiles"))
                             + ", replayed from a CUDA graph",
                   "autotuned": {"rows": rows, "blocks_per_sm": bpsm, "probe_ms_per_step": tuned_ms},
                   "l2": "flushed between timed steps (512 MiB write); 1.2 GB working set",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "axon_steps_per_s": world * cone_updates * args.steps / (total_ms / 1e3),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": recorded_traffic("persist" if mode == 1 else "step", "c4"),
                     "kernel": "persist" if mode == 1 else "step launches (per run)", "peak_kind": peak_kind,
                     "launches": args.steps, "avg_launch_us": per_launch_s * 1e6, "steps_per_launch": T,
                     "algorithmic_bytes_per_launch": 8.0 * cells * T},
        # persistent: the kernel + the step advance; per step: one launch per time step (streamed tiles
        # with the cone chunks) or two (cone chunks, then tiles), + the advance
        "clocks": clocks,
        "gpu_launches": args.steps * (2 if mode == 1 else (T if rows > 4 else 2 * T) + 1),
    }
    # the one-instance-per-launch plain solver on the first 32 instances (100 steps each), and
    # the same instances one after another through sim_run on the library's own path choice
    # every instance, 100 steps each (a rate, so the batch's 1,000-step runs compare directly); each
    # Simulation has its own stream, so instances may overlap on the GPU: a conservative baseline
    sub = ws
    sub_cells = sum(w.n_cells for w in sub)
    Tb = 100

    def sequential_rate(path):
        sims = [cue.Simulation(w, device=dev, path=path) for w in sub]
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
        return sub_cells * Tb / dt

    plain_rate = sequential_rate(cue.CUE_PATH_PLAIN)
    auto_rate = sequential_rate(cue.CUE_PATH_AUTO)
    line["baseline_sequential_sim_run"] = {
        "value": auto_rate, "unit": UNIT, "speedup": value / world / auto_rate,
        "sample": f"all {len(sub)} instances x {Tb} steps, one sim_run per instance in turn (resident, "
                  "persistent or fused path as the library picks)"}
    line["baseline_plain_per_instance"] = {
        "value": plain_rate, "unit": UNIT, "speedup": value / world / plain_rate,
        "sample": f"all {len(sub)} instances x {Tb} steps, each instance its own cone and field launches per step"}
    if not args.no_e2e:
        # end to end: every instance's state from pinned host memory, the run, the fields back
        host = [tuple(t.cpu().pin_memory() for t in st) for st in init]
        outs = [torch.empty_like(h[0]).pin_memory() for h in host]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        with torch.cuda.stream(stream):
            for i, (C, p, d, a) in enumerate(host):
                b.fields[i][0].copy_(C, non_blocking=True)
                b.pos[i].copy_(p, non_blocking=True)
                b.dir[i].copy_(d, non_blocking=True)
                b.active[i].copy_(a, non_blocking=True)
        b.reset_state()
        b.run(T)
        cur = b.get_option(B.CUE_BINFO_CUR)
        with torch.cuda.stream(stream):
            for i in range(len(ws)):
                outs[i].copy_(b.fields[i][cur], non_blocking=True)
        e1.record(stream)
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


def adjoint_timing(cue, torch, sim, w, reset, stream, flush, forward_ms):
    """Time sim_adjoint (forward with checkpoints every 64 steps, recompute, adjoint) on the
    same workload; the ratio divides by the timed forward run."""
    k = 64
    reset()
    sim.adjoint(w.targets, w.nsteps, k)          # warm
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        flush.zero_()
    reset()
    e0.record(stream)
    g = sim.adjoint(w.targets, w.nsteps, k)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    # the plain forward solver (one cone and one field launch per step) on the same workload
    plain = cue.Simulation(w, device=sim.device, path=cue.CUE_PATH_PLAIN)
    plain.sim_run(w.nsteps)
    torch.cuda.synchronize()
    plain.load(C=w.field0(), pos=w.pos, dir=w.dir, active=w.active, step=0)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(plain.stream)
    plain.sim_run(w.nsteps)
    p1.record(plain.stream)
    p1.synchronize()
    plain_ms = p0.elapsed_time(p1)
    plain.check()
    plain.close()
    return {"ms_per_run": ms, "forward_ms_per_run": forward_ms, "ratio_to_forward": ms / forward_ms,
            "plain_forward_ms_per_run": plain_ms, "ratio_to_plain_forward": ms / plain_ms,
            "ckpt_every": k, "loss": float(g["loss"]), "dL_dD": float(g["dD"]),
            "dL_dlambda": float(g["dlambda"]), "dL_de_max": float(g["dsrc"].abs().max()),
            "dL_dM_max": float(g["dmap"].abs().max())}


def launches_per_run(sim, w):
    """Launches of the dominant kernel in one run (K steps per launch on the fused path, the
    whole run per launch on the persistent and resident paths)."""
    from paper_1405_3331_gb300 import cue
    if sim.fused_active():
        K = sim.get_option(cue.CUE_INFO_DEPTH)
        return (w.nsteps + K - 1) // K
    if sim_path_used(sim) in ("persist", "resident"):
        return 1
    return w.nsteps


def sim_path_used(sim):
    from paper_1405_3331_gb300 import cue
    return {cue.CUE_PATH_FUSED: "fused", cue.CUE_PATH_PERSIST: "persist",
            cue.CUE_PATH_RESIDENT: "resident"}.get(sim.last_path(), "plain")


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
