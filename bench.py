"""Benchmark of the boosted-frame PIC step (one JSON line on rank 0).

Workload: the 2D boosted-frame 0.1 GeV-class stage, 4096 (z) x 256 (x) cells,
n0 = 1e19 cm^-3, 16 particles per cell, gamma_boost = 13, CK solver, 16-cell
PML, Friedman theta = 0.1, 4 bilinear passes + compensation, cubic shapes,
FP32 fields/momenta with FP64 positions (mixed precision). The box is full of
plasma that keeps streaming in through the +z plane. A step is one full PIC
step (Faraday/Friedman/PML, gather-field filter, gather/push/deposit,
antenna, ion current, current filter + Ampere/PML, inflow, periodic sort).

value: electron particle-steps per second of the whole job (all ranks),
device-timed with CUDA events over exactly K steps after W warm-up steps.
e2e: the same metric through the public API with host-side wall clock, each
step followed by a device->host read of the step's diagnostics (pic_get_stats),
including context creation and plasma loading.
The particle arrays (~0.9 GB) exceed the 129 MB L2, so no L2 flush is needed.

--impl reference times the FP64 CPU oracle (the plain restatement of the
method used by the tests) on the host cores, on a bounded sample of the same
workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# algorithmic bytes per electron particle-step of the push kernel (mixed): read x,z (2x8),
# u (3x4), w (4); write x,z (2x8), u (3x4)
BYTES_PER_PARTICLE = {"mixed": 60, "fp64": 88}
# 3D: read and write x, y, z (3 x 8), u (3 x 4 or 3 x 8), read w
BYTES_PER_PARTICLE_3D = {"mixed": 76, "fp64": 104}
# algorithmic bytes per cell-step of the field kernels (mixed, with Friedman): see the design notes
BYTES_PER_CELL = {"mixed": 168, "fp64": 336}
# measured DRAM bytes (read + write) per particle of one push launch (k_push), mixed precision, cubic shapes,
# the Yee-located gather, for every layout the autotuner can return, keyed by (tile_x, tile_z, sort_every):
# ncu dram__bytes_read.sum + dram__bytes_write.sum on the 2048 x 256 stage box (bench.py --layout-sweep, the
# 2nd and 3rd push of each layout), scaled to the full box by its particle count. Below the 56 bytes of stored
# state: the last writes of a launch are still in the 129 MB L2 when it ends.
TRAFFIC_BYTES_PER_PARTICLE = {
    (8, 8, 8): 49.71, (8, 8, 16): 49.61, (8, 8, 32): 49.58, (8, 8, 64): 49.49, (8, 8, 128): 49.62, (8, 16, 8): 49.58,
    (8, 16, 16): 49.63, (8, 16, 32): 49.61, (8, 16, 64): 49.49, (8, 16, 128): 49.63, (8, 32, 8): 49.83,
    (8, 32, 16): 49.81, (8, 32, 32): 49.78, (8, 32, 64): 49.71, (8, 32, 128): 49.74, (16, 8, 8): 49.64,
    (16, 8, 16): 49.6, (16, 8, 32): 49.74, (16, 8, 64): 49.58, (16, 8, 128): 49.72, (16, 16, 8): 49.79,
    (16, 16, 16): 49.73, (16, 16, 32): 49.78, (16, 16, 64): 49.69, (16, 16, 128): 49.68, (16, 32, 8): 49.07,
    (16, 32, 16): 49.13, (16, 32, 32): 49.08, (16, 32, 64): 48.96, (16, 32, 128): 49.09, (32, 8, 8): 49.53,
    (32, 8, 16): 49.53, (32, 8, 32): 49.54, (32, 8, 64): 49.52, (32, 8, 128): 49.47, (32, 16, 8): 49.05,
    (32, 16, 16): 49.3, (32, 16, 32): 49.07, (32, 16, 64): 49.05, (32, 16, 128): 49.2, (32, 32, 8): 48.87,
    (32, 32, 16): 48.85, (32, 32, 32): 48.84, (32, 32, 64): 48.94, (32, 32, 128): 48.95,
}
# the push's instruction and FP32 arithmetic counts per particle (mixed, cubic, Yee-located gather; ncu
# smsp__inst_executed.sum and smsp__sass_thread_inst_executed_op_{fadd,fmul,ffma}_pred_on.sum of three pushes
# at steps 5-7 of the 2048 x 256 stage box, 8 x 16-cell tiles, sort every 64): warp instructions, and FLOPs
# counted as FADD + FMUL + 2 FFMA (the packed two-lane FMAs of the gather are not in these counters). The
# warp instructions were 20.7 there before each thread's next particle was copied into shared memory ahead
# of its push; that copy adds 1.6% (22.29 -> 22.64 warp instructions per particle in the full captures at
# step 76), hence 21.0. The arithmetic is unchanged.
PUSH_WARP_INST_PER_PARTICLE = 21.0
PUSH_FLOPS_PER_PARTICLE = 174.0
# 3D: ncu dram bytes of k3_push_tiles on the 256 x 128 x 128 box (189.5 MB for 2,356,608 electrons), scaled
# to the full box by its particle count
TRAFFIC_BYTES_PER_PARTICLE_3D = {("mixed", 3): 80.4}


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(p))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(v: float, ws: int) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(v: float, ws: int) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(units: float, ms: float, ws: int) -> tuple:
    """Whole-job throughput of independent replicas (weak scaling): the units all ranks processed
    divided by the slowest rank's time. Returns (units/s, max ms)."""
    ms_max = max_over_ranks(ms, ws)
    return sum_over_ranks(units, ws) / (ms_max * 1e-3), ms_max


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ----------------------------------------------------------------------------
# The CPU baseline: the FP64 oracle as it stands (single-threaded C), on a slice of the workload: all of
# its transverse cells and particles per cell, ORACLE_ROWS cells along z. On all host cores it runs as one
# independent copy per core (spawned processes), the oracle itself unchanged.
ORACLE_ROWS = 256
ORACLE_ROWS_3D = 128


def host_cpu() -> dict:
    """the host's core count and CPU model (lscpu, else /proc/cpuinfo)"""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu model")):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"nproc": os.cpu_count(), "model": model}


def oracle_slice(w: dict, three: bool, rows: int = 0) -> dict:
    from paper_1009_2727_gb300 import workloads as W
    if three:
        ws = W.shrink3(w, 64, 64, rows or ORACLE_ROWS_3D)
    else:
        ws = W.shrink(w, w["nx"], rows or ORACLE_ROWS)
    ws["precision"] = "fp64"
    return ws


def _oracle_worker(job):
    """one oracle copy (run in its own spawned process, or inline): warm-up steps untimed, then timed steps
    until `steps` are done or `seconds` have passed; returns (particles, timed steps, seconds)"""
    ws, three, warmup, steps, seconds = job
    import oracle
    s = oracle.Sim3(ws) if three else oracle.Sim(ws)
    if warmup > 0:
        s.step(warmup)
    n = len(s.particles(0)["x"])
    k = 0
    t0 = time.perf_counter()
    while k < steps and (time.perf_counter() - t0) < seconds:
        s.step(1)
        k += 1
    return n, k, time.perf_counter() - t0


def oracle_throughput(ws: dict, three: bool, procs: int, warmup: int, steps: int, seconds: float) -> dict:
    """particle-steps/s of `procs` copies of the oracle side by side (1: inline, single thread)"""
    import oracle
    oracle.build()
    job = (ws, three, warmup, steps, seconds)
    if procs <= 1:
        res = [_oracle_worker(job)]
    else:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(procs) as pool:
            res = pool.map(_oracle_worker, [job] * procs)
    tot = sum(n * k for n, k, _ in res)
    wall = max(dt for _, _, dt in res)
    return {"value": tot / wall, "particles": res[0][0], "steps": min(k for _, k, _ in res), "seconds": wall,
            "copies": len(res)}


def cpu_baseline_line(w: dict, three: bool, seconds: float = 8.0) -> dict:
    """the oracle on the workload's slice: one thread, then one copy per host core"""
    ws = oracle_slice(w, three)
    cpu = host_cpu()
    one = oracle_throughput(ws, three, 1, 1, 40, seconds)
    allc = oracle_throughput(ws, three, cpu["nproc"] or 1, 1, 40, seconds)
    box = f"{ws['nz']} x {ws['ny']} x {ws['nx']}" if three else f"{ws['nz']} x {ws['nx']}"
    return {"value": allc["value"], "unit": "particle-steps/s", "cores": allc["copies"], "kind": "oracle",
            "single_thread": one["value"], "cpu": cpu,
            "sample": (f"{w['name']} on a {box}-cell slice ({one['particles']} electrons + as many ions): "
                       f"{allc['copies']} independent copies of the single-threaded oracle, one per host core, "
                       f"{allc['steps']}+ steps in {allc['seconds']:.1f} s; one copy alone {one['steps']} steps in "
                       f"{one['seconds']:.1f} s")}


REF_BUDGET_S = 150.0      # wall-clock bound of the reference arm's steps


def run_reference(args, w):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    three = w.get("dim", 2) == 3
    cpu = host_cpu()
    procs = cpu["nproc"] or 1
    # the sample: the same slice as the main arm's cpu_baseline, shortened when one step projects the
    # whole --steps/--warmup run past REF_BUDGET_S (the oracle's throughput per particle does not depend on it)
    wsmp = oracle_slice(w, three)
    t1 = _oracle_worker((wsmp, three, 0, 1, 1e9))[2]
    projected = t1 * (args.steps + args.warmup)
    if projected > REF_BUDGET_S and not three:
        # at least 96 rows: the first ~60 hold the PML, the guard and the antenna but no plasma
        rows = max(96, int(ORACLE_ROWS * REF_BUDGET_S / projected) // 16 * 16)
        wsmp = oracle_slice(w, three, rows)
    r = oracle_throughput(wsmp, three, procs, args.warmup, args.steps, REF_BUDGET_S)
    v = r["value"]
    box = f"{wsmp['nz']} x {wsmp['ny']} x {wsmp['nx']}" if three else f"{wsmp['nz']} x {wsmp['nx']}"
    line = {"metric": "particle-steps/s", "value": v, "unit": "particle-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["seconds"] / max(r["steps"], 1) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": w["name"] + f" (bounded sample: {box} cells)",
                       "grid": [w["nz"], w["ny"], w["nx"]] if three else [w["nz"], w["nx"]],
                       "ppc": 2 if three else 16, "precision": "fp64 oracle"},
            "cpu_baseline": {"kind": "oracle", "cores": r["copies"], "value": v, "unit": "particle-steps/s",
                             "cpu": cpu,
                             "sample": f"{box}-cell slice, {r['particles']} electrons per copy, {r['copies']} "
                                       f"copies of the single-threaded oracle (one per host core), {r['steps']} "
                                       f"timed steps after {args.warmup}, {r['seconds']:.1f} s"},
            "e2e": {"value": v, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ensemble(args):
    """N uneven runs (seeded recipe) advanced together; also the same runs one after the other."""
    import torch
    from paper_1009_2727_gb300 import workloads as W
    from paper_1009_2727_gb300.pic import Ensemble
    torch.cuda.set_device(0)
    ws = W.ensemble_2d(args.ensemble)
    t_tune = time.perf_counter()
    ens = Ensemble(ws, tune=args.tune or False)
    t_tune = time.perf_counter() - t_tune
    ens_tuned = ens.tuned
    ens.step(max(args.warmup, 3))
    ens.sync()
    n0 = sum(m.stats()["n_electrons"] for m in ens.members)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    l0 = ens.launches()
    torch.cuda.synchronize()
    ev0.record(stream)
    ens.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    launches = ens.launches() - l0
    ens.sync()
    # batched mode: the same steps with the kernels launched directly instead of replayed from graphs
    direct_ms = None
    if ens.batched:
        ens.use_graphs(False)
        torch.cuda.synchronize()
        ev0.record(stream)
        ens.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        direct_ms = ev0.elapsed_time(ev1) / args.steps
        ens.use_graphs(True)
        ens.sync()
    # host time to enqueue one ensemble step on idle queues (does the host or the GPU set the pace?)
    enq = []
    for _ in range(5):
        torch.cuda.synchronize()
        th0 = time.perf_counter()
        ens.step(1)
        enq.append((time.perf_counter() - th0) * 1e3)
    enqueue_ms = float(sorted(enq)[len(enq) // 2])
    torch.cuda.synchronize()
    n1 = sum(m.stats()["n_electrons"] for m in ens.members)
    cells = sum(w["nx"] * w["nz"] for w in ws)
    ens_batched = ens.batched
    # the same runs one at a time, each on the caller's stream
    seq_ms = 0.0
    ens.close()
    from paper_1009_2727_gb300.pic import Simulation
    for i, w in enumerate(ws):
        lay = {"tile": ens_tuned[i]["tile"], "sort_every": ens_tuned[i]["sort_every"]} if args.tune else {}
        s = Simulation(w, **lay)
        s.step(max(args.warmup, 3))
        torch.cuda.synchronize()
        ev0.record(stream)
        s.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        seq_ms += ev0.elapsed_time(ev1)
        s.close()
    ps = 0.5 * (n0 + n1) * args.steps
    line = {"metric": "ensemble particle-steps/s", "value": ps / (ms * 1e-3), "unit": "particle-steps/s",
            "n_gpus": 1, "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"ensemble_2d({args.ensemble}) seeded uneven runs", "runs": len(ws),
                       "cells": cells, "electrons": int(0.5 * (n0 + n1))},
            "sequential_ms_per_step": seq_ms / args.steps, "speedup_vs_sequential": seq_ms / ms,
            "host_enqueue_ms_per_step": enqueue_ms,
            "batched": bool(ens_batched), "gpu_launches": int(launches),
            "launches_per_step": launches / args.steps, "direct_launch_ms_per_step": direct_ms,
            "clocks": clocks,
            "autotuned": args.tune or None, "setup_s": t_tune,
            "ensemble_trials": ens_tuned[0].get("trials") if args.tune == "ensemble" else None,
            "tiles": sorted({(t["tile"][0], t["tile"][1], t["sort_every"]) for t in ens_tuned}) if args.tune else None}
    print(json.dumps(line), flush=True)
    return 0


def run_surrogate(args):
    """Stage surrogate: label N seeded stage runs through the ensemble, train the library's MLP on the valid
    ones, score it on 50 fresh held-out runs (seed 5), and time serving in batches of 1e5 queries, device
    resident and host to host."""
    import numpy as np
    import torch
    from paper_1009_2727_gb300 import workloads as W
    from paper_1009_2727_gb300 import surrogate as S
    torch.cuda.set_device(0)
    n_tr = args.surrogate
    tr, te = W.surrogate_runs(n_tr, seed=1), W.surrogate_runs(50, seed=5)
    t0 = time.time()
    Xtr, Ytr, oktr = S.stage_labels(tr)
    t_label = time.time() - t0
    t0 = time.time()
    Xte, Yte, okte = S.stage_labels(te)
    t_pic_heldout = time.time() - t0
    sur = S.Surrogate(hidden=(256, 256, 256), seed=0)
    epochs, batch = 1500, 64
    t0 = time.time()
    curve = sur.fit(Xtr[oktr], Ytr[oktr], epochs=epochs, batch=batch, lr=1e-3, weight_decay=1e-4)
    torch.cuda.synchronize()
    t_fit = time.time() - t0
    pred, inside = sur.predict(Xte[okte])
    yt, pt = Yte[okte][inside], pred[inside]
    # R^2 per output; none for an output that does not vary over the held-out runs
    var = yt.var(0)
    r2 = [float(1.0 - ((pt[:, k] - yt[:, k]) ** 2).mean() / var[k]) if var[k] > 1e-12 else None
          for k in range(yt.shape[1])]
    g, gp = yt[:, 0], pt[:, 0]
    big = np.abs(g) > 5.0
    rel = np.abs(gp - g)[big] / np.abs(g[big])
    # serving: batches of 1e5 standardised queries resident on the device, events on the MLP's stream
    Q = 100000
    rng = np.random.default_rng(0)
    q = rng.uniform(Xtr.min(0), Xtr.max(0), (Q, 6))
    xd = torch.as_tensor(((q - sur.xm) / sur.xs).astype(np.float32)).cuda()
    yd = torch.empty((Q, len(S.OUTPUTS)), dtype=torch.float32, device="cuda")
    net = sur.net
    stream = net.stream

    def serve_ms():
        for _ in range(max(args.warmup, 3)):
            net.forward_device(xd.data_ptr(), Q, yd.data_ptr())
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            net.forward_device(xd.data_ptr(), Q, yd.data_ptr())
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    # CUDA-core GEMMs for comparison, then the fused tcgen05 kernel (the default path)
    net.use_tensor_cores(False)
    ms_cc = serve_ms()
    net.use_tensor_cores(True)
    ms = serve_ms()
    t0 = time.time()
    for _ in range(args.steps):
        sur.predict(q)
    e2e_s = (time.time() - t0) / args.steps
    w = [6, 256, 256, 256, len(S.OUTPUTS)]
    flops = 2 * sum(w[i] * w[i + 1] for i in range(len(w) - 1))
    peaks = measured_peaks()
    achieved = flops * Q / (ms * 1e-3) / 1e12
    run_steps = sum(r["steps"] for r in tr)
    line = {"metric": "surrogate queries/s", "value": Q / (ms * 1e-3), "unit": "queries/s", "n_gpus": 1,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True,
            "dtype": "bf16 (fp32 accumulate)", "data": "synthetic",
            "config": {"workload": "stage surrogate 6-256-256-256-4 over surrogate_runs (1600 x 96 cells, mixed)",
                       "train_runs": n_tr, "valid_train_runs": int(oktr.sum()), "heldout_runs": int(okte.sum()),
                       "queries_per_step": Q},
            "heldout": {"r2": dict(zip(S.OUTPUTS, [None if v is None else round(v, 4) for v in r2])),
                        "gain_rms_mev": float(np.sqrt(((gp - g) ** 2).mean())),
                        "gain_rel_err_median": float(np.median(rel)) if rel.size else None,
                        "gain_within_5pct": float(np.mean(rel < 0.05)) if rel.size else None,
                        "inside_box": float(inside.mean()),
                        "pic_s_per_run": t_pic_heldout / len(te)},
            "labeling": {"runs_per_s": n_tr / t_label, "run_steps_per_s": run_steps / t_label, "seconds": t_label},
            "training": {"seconds": t_fit, "epochs": epochs, "batch": batch, "final_loss": float(curve[-1])},
            "cuda_core_path": {"ms_per_batch": ms_cc, "queries_per_s": Q / (ms_cc * 1e-3)},
            "roofline": {"kernel": "k_mlp_fwd_tc (tcgen05, fused layers)", "bound": "tensor", "achieved": achieved,
                         "peak": peaks.get("bf16_tflops"), "unit": "TFLOP/s",
                         "frac": achieved / peaks["bf16_tflops"] if peaks.get("bf16_tflops") else None,
                         "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst, of measured)",
                         "flops_per_query": flops, "traffic": None},
            "e2e": {"value": Q / e2e_s, "unit": "queries/s", "h2d_bytes_per_step": Q * 6 * 4,
                    "d2h_bytes_per_step": Q * len(S.OUTPUTS) * 4}}
    print(json.dumps(line), flush=True)
    return 0


BYTES_PER_PARTICLE_1D = {"mixed": 44, "fp64": 64}


def run_1d(args):
    """App. I's 1D scaled stage (952 cells of lambda/24, 10 particles per cell, lab frame, window at c,
    c dt = dz, one bilinear pass on the current): particle-steps/s of the whole step, the push's roofline
    and the oracle on the same workload"""
    import torch
    from paper_1009_2727_gb300 import workloads as W
    from paper_1009_2727_gb300.pic import Simulation
    torch.cuda.set_device(0)
    w = W.app1_lwfa(True)
    w["precision"] = args.precision
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        wo = dict(w)
        wo["precision"] = "fp64"
        o = oracle.Sim1(wo)
        o.step(200)
        n = o.diag()["n_e"]
        t0 = time.perf_counter()
        k = 0
        while k < 4000 and time.perf_counter() - t0 < 10.0:
            o.step(100)
            k += 100
        dt = time.perf_counter() - t0
        cpu = {"value": n * k / dt, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
               "sample": f"{w['name']}: {int(n)} electrons, {k} steps after 200, {dt:.1f} s, single thread"}
    sim = Simulation(w, precision=args.precision)
    sim.step(max(args.warmup, 3) + 200)
    sim.sync()
    n0 = sim.stats()["n_electrons"]
    stream = torch.cuda.current_stream()
    sim.timing(True, 0)
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    torch.cuda.synchronize()
    l0 = sim.launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    sim.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    launches = sim.launches() - l0
    ms = ev0.elapsed_time(ev1)
    push_ms, push_n = sim.timing(False)
    n1 = sim.stats()["n_electrons"]
    n_avg = 0.5 * (n0 + n1)
    value = n_avg * args.steps / (ms * 1e-3)
    peaks = measured_peaks()
    peak = peaks.get("hbm_gbs", 6800.0)
    bpp = BYTES_PER_PARTICLE_1D[args.precision]
    push_avg = push_ms / max(push_n, 1)
    achieved = n_avg * bpp / (push_avg * 1e-3) / 1e9
    roof = {"kernel": "k1_push (1D gather + Boris + Esirkepov)", "bound": "hbm", "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": achieved / peak, "traffic": None,
            "note": "9e3 particles and 953 nodes: the 1D step is launch- and latency-bound (about ten launches "
                    "of a few microseconds); the byte roofline does not bind",
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks else "fallback",
            "algorithmic_bytes_per_particle": bpp, "push_ms_per_step": push_avg}
    sim.close()
    e2e = None
    if not args.no_e2e:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = Simulation(w, precision=args.precision)
        k2 = args.steps
        for _ in range(k2):
            s2.step(1)
            st = s2.stats()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        e2e = {"value": st["n_electrons"] * k2 / wall, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
               "d2h_bytes_per_step": 160,
               "note": f"wall clock of pic_init + pic_load_plasma + {k2} x (pic_step + pic_get_stats)"}
        s2.close()
    line = {"metric": "particle-steps/s", "value": value, "unit": "particle-steps/s", "n_gpus": 1,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": w["name"],
                       "positions": ("int32 cell + f32 in-cell offset (z in the plasma's drifting frame)"
                                     if args.precision == "mixed" else "f64"), "grid": [w["nz"]], "ppc": 10, "gamma_boost": 1.0,
                       "solver": "Yee (1D)", "c_dt_over_dz": 1.0, "filter": "1 pass, no compensation",
                       "shape_order": 3, "precision": args.precision, "electrons": int(n_avg),
                       "moving_window": "lab frame at c", "l2": "fits in L2 (a 1D run is small)",
                       "parallelism": "1 GPU"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


def run_stage3d(args):  # noqa: C901
    """Config 3 as a whole run: the 3D stage (1024 x 128 x 128 cells, gamma 30, CK2 at c dt = dz/sqrt(2),
    Friedman 0.1, 16-cell PML, 4 passes + compensation) stepped --stage3d steps with lab-frame snapshots: one
    lab time per 50 boosted steps (the lab time at which the box centre's boosted time is a multiple of 50
    steps), each sampled at 16 lab stations across the box. Reports the throughput over the whole run, the
    field energy every 1000 steps, the lab rows filled and the wall time."""
    import ctypes
    import numpy as np
    import torch
    from paper_1009_2727_gb300 import capi
    from paper_1009_2727_gb300 import workloads as W
    from paper_1009_2727_gb300.pic import Simulation
    torch.cuda.set_device(0)
    w = W.stage_3d()
    w["precision"] = args.precision
    if args.theta >= 0.0:
        w["theta"] = args.theta
    sim = Simulation(w, precision=args.precision)
    st = sim.stats()
    dt, dz, gam, be = st["dt"], st["dz"], st["gamma"], st["beta"]
    c = 299792458.0
    every, n_st = 50, 16
    n_snap = max(args.stage3d // every, 1)
    zlo, zhi = st["gz_lo"] * dz, st["gz_hi"] * dz
    zc = 0.5 * (zlo + zhi)
    zl, tl = [], []
    for j in range(1, n_snap + 1):
        tp = j * every * dt
        t_lab = gam * (tp + be * zc / c)
        z_c = gam * (zc + be * c * tp)
        half = 0.5 * (zhi - zlo) / gam
        for q in range(n_st):
            zl.append(z_c - half + (q + 0.5) * 2.0 * half / n_st)
            tl.append(t_lab)
    sim.btd_set(np.array(zl), np.array(tl))
    n0 = sim.stats()["n_electrons"]
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    energy = []
    t_wall = time.perf_counter()
    torch.cuda.synchronize()
    ev0.record(stream)
    done = 0
    while done < args.stage3d:
        k = min(1000, args.stage3d - done)
        sim.step(k)
        done += k
        sim.sync()
        fe = sim.stats()["field_energy"]
        energy.append([done, fe])
        if not np.isfinite(fe):
            break
    ev1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    n1 = sim.stats()["n_electrons"]
    o = capi.PicBtdOut()
    o.struct_size = ctypes.sizeof(capi.PicBtdOut)
    o.version = capi.API_VERSION
    o.data = None
    o.done = None
    o.on_device = 0
    sim._check(sim.L.pic_boosted_to_lab_diag(sim.h, None, ctypes.byref(o)), "pic_boosted_to_lab_diag")
    e = np.array(energy)
    peak_emit = e[:, 1].max()
    line = {"metric": "particle-steps/s", "value": 0.5 * (n0 + n1) * done / (ms * 1e-3), "unit": "particle-steps/s",
            "n_gpus": 1, "steps": done, "ms_per_step": ms / done, "higher_is_better": True,
            "dtype": "f32" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": w["name"] + " (whole run)", "grid": [w["nz"], w["ny"], w["nx"]], "ppc": 2,
                       "gamma_boost": w["gamma_boost"], "solver": "CK2", "c_dt_over_dz": 1 / np.sqrt(2.0),
                       "theta": w["theta"], "filter": "4 passes + compensation", "precision": args.precision,
                       "electrons": int(0.5 * (n0 + n1)),
                       "lab_snapshots": {"every_steps": every, "snapshots": n_snap, "stations_each": n_st,
                                         "rows": len(zl), "rows_filled": int(o.n_rows_filled)}},
            "field_energy_every_1000_steps": e.tolist(),
            "finite": bool(np.isfinite(e[:, 1]).all()),
            "final_over_peak_energy": float(e[-1, 1] / peak_emit) if peak_emit > 0 else None,
            "wall_s": wall, "clocks": clocks, "gpu_launches": int(sim.launches())}
    sim.close()
    print(json.dumps(line), flush=True)
    return 0


def run_layout_sweep(args):
    """every particle layout the autotuner can return (tiles {8, 16, 32}^2, sort cadences 8, 16, 32, 64, 128;
    --sweep-cadences restricts the cadences) on the given box, a few steps each: run under ncu with the DRAM
    byte counters to tabulate the push kernel's traffic per particle for each layout (prints one line per
    layout with its electron count)"""
    import torch
    from paper_1009_2727_gb300 import workloads as W
    from paper_1009_2727_gb300.pic import Simulation
    torch.cuda.set_device(0)
    w = W.stage_2d()
    if args.nz:
        w = W.shrink(w, w["nx"], args.nz)
    for tx in (8, 16, 32):
        for tz in (8, 16, 32):
            for se in (int(v) for v in args.sweep_cadences.split(",")):
                sim = Simulation(w, precision=args.precision, tile=(tx, tz), sort_every=se)
                sim.step(args.steps)
                sim.sync()
                print(json.dumps({"tile": [tx, tz], "sort_every": se, "steps": args.steps,
                                  "electrons": sim.stats()["n_electrons"]}), flush=True)
                sim.close()
    return 0


def run_solver_accuracy(args):
    """Sec. 5.1.2's comparison of damping and smoothing against the frame: the scaled stage (n_e = 1e19 cm^-3,
    workloads.scaled_stage) in frames boosted by gamma = 2, 3, 5, 8, 13 (gamma_w = 13.2), each with the CK solver
    undamped (the reference), the Yee-Friedman solver at theta = 1, and the Yee solver with the wide-band
    filter S(1:2:4); the test beam's energy gain at the end of the stage (the same physical time in every
    run of a frame), its deviation from the reference, and the GPU time of each run"""
    import numpy as np
    import torch
    from paper_1009_2727_gb300 import workloads as W
    from paper_1009_2727_gb300.pic import Simulation
    torch.cuda.set_device(0)
    me_mev = 0.51099895000
    cases = (("ck", "ck", 0.0, None), ("ck_friedman_0.1", "ck", 0.1, None), ("yee_friedman_1", "yee", 1.0, None),
             ("yee_S124", "yee", 0.0, (1, 2, 4)))
    out = []
    for g in (2.0, 3.0, 5.0, 8.0, 13.0):
        row = {"gamma_boost": g}
        for name, solver, theta, strides in cases:
            w = W.scaled_stage(g, solver, theta, strides)
            w["precision"] = args.precision
            dt_ref = W.scaled_stage(g)["dt"]
            sim = Simulation(w, precision=args.precision)
            st = sim.stats()
            steps = int(np.ceil(w["steps"] * dt_ref / st["dt"]))
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            stream = torch.cuda.current_stream()
            torch.cuda.synchronize()
            ev0.record(stream)
            sim.step(steps)
            ev1.record(stream)
            torch.cuda.synchronize()
            sim.sync()
            st = sim.stats()
            gain = (st["beam_gamma_lab"] - w["gamma_w"]) * me_mev if st["n_beam_active"] > 0 else None
            row[name] = {"gain_mev": gain, "steps": steps, "dt_s": st["dt"], "gpu_ms": ev0.elapsed_time(ev1),
                         "beam_active": int(st["n_beam_active"]), "field_energy": st["field_energy"]}
            sim.close()
        ref = row["ck"]["gain_mev"]
        for name, _, _, _ in cases[1:]:
            gn = row[name]["gain_mev"]
            row[name]["rel_dev_from_ck"] = abs(gn - ref) / abs(ref) if (gn is not None and ref) else None
        out.append(row)
        print(json.dumps(row), flush=True)
    line = {"metric": "beam energy gain deviation from the undamped run", "unit": "relative",
            "higher_is_better": False, "data": "synthetic",
            "config": {"workload": "scaled_stage (n_e 1e19 cm^-3, a0 1.5, w0 12 um, tau 30 fs, L 0.4 mm)",
                       "precision": args.precision, "gamma_w": W.scaled_stage(13.0)["gamma_w"]},
            "rows": out}
    print(json.dumps(line), flush=True)
    return 0


def run_app1(args):
    """App. I on the GPU: the Nyquist (odd-even) mode grows without the current filter and is removed by
    one bilinear pass"""
    import torch
    torch.cuda.set_device(0)
    from paper_1009_2727_gb300 import stability
    t0 = time.time()
    runs = stability.app1_runs(20000, every=2000)
    line = {"metric": "nyquist_share_Ey", "unit": "share of the E_y power at k dz > 3 pi / 4",
            "higher_is_better": False, "data": "synthetic",
            "config": {"workload": "app1_lwfa_952", "precision": "mixed", "steps": 20000, "c_dt_over_dz": 1.0},
            "runs": runs, "wall_s": time.time() - t0}
    print(json.dumps(line), flush=True)
    return 0


def run_dt_scan(args):
    """the time-step scan of the instability (Sec. 5) for the Yee-located and the node-interpolated gather"""
    import torch
    torch.cuda.set_device(0)
    from paper_1009_2727_gb300 import stability
    t0 = time.time()
    runs = stability.dt_scan((0.5, 0.55, 0.6, 0.65, 0.7071, 0.75, 0.8))
    line = {"metric": "high_k_Ez_power", "unit": "(V/m)^2 summed over k dz > pi/4", "higher_is_better": False,
            "data": "synthetic", "config": {"workload": "stage_2d_4096x256_g13", "precision": "mixed",
                                            "times": "t = m dz/(sqrt(2) c), m = 1200, 1800, 2400"},
            "runs": runs, "wall_s": time.time() - t0}
    print(json.dumps(line), flush=True)
    return 0


def wide_band(w, strides, three):
    """the stage with a wide-band filter (its passes + compensation at each stride); the default particle
    guard grows with the halo, so the antenna moves to 4 cells inside the particle domain"""
    w = dict(w)
    w["filter_strides"] = strides
    w["laser"] = dict(w["laser"])
    gam = w["gamma_boost"]
    dz = (1.0 + (1.0 - 1.0 / gam ** 2) ** 0.5) * gam * w["dz_lab"]
    halo = (w["filter_passes"] + (1 if w["filter_compensate"] else 0)) * sum(strides)
    guard = (3 if w["order"] == 3 else 2) + halo + 2
    w["laser"]["z_antenna"] = max(w["laser"]["z_antenna"], (w["pml_cells"] + guard + 4) * dz)
    w["name"] = w["name"] + "_S(" + ":".join(str(v) for v in strides) + ")"
    return w


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=8)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--order", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--sweep-cadences", default="8,16,32,64,128",
                    help="sort cadences of --layout-sweep (comma-separated)")
    ap.add_argument("--nz", type=int, default=0, help="smaller box for profiling captures (default: the full 4096)")
    ap.add_argument("--sort-every", type=int, default=0, help="steps between particle sorts (0: the library default)")
    ap.add_argument("--ensemble", type=int, default=0,
                    help="time N uneven runs advanced together (pic_ensemble_*) instead of the stage")
    ap.add_argument("--tune", default="", choices=["", "runs", "ensemble", "layout"],
                    help="with --ensemble: layouts from pic_autotune per run, or from pic_ensemble_autotune; "
                         "layout (default without --ensemble): the single run's tile and sort cadence from "
                         "pic_autotune, before the timed steps")
    ap.add_argument("--no-tune", action="store_true", help="the library's default particle layout")
    ap.add_argument("--tile", default="", help="fixed particle tile x,z (no tuning), e.g. 8,16")
    ap.add_argument("--surrogate", type=int, default=0,
                    help="label N stage runs, train the stage surrogate on them and time its serving")
    ap.add_argument("--dim", type=int, default=2, choices=[1, 2, 3],
                    help="3: the 3D stage (1024 x 128 x 128 cells, gamma 30); 1: App. I's 1D scaled stage")
    ap.add_argument("--app1", action="store_true",
                    help="App. I: the 1D scaled stage at c dt = dz over 20000 steps, unfiltered and with one "
                         "bilinear pass on the current (Nyquist-band share of E_y, wake field)")
    ap.add_argument("--solver", default="", help="field-solver preset instead of the workload's (yee, ck, ck2, ...)")
    ap.add_argument("--theta", type=float, default=-1.0, help="Friedman damping instead of the workload's")
    ap.add_argument("--no-filter", action="store_true", help="no filter on the current and the gathered fields")
    ap.add_argument("--gather", default="energy", choices=["energy", "momentum"],
                    help="momentum: the 'momentum conserving' gather (fields interpolated to the nodes first)")
    ap.add_argument("--dt-scan", action="store_true",
                    help="instability level (high-k E_z power at fixed times) against c dt/dz for both gather schemes")
    ap.add_argument("--solver-accuracy", action="store_true",
                    help="Sec. 5.1.2: beam gain of the scaled stage at gamma 2-13 with CK, Yee-Friedman and Yee + S(1:2:4)")
    ap.add_argument("--layout-sweep", action="store_true",
                    help="step every layout the autotuner can return, a few steps each (for a DRAM traffic table)")
    ap.add_argument("--stage3d", type=int, default=0,
                    help="config 3 as a whole run: N steps of the 3D stage with lab snapshots every 50 steps")
    ap.add_argument("--filter-strides", default="",
                    help="wide-band filter, e.g. 1,2,4: the stage's passes + compensation at each stride "
                         "(the antenna moves past the wider particle guard)")
    args = ap.parse_args()

    from paper_1009_2727_gb300 import workloads as W
    three = args.dim == 3
    w = W.stage_3d() if three else W.stage_2d()
    if args.nz:
        w = W.shrink3(w, w["nx"], w["ny"], args.nz) if three else W.shrink(w, w["nx"], args.nz)
    w["order"] = args.order
    w["precision"] = args.precision
    w["gather"] = args.gather
    if args.solver:
        w["solver"] = W.SOLVERS[args.solver]
    if args.theta >= 0.0:
        w["theta"] = args.theta
    if args.no_filter:
        w["filter_J"] = 0
        w["filter_gather"] = 0
    if args.filter_strides:
        w = wide_band(w, [int(v) for v in args.filter_strides.split(",")], three)
    if args.impl == "reference":
        return run_reference(args, w)
    if args.dt_scan:
        return run_dt_scan(args)
    if args.app1:
        return run_app1(args)
    if args.dim == 1 and args.impl != "reference":
        return run_1d(args)
    if args.stage3d:
        return run_stage3d(args)
    if args.layout_sweep:
        return run_layout_sweep(args)
    if args.solver_accuracy:
        return run_solver_accuracy(args)
    if args.ensemble:
        return run_ensemble(args)
    if args.surrogate:
        return run_surrogate(args)

    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    else:
        torch.cuda.set_device(0)
    from paper_1009_2727_gb300.pic import Simulation

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline_line(w, three)

    tuned = None
    if args.tile:
        tl = tuple(int(v) for v in args.tile.split(","))
        tuned = {"tile": tl, "sort_every": args.sort_every, "wall_s": 0.0, "trials": []}
        sim = Simulation(w, precision=args.precision, tile=tl, sort_every=args.sort_every)
    elif args.tune in ("", "layout") and not args.no_tune and not three and not args.sort_every:
        from paper_1009_2727_gb300.pic import autotune
        t_tune = time.perf_counter()
        # the trials time the bench's own window: its warm-up steps, then its timed steps
        tuned = autotune(w, precision=args.precision, warm=max(args.warmup, 3), steps=args.steps)
        tuned["wall_s"] = time.perf_counter() - t_tune
        sim = Simulation(w, precision=args.precision, tile=tuned["tile"], sort_every=tuned["sort_every"])
    else:
        sim = Simulation(w, precision=args.precision, sort_every=args.sort_every)
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        sim.step(1)
    sim.sync()
    n_e = sim.stats()["n_electrons"]
    # per-kernel timing of the push kernel over the timed steps (events on the library's stream)
    sim.timing(True, 0)
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    barrier(ws)
    torch.cuda.synchronize()
    l0 = sim.launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    sim.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clocks = sampler.stop()
    launches = sim.launches() - l0
    ms = ev0.elapsed_time(ev1)
    push_ms, push_n = sim.timing(False)
    # field kernels (Faraday, filters, Ampere) over a shorter run after the timed region
    kf = max(min(args.steps, 50), 1)
    sim.timing(True, 1)
    sim.step(kf)
    field_ms, _ = sim.timing(False)
    sim.sync()
    st1 = sim.stats()
    n_e1 = st1["n_electrons"]
    dt_s = st1["dt"]
    n_avg = 0.5 * (n_e + n_e1)
    value, ms_max = job_throughput(n_avg * args.steps, ms, ws)
    # roofline of the dominant kernel
    peaks = measured_peaks()
    peak = peaks.get("hbm_gbs", 6800.0)
    bpp = (BYTES_PER_PARTICLE_3D if three else BYTES_PER_PARTICLE)[args.precision]
    push_avg_ms = push_ms / max(push_n, 1)
    achieved = n_avg * bpp / (push_avg_ms * 1e-3) / 1e9
    if three:
        tpp = TRAFFIC_BYTES_PER_PARTICLE_3D.get((args.precision, args.order)) if args.gather == "energy" else None
    else:
        lay = (tuple(tuned["tile"]) + (tuned["sort_every"],)) if tuned else None
        ok = args.precision == "mixed" and args.order == 3 and args.gather == "energy"
        tpp = TRAFFIC_BYTES_PER_PARTICLE.get(lay) if ok and lay else None
    roof = {"kernel": "k3_push_tiles (3D gather + Boris + Esirkepov)" if three else "k_push (gather + Boris + Esirkepov)",
            "bound": "hbm", "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": achieved / peak, "traffic": tpp * n_avg if tpp else None,
            "traffic_source": ("ncu dram bytes of k3_push_tiles, 256 x 128 x 128 box, scaled by particles" if three
                               else "ncu dram bytes of k_push, 2048 x 256 box, this layout, scaled by particles") if tpp else None,
            "note": ("3D push on sorted 4x4x16-cell tiles with shared-memory windows: issue- and latency-bound at "
                     "three CTAs per SM (ncu: 44% issue slots, 37% warps active, 4.5k thread-instructions per "
                     "particle, 4% DRAM)" if three else
                     "at cubic order the push is bound by instruction issue and the L1/shared pipe "
                     "(ncu: 64-65% issue slots, 69% L1/TEX, 17% DRAM), not by HBM; see issue and alu"),
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks else "fallback",
            "algorithmic_bytes_per_particle": bpp, "push_ms_per_step": push_avg_ms,
            "field_kernels_ms_per_step": field_ms / kf,
            "share_of_step": push_avg_ms / (ms / args.steps)}
    # the field kernels' roofline (Faraday + Friedman + PML, gather filter, current filter + Ampere): SURVEY's
    # algorithmic bytes per cell-step (all six E/B components and the current, fused) over their measured time
    cells = w["nx"] * w.get("ny", 1) * w["nz"]
    bpc = BYTES_PER_CELL[args.precision]
    field_avg_ms = field_ms / kf
    field_ach = cells * bpc / (field_avg_ms * 1e-3) / 1e9 if field_avg_ms > 0 else None
    roof["field_kernels"] = {"kernels": "k3_faraday_tile, k3_friedman, k3_filter_*, k3_ampere" if three else
                             "k_faraday_fused (k_faraday where it does not apply), k_filter_fields, k_ampere", "bound": "hbm", "achieved": field_ach,
                             "peak": peak, "unit": "GB/s", "frac": field_ach / peak if field_ach else None,
                             "algorithmic_bytes_per_cell": bpc, "ms_per_step": field_avg_ms,
                             "cell_steps_per_s": cells / (field_avg_ms * 1e-3) if field_avg_ms > 0 else None}
    if not three and args.precision == "mixed" and args.order == 3 and args.gather == "energy":
        # the push's instruction-issue and FP32 rooflines: instruction and FLOP counts per particle from ncu,
        # time from the CUDA events above; issue peak = 4 warp-instructions per SM per cycle at the median SM
        # clock sampled during the timed steps; FP32 peak measured by the library's FMA microbenchmark
        nsm = torch.cuda.get_device_properties(0).multi_processor_count
        mhz = clocks.get("sm_mhz") or 2070.0
        issue_peak = 4.0 * nsm * mhz * 1e6
        issue_ach = PUSH_WARP_INST_PER_PARTICLE * n_avg / (push_avg_ms * 1e-3)
        import ctypes
        from paper_1009_2727_gb300 import capi
        sc, pk = ctypes.c_double(0.0), ctypes.c_double(0.0)
        fp32_peak = None
        if capi.load().pic_measure_fp32_peak(ctypes.byref(sc), ctypes.byref(pk)) == 0:
            fp32_peak = max(sc.value, pk.value)
        alu_ach = PUSH_FLOPS_PER_PARTICLE * n_avg / (push_avg_ms * 1e-3) / 1e12
        roof["issue"] = {"achieved": issue_ach, "peak": issue_peak, "unit": "warp-instructions/s",
                         "frac": issue_ach / issue_peak, "warp_instructions_per_particle": PUSH_WARP_INST_PER_PARTICLE,
                         "peak_source": f"4 per SM per cycle x {nsm} SMs x {mhz:g} MHz (sampled)"}
        roof["alu"] = {"achieved": alu_ach, "peak": fp32_peak, "unit": "TFLOP/s",
                       "frac": alu_ach / fp32_peak if fp32_peak else None,
                       "flops_per_particle": PUSH_FLOPS_PER_PARTICLE,
                       "peak_source": "pic_measure_fp32_peak (FMA microbenchmark, measured in this run)"}
    sim.close()
    del sim

    e2e = None
    if not args.no_e2e:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if tuned and args.tile:
            s2 = Simulation(w, precision=args.precision, tile=tuned["tile"], sort_every=args.sort_every)
        elif tuned:
            # the public call with tune=True: pic_autotune_window (its result cached per run shape and window)
            # and pic_init
            s2 = Simulation(w, precision=args.precision, tune=True, tune_window=(max(args.warmup, 3), args.steps))
        else:
            s2 = Simulation(w, precision=args.precision, sort_every=args.sort_every)
        k2 = args.steps
        for _ in range(k2):
            s2.step(1)
            st = s2.stats()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        n2 = st["n_electrons"]
        import ctypes
        from paper_1009_2727_gb300 import capi
        h2d = (ctypes.sizeof(capi.PicConfig) + ctypes.sizeof(capi.PicPlasma) + ctypes.sizeof(capi.PicLaser)) / k2
        e2e_v, _ = job_throughput(n2 * k2, wall * 1e3, ws)
        e2e = {"value": e2e_v, "unit": "particle-steps/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": ctypes.sizeof(capi.PicStats),
               "note": ("wall clock of " + ("pic_autotune_window (cached per run shape and window) + " if tuned else "") +
                        f"pic_init + pic_load_plasma + {k2} x (pic_step + pic_get_stats)")}
        s2.close()

    if rank == 0:
        line = {
            "metric": "particle-steps/s", "value": value, "unit": "particle-steps/s", "n_gpus": ws,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": w["name"],
                       "positions": ("int32 cell + f32 in-cell offset (z in the plasma's drifting frame)"
                                     if args.precision == "mixed" else "f64"),
                       "grid": [w["nz"], w["ny"], w["nx"]] if three else [w["nz"], w["nx"]],
                       "ppc": 2 if three else 16, "gamma_boost": w["gamma_boost"],
                       "solver": args.solver or ("CK2" if three else "CK"), "theta": w["theta"],
                       "filter": "none" if args.no_filter else "4 passes + compensation" + (
                           " at each stride of S(" + ":".join(str(v) for v in w["filter_strides"]) + ")"
                           if w.get("filter_strides") else ""),
                       "shape_order": args.order, "precision": args.precision, "electrons": int(n_avg),
                       "gather": args.gather, "dt_s": dt_s,
                       "layout": ({"tile_x": tuned["tile"][0], "tile_z": tuned["tile"][1],
                                   "sort_every": tuned["sort_every"],
                                   "source": "--tile" if args.tile else "pic_autotune",
                                   "tune_wall_s": tuned["wall_s"], "trials": len(tuned["trials"])}
                                  if tuned else "library default"),
                       "cell_steps_per_s": w["nx"] * w.get("ny", 1) * w["nz"] * args.steps * ws / (ms_max * 1e-3),
                       "l2": "inputs larger than L2 (particle arrays ~0.5 GB, fields ~2.6 GB)" if three else
                             "inputs larger than L2 (particle arrays ~0.9 GB)",
                       "parallelism": f"{ws} independent replicas" if ws > 1 else "1 GPU"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
