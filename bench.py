"""Benchmark: exact DBSCAN throughput (Mpts/s) on one GB300 per rank.

Workload: 3D seed-spreader points, n = 2,000,000, stored FP32, eps = 100,
minPts = 100 (100 random walkers in [0,1e5]^3, ball radius 100, step 50 per
100 points, 0.01% noise).  One step = one full run of the hot path (cells,
MarkCore, BCP connectivity with union-find, labels, border counts) through the
C ABI on inputs resident in device memory.  The 24 MB input fits in L2, so L2
is flushed (256 MiB write) before every timed step, outside the timed interval.

``--impl reference`` times the CPU oracle (FP64, OpenMP on the host cores) on
a bounded sample of the same workload instead.

Under torchrun (N > 1) every rank runs its own replica of the workload on its
own GPU (the problem is one instance, so the ranks share nothing); value =
N * n / (max over ranks of the step time).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "exact DBSCAN Mpts/s on 1 GB300 (3D seed spreader n=2e6, eps=100, minPts=100)"
UNIT = "Mpts/s"
SAMPLE_SLAB = 5e3  # CPU sample: points with x < 5e3 (5% of the box, same local density)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


_N = 2_000_000


def _workload():
    from paper_1912_06255_gb300 import synth
    return synth.spreader_3d_2m(n=_N)


def _cpu_sample(I):
    sel = I.points[:, 0] < SAMPLE_SLAB
    return np.ascontiguousarray(I.points[sel])


def _time_oracle(X, eps, mp, reps=1):
    import oracle
    oracle.build()
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.dbscan(X, eps, mp)
        ts.append(time.perf_counter() - t0)
    return ts, oracle.num_threads()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    I = _workload()
    X = _cpu_sample(I)
    ts, cores = [], 1
    for i in range(args.warmup + args.steps):
        t, cores = _time_oracle(X, I.eps, I.min_pts)
        if i >= args.warmup:
            ts.append(t[0])
    t = statistics.median(ts)
    v = len(X) / t / 1e6
    sample = (f"all {len(X)} points with x < {SAMPLE_SLAB:g} of the {len(I.points)}-point workload "
              f"(same local density); full oracle run per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": I.name, "n": len(I.points), "d": 3, "eps": I.eps, "min_pts": I.min_pts,
                   "sample_n": len(X)},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_gpu(args):
    import torch

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1912_06255_gb300 import DBSCAN, build

    build.build()
    I = _workload()
    n = len(I.points)
    dev = torch.device("cuda", local)
    X = torch.from_numpy(I.points).to(dev)
    ctx = DBSCAN(n, 3, precision=args.precision, schedule=args.schedule)
    core = torch.empty(n, dtype=torch.uint8, device=dev)
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    offs = torch.empty(n + 1, dtype=torch.int64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if dist is not None:
            dist.barrier()

    def step():
        ctx.run(X, I.eps, I.min_pts, border=False, out=(core, labels, offs))

    if args.profile:
        # profiling mode (for ncu): warm-up and timed steps only, no extra runs
        for _ in range(args.warmup + args.steps):
            step()
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"profile": I.name, "steps": args.steps, "warmup": args.warmup}), flush=True)
        return
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    # pair tests per kernel, counted once in an untimed run
    cctx = DBSCAN(n, 3, precision=args.precision, schedule=args.schedule, collect_stats=True)
    cctx.run(X, I.eps, I.min_pts, border=False)
    ev_phase = cctx.stats()["distance_evals_phase"]
    _PAIR_EVALS[4], _PAIR_EVALS[6] = ev_phase[0], ev_phase[1]
    cctx.close()

    # timed region: device time per step with CUDA events; L2 flushed before each step
    ctx.set_option(4, 1)  # phase timing
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    phases = []
    launches = 0
    clocks = ClockSampler(local) if rank == 0 else None
    barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(float(k))
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
        st = ctx.stats()
        phases.append(st["phase_ms"])
        launches += st["kernel_launches"]
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop() if clocks else None
    ms = [a.elapsed_time(b) for a, b in evs]
    t_ms = sum(ms) / len(ms)
    stats = ctx.stats()
    ctx.set_option(4, 0)

    # the plain FP64 path on the same input (a few steps, same flush rule)
    ctx64 = DBSCAN(n, 3, precision="fp64", schedule=args.schedule)
    for _ in range(3):
        ctx64.run(X, I.eps, I.min_pts, border=False, out=(core, labels, offs))
    ms64 = []
    for k in range(max(3, min(args.steps, 5))):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx64.run(X, I.eps, I.min_pts, border=False, out=(core, labels, offs))
        b.record(stream)
        torch.cuda.synchronize()
        ms64.append(a.elapsed_time(b))
    ctx64.close()

    # end to end through the host-buffer entry point (pinned host memory)
    hX = torch.from_numpy(I.points).pin_memory()
    hcore = torch.empty(n, dtype=torch.uint8).pin_memory()
    hlab = torch.empty(n, dtype=torch.int32).pin_memory()
    for _ in range(2):
        ctx.run_host(hX, I.eps, I.min_pts, core=hcore, labels=hlab)
    e2e_ms = []
    for k in range(args.steps):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.run_host(hX, I.eps, I.min_pts, core=hcore, labels=hlab)
        b.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(a.elapsed_time(b))

    def max_over_ranks(x):
        if dist is None:
            return x
        t = torch.tensor([x], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    t_ms = max_over_ranks(t_ms)
    t64 = max_over_ranks(sum(ms64) / len(ms64))
    te2e = max_over_ranks(sum(e2e_ms) / len(e2e_ms))
    if rank == 0:
        ph = [sum(p[i] for p in phases) / len(phases) for i in range(8)]
        pair_tests = {"markcore": _PAIR_EVALS.get(4), "connect": _PAIR_EVALS.get(6)}
        names = ["bbox", "bbox_readback", "keys_sort", "cells_hash_neighbors", "markcore",
                 "compact_schedule", "connect_bcp_uf", "labels_border"]
        # dominant kernel: the MarkCore launch (one kernel, phase 4) or the BCP launch (phase 6)
        dom = 4 if ph[4] >= ph[6] else 6
        roof = _roofline(dom, ph[dom], stats, n)
        line = {
            "metric": METRIC,
            "value": ws * n / (t_ms * 1e-3) / 1e6,
            "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else "f64",
            "data": "synthetic",
            "config": {"workload": I.name, "n": n, "d": 3, "eps": I.eps, "min_pts": I.min_pts,
                       "precision": "fp32 band + fp64 recheck" if args.precision == "fp32" else "fp64",
                       "schedule": args.schedule, "parallelism": f"replicas{ws}",
                       "l2": "flushed (256 MiB write) before every timed step"},
            "fp64_path": {"value": ws * n / (t64 * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": t64},
            "e2e": {"value": ws * n / (te2e * 1e-3) / 1e6, "unit": UNIT,
                    "h2d_bytes_per_step": int(I.points.nbytes), "d2h_bytes_per_step": int(n * 5)},
            "gpu_launches": int(launches),
            "phase_ms": dict(zip(names, [round(x, 4) for x in ph])),
            "roofline": roof,
            "pair_tests": pair_tests,
            "run_stats": {k: stats[k] for k in ("num_cells", "num_core_cells", "num_candidate_pairs",
                                                 "num_pairs_tested", "num_pairs_skipped", "num_core_points",
                                                 "num_border_points", "band_rechecks", "key_bits")},
        }
        if clk:
            line["clocks"] = clk
        if not args.no_cpu_baseline:
            Xs = _cpu_sample(I)
            ts, cores = _time_oracle(Xs, I.eps, I.min_pts)
            line["cpu_baseline"] = {"value": len(Xs) / ts[0] / 1e6, "unit": UNIT, "cores": cores,
                                    "kind": "oracle",
                                    "sample": f"{len(Xs)} points with x < {SAMPLE_SLAB:g} (same local density), "
                                              f"one full oracle run"}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def _roofline(phase, ms, stats, n):
    """Roofline of the dominant kernel.  MarkCore and BCP are pair-distance
    loops bound by the FP32 pipe: achieved = pair tests x 3d flop / kernel time
    (pair tests counted by a separate counting run), peak = 152 SMs x 128 FP32
    lanes x 2 flop x max SM clock."""
    peaks, kind = _peaks()
    clk = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    peak_tflops = 152 * 128 * 2 * clk / 1e12
    evals = _PAIR_EVALS.get(phase)
    if evals is None or ms <= 0:
        return None
    achieved = evals * 9.0 / (ms * 1e-3) / 1e12  # 3d flop per pair test, d = 3
    return {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
            "frac": achieved / peak_tflops, "traffic": None,
            "kernel": "k_markcore" if phase == 4 else "k_connect",
            "peak_source": f"FP32 lanes x max SM clock ({kind} clock)"}


_PAIR_EVALS = {}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--schedule", default="size", choices=["size", "none"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile", action="store_true",
                    help="run warm-up + timed steps only and print no bench line (for ncu)")
    ap.add_argument("--n", type=int, default=2_000_000,
                    help="points of the seed-spreader workload (the bench line is defined at 2,000,000)")
    args = ap.parse_args()
    global _N
    _N = args.n
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
