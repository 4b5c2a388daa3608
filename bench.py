"""Benchmark: exact DBSCAN throughput (Mpts/s) on one GB300 per rank.

Default workload (``--workload spreader3d``): 3D seed-spreader points,
n = 2,000,000, stored FP32, eps = 100, minPts = 100 (100 random walkers in
[0,1e5]^3, ball radius 100, step 50 per 100 points, 0.01% noise).  One step =
one full run of the hot path (cells, MarkCore, BCP connectivity with
union-find, labels, border counts) through the C ABI on inputs resident in
device memory.  The 24 MB input fits in L2, so L2 is flushed (256 MiB write)
before every timed step, outside the timed interval.

``--workload batch256``: 256 independent 2D/3D blob-plus-noise instances with
log-uniform sizes in [1e3, 1e6] (about 36M points), per-instance eps in
[0.2, 1.0] and minPts in [5, 50], FP32, in one dbscan_run_batch call (one
replayed CUDA graph).

``--impl reference`` times the CPU oracle (FP64, OpenMP on the host cores) on
a bounded sample of the same workload instead.

Under torchrun (N > 1) every rank runs its own replica of the workload on its
own GPU (the problem does not shard, so the ranks share nothing); value =
N * points / (max over ranks of the step time).
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

UNIT = "Mpts/s"
PHASES = ["bbox", "bbox_readback", "cells", "boxes_neighbors", "markcore", "compact_schedule",
          "connect_bcp_uf", "labels_border"]


# ----------------------------------------------------------------- workloads
class SingleInstance:
    """One instance of a seed-spreader workload in one call."""
    SLAB = 5e3  # CPU sample: points with x0 < SLAB (same local density)

    def __init__(self, n):
        self.I = self.make(n if n else self.DEFAULT_N)
        self.n = len(self.I.points)
        self.d = self.I.points.shape[1]
        self.name = self.I.name
        self.config = {"workload": self.I.name, "n": self.n, "d": self.d, "eps": self.I.eps,
                       "min_pts": self.I.min_pts}

    def make_ctx(self, DBSCAN, **kw):
        return DBSCAN(self.n, self.d, **kw)

    def device_input(self, dev):
        import torch
        return torch.from_numpy(self.I.points).to(dev)

    def run(self, ctx, X, out):
        ctx.run(X, self.I.eps, self.I.min_pts, border=False, out=out)

    def run_e2e(self, ctx, hbuf):
        ctx.run_host(hbuf["X"], self.I.eps, self.I.min_pts, core=hbuf["core"], labels=hbuf["labels"])

    def host_buffers(self):
        import torch
        return {"X": torch.from_numpy(self.I.points).pin_memory(),
                "core": torch.empty(self.n, dtype=torch.uint8).pin_memory(),
                "labels": torch.empty(self.n, dtype=torch.int32).pin_memory()}

    def h2d_bytes(self):
        return int(self.I.points.nbytes)

    def heldout(self, dev):
        """A held-out input of the same family (another seed), on the device."""
        import torch
        if getattr(self, "_held", None) is None:
            T = self.make(self.n, seed=self.TRAIN_SEED)
            self._held = (T, torch.from_numpy(T.points).to(dev))
        return self._held

    def log_run(self, ctx, dev):
        """One run on the held-out input, for the scheduler's training log."""
        T, X = self.heldout(dev)
        ctx.run(X, T.eps, T.min_pts, border=False)
        return T.name

    def autotune(self, ctx, dev):
        T, X = self.heldout(dev)
        return ctx.autotune(X, T.eps, T.min_pts, reps=5), T.name

    def cpu_sample(self):
        X = np.ascontiguousarray(self.I.points[self.I.points[:, 0] < self.SLAB])
        desc = (f"{len(X)} points with x0 < {self.SLAB:g} of the {self.n}-point workload (same local density), "
                f"one full oracle run")
        return [(X, self.I.eps, self.I.min_pts)], desc


class Spreader3D(SingleInstance):
    """The 2M-point 3D instance (eps 100, minPts 100)."""
    metric = "exact DBSCAN Mpts/s on 1 GB300 (3D seed spreader n=2e6, eps=100, minPts=100)"
    TRAIN_SEED = 2001
    DEFAULT_N = 2_000_000

    def make(self, n, seed=1001):
        from paper_1912_06255_gb300 import synth
        return synth.spreader_3d_2m(seed=seed, n=n)


class Mixed5D(SingleInstance):
    """The 10M-point 5D instance: half uniform, half seed spreader (minPts 10)."""
    metric = "exact DBSCAN Mpts/s on 1 GB300 (5D mixed uniform + spreader n=1e7, minPts=10)"
    TRAIN_SEED = 2002
    DEFAULT_N = 10_000_000
    EPS = 200.0
    SLAB = 1e3

    def make(self, n, seed=1002):
        from paper_1912_06255_gb300 import synth
        return synth.spreader_5d_10m(seed=seed, n=n, eps=self.EPS)


class VarDen7D(SingleInstance):
    """The 10M-point 7D varying-density instance (minPts 100)."""
    metric = "exact DBSCAN Mpts/s on 1 GB300 (7D varying-density spreader n=1e7, minPts=100)"
    TRAIN_SEED = 2004
    DEFAULT_N = 10_000_000
    EPS = 1000.0
    SLAB = 2e3

    def make(self, n, seed=1004):
        from paper_1912_06255_gb300 import synth
        return synth.spreader_7d_10m(seed=seed, n=n, eps=self.EPS)


class Batch256:
    """256 independent 2D/3D instances in one batched call."""
    metric = "exact DBSCAN Mpts/s on 1 GB300 (batch of 256 2D/3D instances, about 36M points)"

    INSTANCES = 256

    def __init__(self, n):
        from paper_1912_06255_gb300 import synth
        self.B = synth.batch_256(count=self.INSTANCES)
        self.n = sum(len(b.points) for b in self.B)
        P = np.zeros((self.n, 3), np.float32)
        row = 0
        for b in self.B:
            P[row:row + len(b.points), :b.points.shape[1]] = b.points
            row += len(b.points)
        self.P = P
        self.inst = [(len(b.points), b.points.shape[1], b.eps, b.min_pts) for b in self.B]
        self.name = f"batch{len(self.B)}-n{self.n}-f32"
        self.config = {"workload": self.name, "instances": len(self.B), "n": self.n, "d": "2/3",
                       "eps": "U[0.2,1.0]", "min_pts": "U{5..50}"}

    def make_ctx(self, DBSCAN, **kw):
        return DBSCAN(self.n, 3, **kw)

    def device_input(self, dev):
        import torch
        return torch.from_numpy(self.P).to(dev)

    def run(self, ctx, X, out):
        ctx.run_batch(X, self.inst, border=False, out=out)

    def run_e2e(self, ctx, hbuf):
        # the public API path: pinned host -> device, batched run, results -> pinned host
        hbuf["dX"].copy_(hbuf["X"], non_blocking=True)
        ctx.run_batch(hbuf["dX"], self.inst, border=False, out=hbuf["out"])
        hbuf["core"].copy_(hbuf["out"][0], non_blocking=True)
        hbuf["labels"].copy_(hbuf["out"][1], non_blocking=True)

    def host_buffers(self):
        import torch
        return {"X": torch.from_numpy(self.P).pin_memory(), "dX": torch.empty_like(torch.from_numpy(self.P)).cuda(),
                "out": (torch.empty(self.n, dtype=torch.uint8, device="cuda"),
                        torch.empty(self.n, dtype=torch.int32, device="cuda"), None),
                "core": torch.empty(self.n, dtype=torch.uint8).pin_memory(),
                "labels": torch.empty(self.n, dtype=torch.int32).pin_memory()}

    def h2d_bytes(self):
        return int(self.P.nbytes)

    def heldout(self, dev):
        """A held-out batch of 48 instances of the same family (seed 2003), on the device."""
        import torch
        from paper_1912_06255_gb300 import synth
        if getattr(self, "_held", None) is None:
            B = synth.batch_256(seed=2003, count=48)
            n = sum(len(b.points) for b in B)
            P = np.zeros((n, 3), np.float32)
            row = 0
            for b in B:
                P[row:row + len(b.points), :b.points.shape[1]] = b.points
                row += len(b.points)
            inst = [(len(b.points), b.points.shape[1], b.eps, b.min_pts) for b in B]
            self._held = (torch.from_numpy(P).to(dev), inst, f"batch_256(seed=2003, count=48), {n} points")
        return self._held

    def log_run(self, ctx, dev):
        X, inst, name = self.heldout(dev)
        ctx.run_batch(X, inst, border=False)
        return name

    def autotune(self, ctx, dev):
        X, inst, name = self.heldout(dev)
        return ctx.autotune_batch(X, inst, reps=5), name

    def cpu_sample(self):
        order = sorted(range(len(self.B)), key=lambda i: len(self.B[i].points))
        pick, tot = [], 0
        for i in order[::8]:  # every 8th instance by size: a spread of sizes
            if tot + len(self.B[i].points) > 400_000:
                break
            pick.append(i)
            tot += len(self.B[i].points)
        desc = f"{len(pick)} of the 256 instances (every 8th by size), {tot} points, one oracle run each"
        return [(self.B[i].points, self.B[i].eps, self.B[i].min_pts) for i in pick], desc


WORKLOADS = {"spreader3d": Spreader3D, "batch256": Batch256, "mixed5d": Mixed5D, "varden7d": VarDen7D}


# ----------------------------------------------------------------- helpers
def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _max_over_ranks(x, dist, dev):
    """The largest of every rank's x (the step time of the slowest replica)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _time_oracle(samples):
    import oracle
    oracle.build()
    n = 0
    t0 = time.perf_counter()
    for X, eps, mp in samples:
        oracle.dbscan(X, eps, mp)
        n += len(X)
    return n, time.perf_counter() - t0, oracle.num_threads()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
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


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


# DRAM bytes per launch of the dominant kernel, from one ncu capture of the
# same command (dram__bytes_read.sum + dram__bytes_write.sum); None when the
# kernel changed after the capture.  Keyed by (kernel, workload name).
TRAFFIC = {
    # profiles/launches_spreader3d_n2m.md: DRAM read + write per launch at the
    # captured setting (list order, one connect wave, 8 cells per work item);
    # the connect figure holds for one wave only
    ("k_markcore", "spreader3d-n2000000-eps100-minpts100-f32", None): 55439872 + 457472,
    ("k_connect", "spreader3d-n2000000-eps100-minpts100-f32", 1): 47500032 + 50688,
}


def _roofline(kernel, ms, work_pairs, d, workload, executed_pairs=None, waves=None):
    """Roofline of the dominant kernel.  MarkCore and BCP are pair-distance
    loops bound by the FP32 pipe: achieved = algorithmic pair tests x 3d flop
    (d subtractions and d multiply-adds) / the kernel's time, measured with
    CUDA events on the run's stream in the timed steps.  MarkCore's
    algorithmic work is the scan without early exit (the sum over cells
    with fewer than minPts points of |g| times the points of their
    neighbouring cells); BCP's is the pair tests the schedule ran.
    Peak = 152 SMs x 128 FP32 lanes x 2 flop x max SM clock."""
    peaks, kind = _peaks()
    clk = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    peak_tflops = 152 * 128 * 2 * clk / 1e12
    if not work_pairs or ms <= 0:
        return None
    achieved = work_pairs * 3 * d / (ms * 1e-3) / 1e12
    out = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
           "frac": achieved / peak_tflops, "traffic": TRAFFIC.get((kernel, workload, waves)), "kernel": kernel,
           "work_pair_tests": int(work_pairs), "kernel_ms": ms}
    if executed_pairs is not None:
        ex = executed_pairs * 3 * d / (ms * 1e-3) / 1e12
        out.update(executed_pair_tests=int(executed_pairs), executed_achieved=ex, executed_frac=ex / peak_tflops)
    out["peak_source"] = f"152 SMs x 128 FP32 lanes x 2 flop x max SM clock ({kind} clock)"
    return out


# ----------------------------------------------------------------- arms
def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    W = WORKLOADS[args.workload](args.points)
    samples, desc = W.cpu_sample()
    ts, npts, cores = [], 0, 1
    for i in range(args.warmup + args.steps):
        npts, t, cores = _time_oracle(samples)
        if i >= args.warmup:
            ts.append(t)
    t = statistics.median(ts)
    v = npts / t / 1e6
    line = {
        "impl": "reference", "metric": W.metric, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(W.config, sample_n=npts),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


SCHED_CODES = {"size": 0, "none": 1, "learned": 2}


def _train_scheduler(W, ctx, dev):
    """Log every undecided core-cell pair of a held-out input with its exact BCP
    outcome, then fit the scheduler network to the log on the GPU."""
    import torch
    t0 = time.perf_counter()
    ctx.enable_pair_log(1 << 24)
    src = W.log_run(ctx, dev)
    torch.cuda.synchronize()
    records = ctx.stats()["num_pairs_listed"]
    losses = ctx.train_scheduler(epochs=30, batch=4096, lr=3e-3, seed=1)
    ctx.enable_pair_log(0)
    return {"log_source": src, "records": int(min(records, 1 << 24)), "epochs": 30,
            "loss_first": round(losses[0], 4), "loss_last": round(losses[-1], 4),
            "seconds": round(time.perf_counter() - t0, 2)}


def _compare_schedules(W, ctx, X, out, flush, stream, steps):
    """Device time and BCP test counts of each pair schedule on the timed input."""
    import torch
    res = {}
    for name, code in SCHED_CODES.items():
        ctx.set_option(1, code)
        for _ in range(2):
            W.run(ctx, X, out)
        ms = []
        for k in range(steps):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            W.run(ctx, X, out)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        st = ctx.stats()
        res[name] = {"ms_per_step": round(sum(ms) / len(ms), 4), "value": round(W.n / (sum(ms) / len(ms) * 1e-3) / 1e6, 1),
                     "pairs_tested": st["num_pairs_tested"], "pairs_skipped": st["num_pairs_skipped"],
                     "pairs_box_decided": st["num_pairs_box_decided"], "pairs_listed": st["num_pairs_listed"],
                     "bcp_distance_evals": st["distance_evals_phase"][1]}
    return res


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
    W = WORKLOADS[args.workload](args.points)
    n = W.n
    dev = torch.device("cuda", local)
    X = W.device_input(dev)
    ctx = W.make_ctx(DBSCAN, precision=args.precision, schedule="size")
    training = _train_scheduler(W, ctx, dev) if not args.profile or args.schedule == "learned" else None
    ctx.set_option(1, SCHED_CODES[args.schedule])
    tuned = None
    if args.tuning:
        ctx.set_tuning(json.loads(args.tuning))
    elif args.autotune and not args.profile:
        # the autotuner picks schedule, box decisions, waves, work-item size
        # and blocks per SM on the held-out input; the timed runs use its choice
        choice, src = W.autotune(ctx, dev)
        tuned = dict(choice, tuned_on=src)
    setting = ctx.tuning()
    out = (torch.empty(n, dtype=torch.uint8, device=dev), torch.empty(n, dtype=torch.int32, device=dev),
           torch.empty(n + 1, dtype=torch.int64, device=dev))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if dist is not None:
            dist.barrier()

    def step():
        W.run(ctx, X, out)

    if args.profile:
        # profiling mode (for ncu): warm-up and timed steps only, no extra runs
        for _ in range(args.warmup + args.steps):
            step()
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"profile": W.name, "steps": args.steps, "warmup": args.warmup}), flush=True)
        return
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    # pair tests per kernel, counted once in an untimed run
    cctx = W.make_ctx(DBSCAN, precision=args.precision, schedule=args.schedule, collect_stats=True)
    cctx.set_scheduler_weights(ctx.scheduler_weights())
    cctx.set_tuning(setting)
    W.run(cctx, X, out)
    ev_phase = cctx.stats()["distance_evals_phase"]
    mc_bound = cctx.stats()["markcore_pair_bound"]
    band_rechecks = cctx.stats()["band_rechecks"]
    cctx.close()

    # timed region: device time per step with CUDA events; L2 flushed before each
    # step.  The library's phase timing (events between its phases, on the same
    # stream) adds a little time to a step, so it runs in a second timed pass of
    # the same steps, which gives phase_ms and the kernel times of the roofline;
    # a batch replays its captured graph in the first pass and enqueues directly
    # in the second.
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches = 0
    clocks = ClockSampler(local) if rank == 0 else None
    barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(float(k))
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
        launches += ctx.stats()["kernel_launches"]
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop() if clocks else None
    ms = [a.elapsed_time(b) for a, b in evs]
    t_ms = sum(ms) / len(ms)
    stats = ctx.stats()
    # second pass: per-phase CUDA events inside each step
    ctx.set_option(4, 1)
    phases = []
    for k in range(args.steps):
        flush.fill_(float(k))
        step()
        phases.append(ctx.stats()["phase_ms"])
    torch.cuda.synchronize()
    ctx.set_option(4, 0)

    # the plain FP64 path on the same input (a few steps, same flush rule)
    ctx64 = W.make_ctx(DBSCAN, precision="fp64", schedule=args.schedule)
    ctx64.set_scheduler_weights(ctx.scheduler_weights())
    ctx64.set_tuning({k: v for k, v in setting.items() if k != "cell_bounds"})
    for _ in range(3):
        W.run(ctx64, X, out)
    ms64 = []
    for k in range(max(3, min(args.steps, 5))):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        W.run(ctx64, X, out)
        b.record(stream)
        torch.cuda.synchronize()
        ms64.append(a.elapsed_time(b))
    ctx64.close()

    # end to end through the public API from pinned host memory
    hbuf = W.host_buffers()
    for _ in range(2):
        W.run_e2e(ctx, hbuf)
    torch.cuda.synchronize()
    e2e_ms = []
    for k in range(args.steps):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        W.run_e2e(ctx, hbuf)
        b.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(a.elapsed_time(b))

    schedules = _compare_schedules(W, ctx, X, out, flush, stream, max(3, min(args.steps, 5)))
    ctx.set_tuning(setting)

    def max_over_ranks(x):
        return _max_over_ranks(x, dist, dev)

    t_ms = max_over_ranks(t_ms)
    t64 = max_over_ranks(sum(ms64) / len(ms64))
    te2e = max_over_ranks(sum(e2e_ms) / len(e2e_ms))
    if rank == 0:
        ph = [sum(p[i] for p in phases) / len(phases) for i in range(8)]
        dom = 4 if ph[4] >= ph[6] else 6
        dd = getattr(W, "d", 3)
        roof_mc = _roofline("k_markcore", ph[4], mc_bound, dd, W.name, executed_pairs=ev_phase[0])
        roof_cn = _roofline("k_test_pairs" if setting["schedule"] == 2 else "k_connect", ph[6], ev_phase[1], dd,
                            W.name, waves=setting["connect_waves"])
        roof = roof_mc if dom == 4 else roof_cn
        line = {
            "metric": W.metric,
            "value": ws * n / (t_ms * 1e-3) / 1e6,
            "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else "f64",
            "data": "synthetic",
            "config": dict(W.config, precision="fp32 band + fp64 recheck" if args.precision == "fp32" else "fp64",
                           schedule={v: k for k, v in SCHED_CODES.items()}[setting["schedule"]],
                           tuning=setting, parallelism=f"replicas{ws}",
                           l2="flushed (256 MiB write) before every timed step",
                           phase_timing="a second timed pass of the same steps (phase_ms, roofline kernel times)"),
            "fp64_path": {"value": ws * n / (t64 * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": t64},
            "e2e": {"value": ws * n / (te2e * 1e-3) / 1e6, "unit": UNIT,
                    "h2d_bytes_per_step": W.h2d_bytes(), "d2h_bytes_per_step": int(n * 5)},
            "gpu_launches": int(launches),
            "phase_ms": dict(zip(PHASES, [round(x, 4) for x in ph])),
            "roofline": roof,
            "roofline_other": roof_cn if dom == 4 else roof_mc,
            "schedules": dict(schedules, training=training),
            "autotune": tuned,
            "pair_tests": {"markcore": ev_phase[0], "markcore_without_early_exit": mc_bound,
                           "connect": ev_phase[1], "border": ev_phase[2]},
            "run_stats": {k: stats[k] for k in ("num_cells", "num_core_cells", "num_candidate_pairs",
                                                 "num_pairs_tested", "num_pairs_skipped", "num_pairs_box_decided",
                                                 "num_core_points", "num_border_points", "band_rechecks",
                                                 "key_bits")},
        }
        if clk:
            line["clocks"] = clk
        if stats["precision"] == 1:  # FP32 band + FP64 recheck ran
            # pair tests whose FP32 distance fell inside the forward-error band and
            # were decided again in FP64, over all FP32 pair tests of the same run
            line["band_hits"] = {"rechecks": band_rechecks, "fp32_pair_tests": sum(ev_phase),
                                 "fraction": band_rechecks / max(1, sum(ev_phase))}
        if not args.no_cpu_baseline:
            samples, desc = W.cpu_sample()
            npts, t, cores = _time_oracle(samples)
            line["cpu_baseline"] = {"value": npts / t / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
                                    "sample": desc}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="spreader3d", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--schedule", default="size", choices=["size", "none", "learned"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--autotune", action=argparse.BooleanOptionalAction, default=True,
                    help="pick the run settings with the library's autotuner on a held-out input first")
    ap.add_argument("--tuning", default=None,
                    help='explicit settings instead of the autotuner, e.g. \'{"connect_waves": 1, "connect_cells": 8}\'')
    ap.add_argument("--profile", action="store_true",
                    help="run warm-up + timed steps only and print no bench line (for ncu)")
    ap.add_argument("--points", type=int, default=None,
                    help="points of a single-instance workload (default: its defined size, 2e6 in 3D, 1e7 in 5D/7D)")
    ap.add_argument("--eps", type=float, default=None, help="eps of the 5D or 7D workload (default 200 / 1000)")
    ap.add_argument("--instances", type=int, default=None,
                    help="instances of the batch workload (default 256; fewer only for small profiling captures)")
    args = ap.parse_args()
    if args.eps is not None:
        for cls in (Mixed5D, VarDen7D):
            cls.EPS = args.eps
    if args.instances is not None:
        Batch256.INSTANCES = args.instances
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
