"""Benchmark: exact DBSCAN throughput (Mpts/s) on one GB300 per rank.

Default workload (``--workload batch256``), the largest single-GPU one: 256
independent 2D/3D blob-plus-noise instances with log-uniform sizes in
[1e3, 1e6] (36,189,307 points), per-instance eps in [0.2, 1.0] and minPts in
[5, 50], FP32, in one dbscan_run_batch call (one replayed CUDA graph).  One
step = one full pass of the hot path over the batch: cells, neighbour lists,
MarkCore, BCP connectivity with union-find, labels, border counts, and the
border-set fill (dbscan_border_ids), on inputs resident in device memory.

``--workload spreader3d``: 3D seed-spreader points, n = 2,000,000, FP32,
eps = 100, minPts = 100 (100 random walkers in [0,1e5]^3, ball radius 100,
step 50 per 100 points, 0.01% noise); reported beside the batch as an extra
line by default.  ``mixed5d`` / ``varden7d``: the 10M-point 5D and 7D
workloads (``--eps`` picks the sweep point).  ``slabs3d``: one 3D instance of
1e9 points (the seed spreader at the 2M-point workload's local density) on a
context sized for 2.5e8, through dbscan_run_slabs (slabs with halos, merged
exactly); value with device-resident input and outputs, e2e from pinned host
memory to pinned host memory.

L2 is flushed (256 MiB write) before every timed step, outside the timed
interval.  ``e2e`` times the host-buffer C-ABI entry points (dbscan_run_host,
dbscan_run_batch_host) from pinned memory: input upload, the run, and the
download of core flags, labels and the border CSR, every step.

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
METRIC = "exact DBSCAN Mpts/s on 1 GB300: mixed/learned vs plain FP64 path; % roofline"
PHASES = ["bbox", "bbox_readback", "cells", "boxes_lookup", "neighbor_lists", "markcore", "compact_schedule",
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
        return ctx.run(X, self.I.eps, self.I.min_pts, border=True, out=out)

    def run_e2e(self, ctx, hbuf):
        return ctx.run_host(hbuf["X"], self.I.eps, self.I.min_pts, core=hbuf["core"], labels=hbuf["labels"],
                            border=(hbuf["off"], hbuf["ids"]))[2]

    def host_buffers(self, K):
        import torch
        return {"X": torch.from_numpy(self.I.points).pin_memory(),
                "core": torch.empty(self.n, dtype=torch.uint8).pin_memory(),
                "labels": torch.empty(self.n, dtype=torch.int32).pin_memory(),
                "off": torch.empty(self.n + 1, dtype=torch.int64).pin_memory(),
                "ids": torch.empty(max(2 * K, 1024), dtype=torch.int32).pin_memory()}

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
    TRAIN_SEED = 2001
    DEFAULT_N = 2_000_000

    def make(self, n, seed=1001):
        from paper_1912_06255_gb300 import synth
        return synth.spreader_3d_2m(seed=seed, n=n)


class Mixed5D(SingleInstance):
    """The 10M-point 5D instance: half uniform, half seed spreader (minPts 10)."""
    TRAIN_SEED = 2002
    DEFAULT_N = 10_000_000
    EPS = 200.0
    SLAB = 1e3

    def make(self, n, seed=1002):
        from paper_1912_06255_gb300 import synth
        return synth.spreader_5d_10m(seed=seed, n=n, eps=self.EPS)


class VarDen7D(SingleInstance):
    """The 10M-point 7D varying-density instance (minPts 100)."""
    TRAIN_SEED = 2004
    DEFAULT_N = 10_000_000
    EPS = 1000.0
    SLAB = 2e3

    def make(self, n, seed=1004):
        from paper_1912_06255_gb300 import synth
        return synth.spreader_7d_10m(seed=seed, n=n, eps=self.EPS)


def _stack(B):
    n = sum(len(b.points) for b in B)
    P = np.zeros((n, 3), np.float32)
    row = 0
    for b in B:
        P[row:row + len(b.points), :b.points.shape[1]] = b.points
        row += len(b.points)
    return P, [(len(b.points), b.points.shape[1], b.eps, b.min_pts) for b in B]


class Batch256:
    """256 independent 2D/3D instances in one batched call."""
    INSTANCES = 256

    def __init__(self, n):
        from paper_1912_06255_gb300 import synth
        self.B = synth.batch_256(count=self.INSTANCES)
        self.P, self.inst = _stack(self.B)
        self.n = len(self.P)
        self.d = 3
        self.name = f"batch{len(self.B)}-n{self.n}-f32"
        self.config = {"workload": self.name, "instances": len(self.B), "n": self.n, "d": "2/3",
                       "eps": "U[0.2,1.0]", "min_pts": "U{5..50}"}

    def make_ctx(self, DBSCAN, **kw):
        return DBSCAN(self.n, 3, **kw)

    def device_input(self, dev):
        import torch
        return torch.from_numpy(self.P).to(dev)

    def run(self, ctx, X, out):
        return ctx.run_batch(X, self.inst, border=True, out=out)

    def run_e2e(self, ctx, hbuf):
        return ctx.run_batch_host(hbuf["X"], self.inst, core=hbuf["core"], labels=hbuf["labels"],
                                  border=(hbuf["off"], hbuf["ids"]))[2]

    def host_buffers(self, K):
        import torch
        return {"X": torch.from_numpy(self.P).pin_memory(),
                "core": torch.empty(self.n, dtype=torch.uint8).pin_memory(),
                "labels": torch.empty(self.n, dtype=torch.int32).pin_memory(),
                "off": torch.empty(self.n + 1, dtype=torch.int64).pin_memory(),
                "ids": torch.empty(max(2 * K, 1024), dtype=torch.int32).pin_memory()}

    def h2d_bytes(self):
        return int(self.P.nbytes)

    def heldout(self, dev):
        """A held-out batch of 48 instances of the same family (seed 2003), on the device."""
        import torch
        from paper_1912_06255_gb300 import synth
        if getattr(self, "_held", None) is None:
            P, inst = _stack(synth.batch_256(seed=2003, count=48))
            self._held = (torch.from_numpy(P).to(dev), inst, f"batch_256(seed=2003, count=48), {len(P)} points")
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


class Slabs3D:
    """One 3D instance larger than a context's workspace (dbscan_run_slabs):
    the seed spreader scaled to n = 1e9 points at the 2M-point workload's local
    density, eps 100, minPts 100, on a context sized for 2.5e8 points."""
    DEFAULT_N = 1_000_000_000
    CAP = 250_000_000

    def __init__(self, n):
        self.n = int(n) if n else self.DEFAULT_N
        self.d = 3
        self.eps, self.min_pts = 100.0, 100
        self.name = f"slabs3d-spreader-scaled-n{self.n}-eps100-minpts100-f32"
        self.config = {"workload": self.name, "n": self.n, "d": 3, "eps": self.eps, "min_pts": self.min_pts,
                       "context_max_points": min(self.CAP, self.n)}

    def host_input(self):
        """The instance in pinned host memory (generated in place)."""
        import torch
        from paper_1912_06255_gb300 import synth
        X = torch.empty((self.n, 3), dtype=torch.float32, pin_memory=True)
        synth.spreader_3d_scaled(self.n, out=X.numpy())
        return X

    def cpu_sample(self):
        from paper_1912_06255_gb300 import synth
        T = synth.spreader_3d_scaled(100_000, seed=2005)
        desc = "a 100,000-point instance of the same generator (same local density, seed 2005), one oracle run"
        return [(T.points, T.eps, T.min_pts)], desc


WORKLOADS = {"spreader3d": Spreader3D, "batch256": Batch256, "mixed5d": Mixed5D, "varden7d": VarDen7D,
             "slabs3d": Slabs3D}


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


def _time_oracle(samples, threads=0):
    import oracle
    oracle.build()
    n = 0
    t0 = time.perf_counter()
    for X, eps, mp in samples:
        oracle.dbscan(X, eps, mp, threads=threads)
        n += len(X)
    return n, time.perf_counter() - t0, (threads if threads > 0 else oracle.num_threads())


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


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of a
# kernel on a workload, from one ncu capture of this code; a kernel or
# workload not listed reports traffic null.  Keyed by (kernel, workload).
# The batch's neighbour-list kernel was captured on the first 24 instances
# (3,545,259 points: 291.2 MB read + 97.7 MB written in one launch) and is
# scaled to the full batch by its point count (36,189,307 / 3,545,259).
TRAFFIC = {
    ("k_neighbors_super", "batch256-n36189307-f32"): int((291.212032e6 + 97.706752e6) * 36189307 / 3545259),
}


def _neighbor_kernel(d):
    return "k_neighbors_super" if d in (2, 3) else ("k_neighbors" if d <= 4 else "k_lbvh_neighbors")


def _roofline_candidates(ph, run, dd, box, workload, ev_phase):
    """Roofline of the three single-kernel phases; the caller reports the one
    with the longest time.

    Neighbour lists (phase 4, one launch): bound by memory.  Algorithmic bytes
    per cell: its key (8 B; packed coordinates, 16 B, for d >= 5), its point
    box when the FP32-band mode prunes by boxes (32 B; 64 B for d >= 5), the
    two counts it writes (8 B; + an 8 B list offset for d >= 5); plus 4 B per
    list entry written.  achieved = those bytes / the phase's CUDA-event time.

    MarkCore (phase 5) and BCP connectivity (phase 7): bound by the FP32 pipe.
    Work = the pair tests the kernel actually ran (counted in an untimed run
    of the same setting) x 3d flop (d subtractions, d multiply-adds);
    peak = 152 SMs x 128 FP32 lanes x 2 flop x the maximum SM clock."""
    peaks, kind = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    alu = 152 * 128 * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    m, E = run["num_cells"], run["num_neighbor_entries"]
    hd = dd >= 5
    per_cell = (16 if hd else 8) + ((64 if hd else 32) if box else 0) + (16 if hd else 8)
    nbytes = m * per_cell + 4 * E
    kn = _neighbor_kernel(dd)
    out = {}
    if ph[4] > 0:
        a = nbytes / (ph[4] * 1e-3) / 1e9
        out["neighbor_lists"] = {
            "bound": "hbm", "achieved": a, "peak": hbm, "unit": "GB/s", "frac": a / hbm,
            "traffic": TRAFFIC.get((kn, workload)), "kernel": kn, "kernel_ms": ph[4],
            "algorithmic_bytes": int(nbytes), "units": f"{m} cells, {E} list entries",
            "peak_source": f"{kind} copy bandwidth (MEASURED_PEAKS hbm_gbs)" if kind == "measured" else "fallback"}
    for key, kern, i, work in (("markcore", "k_markcore", 5, ev_phase[0]), ("connect", "k_connect", 7, ev_phase[1])):
        if ph[i] > 0:
            a = work * 3 * dd / (ph[i] * 1e-3) / 1e12
            out[key] = {"bound": "alu", "achieved": a, "peak": alu, "unit": "TFLOP/s", "frac": a / alu,
                        "traffic": TRAFFIC.get((kern, workload)), "kernel": kern, "kernel_ms": ph[i],
                        "work_pair_tests": int(work),
                        "peak_source": f"derived: 152 SMs x 128 FP32 lanes x 2 flop x {kind} max SM clock"}
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
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
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


def _timed(fn, flush, stream, steps):
    """CUDA-event times (ms) of `steps` calls of fn, L2 flushed before each."""
    import torch
    ms = []
    for k in range(steps):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    return ms


def _compare_schedules(W, ctx, X, out, flush, stream, steps):
    """Device time and BCP test counts of each pair schedule on the timed input."""
    res = {}
    for name, code in SCHED_CODES.items():
        ctx.set_option(1, code)
        for _ in range(2):
            W.run(ctx, X, out)
        ms = _timed(lambda: W.run(ctx, X, out), flush, stream, steps)
        st = ctx.stats()
        t = sum(ms) / len(ms)
        res[name] = {"ms_per_step": round(t, 4), "value": round(W.n / (t * 1e-3) / 1e6, 1),
                     "pairs_tested": st["num_pairs_tested"], "pairs_skipped": st["num_pairs_skipped"],
                     "pairs_box_decided": st["num_pairs_box_decided"], "pairs_listed": st["num_pairs_listed"]}
    return res


def _measure(W, args, DBSCAN, dev, dist, rank, local, primary):
    """Every number of one workload's line (device-timed steps, phases and
    roofline, the FP64 path, the host-buffer end-to-end leg, schedules)."""
    import torch
    n = W.n
    X = W.device_input(dev)
    ctx = W.make_ctx(DBSCAN, precision=args.precision, schedule="size")
    training = _train_scheduler(W, ctx, dev) if primary else None
    ctx.set_option(1, SCHED_CODES[args.schedule])
    tuned = None
    if args.tuning:
        ctx.set_tuning(json.loads(args.tuning))
    elif args.autotune:
        # the autotuner picks schedule, box decisions, waves, work-item size,
        # blocks per SM and small-cell kernels on the held-out input; the timed
        # runs use its choice
        choice, src = W.autotune(ctx, dev)
        tuned = dict(choice, tuned_on=src)
    setting = ctx.tuning()
    out = (torch.empty(n, dtype=torch.uint8, device=dev), torch.empty(n, dtype=torch.int32, device=dev),
           torch.empty(n + 1, dtype=torch.int64, device=dev))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        return W.run(ctx, X, out)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    # pair tests per kernel and band rechecks, counted once in an untimed run of the same setting
    cctx = W.make_ctx(DBSCAN, precision=args.precision, schedule=args.schedule, collect_stats=True)
    cctx.set_scheduler_weights(ctx.scheduler_weights())
    cctx.set_tuning(setting)
    W.run(cctx, X, out)
    cst = cctx.stats()
    cctx.close()

    # timed region: device time per step with CUDA events, L2 flushed before
    # each step.  The library's phase timing (events between its phases, on the
    # same stream) adds a little time to a step, so it runs in a second timed
    # pass of the same steps, which gives phase_ms and the kernel times of the
    # roofline; a batch replays its captured graph in the first pass and
    # enqueues directly in the second.
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches = 0
    clocks = ClockSampler(local) if (rank == 0 and primary) else None
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(float(k))
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
        launches += ctx.stats()["kernel_launches"]
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop() if clocks else None
    ms = [a.elapsed_time(b) for a, b in evs]
    t_ms = sum(ms) / len(ms)
    stats = ctx.stats()
    K = stats["num_border_memberships"]
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
    ms64 = _timed(lambda: W.run(ctx64, X, out), flush, stream, max(3, min(args.steps, 5)))
    ctx64.close()

    # end to end through the host-buffer C ABI from pinned memory: upload,
    # run, download of core flags, labels and the border CSR
    hbuf = W.host_buffers(K)
    for _ in range(2):
        W.run_e2e(ctx, hbuf)
    torch.cuda.synchronize()
    e2e_ms = _timed(lambda: W.run_e2e(ctx, hbuf), flush, stream, args.steps)
    d2h = n * 1 + n * 4 + 8 * (n + 1) + 4 * K

    schedules = _compare_schedules(W, ctx, X, out, flush, stream, max(3, min(args.steps, 5))) if primary else None
    ctx.set_tuning(setting)

    t_ms = _max_over_ranks(t_ms, dist, dev)
    t64 = _max_over_ranks(sum(ms64) / len(ms64), dist, dev)
    te2e = _max_over_ranks(sum(e2e_ms) / len(e2e_ms), dist, dev)
    ws = 1 if dist is None else dist.get_world_size()
    ph = [sum(p[i] for p in phases) / len(phases) for i in range(len(PHASES))]
    dd = getattr(W, "d", 3)
    box = stats["precision"] == 1 and setting["cell_bounds"] == 1
    ev = cst["distance_evals_phase"]
    cands = _roofline_candidates(ph, stats, dd, box, W.name, ev)
    dom = max(cands, key=lambda key: cands[key]["kernel_ms"]) if cands else None
    res = {
        "value": ws * n / (t_ms * 1e-3) / 1e6, "ms_per_step": t_ms,
        "config": dict(W.config, precision="fp32 band + fp64 recheck" if args.precision == "fp32" else "fp64",
                       schedule={v: k for k, v in SCHED_CODES.items()}[setting["schedule"]], tuning=setting,
                       parallelism=f"replicas{ws}", l2="flushed (256 MiB write) before every timed step",
                       step="one full pass with border sets (run + dbscan_border_ids)",
                       phase_timing="a second timed pass of the same steps (phase_ms, roofline kernel times)"),
        "fp64_path": {"value": ws * n / (t64 * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": t64},
        "e2e": {"value": ws * n / (te2e * 1e-3) / 1e6, "unit": UNIT, "h2d_bytes_per_step": W.h2d_bytes(),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": te2e,
                "path": "dbscan_run_batch_host" if isinstance(W, Batch256) else "dbscan_run_host"},
        "gpu_launches": int(launches),
        "phase_ms": dict(zip(PHASES, [round(x, 4) for x in ph])),
        "roofline": cands.get(dom) if dom else None,
        "roofline_other": {k: v for k, v in cands.items() if k != dom},
        "autotune": tuned,
        "pair_tests": {"markcore": ev[0], "markcore_without_early_exit": cst["markcore_pair_bound"],
                       "connect": ev[1], "border": ev[2]},
        "run_stats": {k: stats[k] for k in ("num_cells", "num_core_cells", "num_neighbor_entries",
                                             "num_candidate_pairs", "num_pairs_tested", "num_pairs_skipped",
                                             "num_pairs_box_decided", "num_core_points", "num_border_points",
                                             "num_border_memberships", "band_rechecks", "key_bits")},
    }
    if schedules is not None:
        res["schedules"] = dict(schedules, training=training)
    if clk:
        res["clocks"] = clk
    if stats["precision"] == 1:  # FP32 band + FP64 recheck ran
        res["band_hits"] = {"rechecks": cst["band_rechecks"], "fp32_pair_tests": sum(ev),
                            "fraction": cst["band_rechecks"] / max(1, sum(ev))}
    ctx.close()
    return res


def _measure_slabs(W, args, DBSCAN, dev, dist, rank, local):
    """Every number of the slab-partition line: device-resident input and
    outputs (value), pinned host input and outputs (e2e), the call's phases,
    and the rooflines of the slab selection and of the slab runs' kernels."""
    import torch
    from paper_1912_06255_gb300 import _lib
    n = W.n
    Xh = W.host_input()
    Xd = Xh.to(dev)
    ctx = DBSCAN(min(W.CAP, n), 3)
    outd = (torch.empty(n, dtype=torch.uint8, device=dev), torch.empty(n, dtype=torch.int32, device=dev),
            torch.empty(n + 1, dtype=torch.int64, device=dev))
    outh = (torch.empty(n, dtype=torch.uint8, pin_memory=True), torch.empty(n, dtype=torch.int32, pin_memory=True),
            torch.empty(n + 1, dtype=torch.int64, pin_memory=True))
    for t in outh:
        t.zero_()  # touch the pinned pages on the host first (first device writes to fresh pages are slow)
    r, st = ctx.run_slabs(Xd, W.eps, W.min_pts, out=outd)
    K = int(r.border_ids.numel())
    idsd = torch.empty(max(2 * K, 1024), dtype=torch.int32, device=dev)
    idsh = torch.zeros(max(2 * K, 1024), dtype=torch.int32, pin_memory=True)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, steps):
        ms = []
        for _ in range(steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return ms

    dev_step = lambda: ctx.run_slabs(Xd, W.eps, W.min_pts, out=outd, ids=idsd)  # noqa: E731
    host_step = lambda: ctx.run_slabs(Xh, W.eps, W.min_pts, out=outh, ids=idsh)  # noqa: E731
    for _ in range(max(3, args.warmup)):
        dev_step()
    clocks = ClockSampler(local) if rank == 0 else None
    torch.cuda.synchronize()
    ms = timed(dev_step, args.steps)
    clk = clocks.stop() if clocks else None
    _, st = dev_step()
    for _ in range(2):
        host_step()
    ms_e2e = timed(host_step, args.steps)
    _, st_e2e = host_step()
    # one untimed call with phase timing and pair-test counts: the last slab's
    # run gives the per-slab kernel times of the roofline
    ctx.set_option(_lib.OPT_PHASE_TIMING, 1)
    ctx.set_option(_lib.OPT_COLLECT_STATS, 1)
    dev_step()
    run = ctx.stats()
    ctx.set_option(_lib.OPT_PHASE_TIMING, 0)
    ctx.set_option(_lib.OPT_COLLECT_STATS, 0)
    ph = run["phase_ms"]
    cands = _roofline_candidates(ph, run, 3, run["precision"] == 1, W.name, run["distance_evals_phase"])
    dom = max(cands, key=lambda key: cands[key]["kernel_ms"]) if cands else None
    peaks, kind = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    sel_bytes = st["slabs"] * n * 12 + (n + st["halo_points"]) * 16
    a = sel_bytes / (st["ms"][1] * 1e-3) / 1e9
    cands["slab_select"] = {"bound": "hbm", "achieved": a, "peak": hbm, "unit": "GB/s", "frac": a / hbm,
                            "traffic": None, "kernel": "k_sl_select", "kernel_ms": st["ms"][1],
                            "algorithmic_bytes": int(sel_bytes),
                            "units": f"{st['slabs']} passes over {n} points, {n + st['halo_points']} selected",
                            "timing": "host-timed selection phase of one call (kernels + count readback)",
                            "peak_source": f"{kind} copy bandwidth (MEASURED_PEAKS hbm_gbs)"}
    t = _max_over_ranks(sum(ms) / len(ms), dist, dev)
    te = _max_over_ranks(sum(ms_e2e) / len(ms_e2e), dist, dev)
    ws = 1 if dist is None else dist.get_world_size()
    line = {"metric": METRIC, "value": ws * n / (t * 1e-3) / 1e6, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(W.config, precision="fp32 band + fp64 recheck", l2="inputs (12 GB) larger than L2",
                           step="one dbscan_run_slabs call with device input and outputs, plus the border-id fetch"),
            "e2e": {"value": ws * n / (te * 1e-3) / 1e6, "unit": UNIT, "h2d_bytes_per_step": int(Xh.numel() * 4),
                    "d2h_bytes_per_step": int(n * 13 + 8 + 4 * K), "ms_per_step": te,
                    "path": "dbscan_run_slabs from pinned host memory, outputs to pinned host memory"},
            "gpu_launches": int(st["kernel_launches"]) * args.steps, "slab_stats": st, "e2e_slab_stats": st_e2e,
            "roofline": dict(cands[dom], note="per-slab kernel: the last slab's run of one call") if dom else None,
            "roofline_other": {k: v for k, v in cands.items() if k != dom}}
    if clk:
        line["clocks"] = clk
    ctx.close()
    return line


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
    dev = torch.device("cuda", local)
    W = WORKLOADS[args.workload](args.points)
    if isinstance(W, Slabs3D):
        line = _measure_slabs(W, args, DBSCAN, dev, dist, rank, local)
        if rank == 0:
            if not args.no_cpu_baseline:
                samples, desc = W.cpu_sample()
                npts, t, cores = _time_oracle(samples)
                line["cpu_baseline"] = {"value": npts / t / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
                                        "sample": desc}
            print(json.dumps(line), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return
    if args.profile:
        # profiling mode (for ncu): warm-up and timed steps only, no extra runs
        X = W.device_input(dev)
        ctx = W.make_ctx(DBSCAN, precision=args.precision, schedule=args.schedule)
        if args.tuning:
            ctx.set_tuning(json.loads(args.tuning))
        out = (torch.empty(W.n, dtype=torch.uint8, device=dev), torch.empty(W.n, dtype=torch.int32, device=dev),
               torch.empty(W.n + 1, dtype=torch.int64, device=dev))
        for _ in range(args.warmup + args.steps):
            W.run(ctx, X, out)
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"profile": W.name, "steps": args.steps, "warmup": args.warmup}), flush=True)
        return
    res = _measure(W, args, DBSCAN, dev, dist, rank, local, primary=True)
    extra = {}
    if args.extra and args.workload != "spreader3d":
        E = Spreader3D(None)
        r = _measure(E, args, DBSCAN, dev, dist, rank, local, primary=False)
        extra[E.name] = {k: r[k] for k in ("value", "ms_per_step", "fp64_path", "e2e", "phase_ms", "roofline",
                                           "autotune", "gpu_launches", "band_hits") if k in r}
        extra[E.name]["unit"] = UNIT
    if args.extra and args.workload == "batch256":
        # the slab partition on a 2e8-point instance with a context for 5e7
        # points (the 1e9-point line is --workload slabs3d)
        S = Slabs3D(200_000_000)
        S.CAP = 50_000_000
        S.config["context_max_points"] = S.CAP
        r = _measure_slabs(S, argparse.Namespace(steps=min(args.steps, 5), warmup=args.warmup), DBSCAN, dev, dist,
                           rank, local)
        extra[S.name] = {k: r[k] for k in ("value", "ms_per_step", "e2e", "roofline", "roofline_other", "gpu_launches",
                                           "slab_stats", "config") if k in r}
        extra[S.name]["unit"] = UNIT
    if rank == 0:
        line = {"metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64",
                "data": "synthetic"}
        line.update({k: v for k, v in res.items() if k not in ("value", "ms_per_step")})
        if extra:
            line["extra_workloads"] = extra
        if not args.no_cpu_baseline:
            samples, desc = W.cpu_sample()
            npts, t, cores = _time_oracle(samples)
            line["cpu_baseline"] = {"value": npts / t / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
                                    "sample": desc}
            npts1, t1, _ = _time_oracle(samples, threads=1)
            line["cpu_baseline_1thread"] = {"value": npts1 / t1 / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
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
    ap.add_argument("--workload", default="batch256", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--schedule", default="size", choices=["size", "none", "learned"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--extra", action=argparse.BooleanOptionalAction, default=True,
                    help="also measure the 2M-point 3D workload (and, with the batch, the slab partition on a "
                         "2e8-point instance) and report them under extra_workloads")
    ap.add_argument("--autotune", action=argparse.BooleanOptionalAction, default=True,
                    help="pick the run settings with the library's autotuner on a held-out input first")
    ap.add_argument("--tuning", default=None,
                    help='explicit settings instead of the autotuner, e.g. \'{"connect_waves": 1, "connect_cells": 8}\'')
    ap.add_argument("--profile", action="store_true",
                    help="run warm-up + timed steps only and print no bench line (for ncu)")
    ap.add_argument("--points", type=int, default=None,
                    help="points of a single-instance workload (default: its defined size, 2e6 in 3D, 1e7 in 5D/7D, "
                         "1e9 for slabs3d)")
    ap.add_argument("--slab-capacity", type=int, default=None,
                    help="max_points of the slabs3d context (default 2.5e8)")
    ap.add_argument("--eps", type=float, default=None, help="eps of the 5D or 7D workload (default 200 / 1000)")
    ap.add_argument("--instances", type=int, default=None,
                    help="instances of the batch workload (default 256; fewer only for small profiling captures)")
    args = ap.parse_args()
    if args.eps is not None:
        for cls in (Mixed5D, VarDen7D):
            cls.EPS = args.eps
    if args.instances is not None:
        Batch256.INSTANCES = args.instances
    if args.slab_capacity is not None:
        Slabs3D.CAP = args.slab_capacity
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
