"""GB300-native exact Euclidean DBSCAN (grid method of Wang, Gu and Shun, SIGMOD 2020).

Python front end of the C ABI declared in include/dbscan_gb300.h.  PyTorch
provides device memory and streams; every clustering step runs in the CUDA
library ``libdbscan_gb300.so``.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

from . import _lib
from ._lib import DbscanError, Stats

__all__ = ["DBSCAN", "Result", "dbscan", "DbscanError", "Stats"]


@dataclass
class Result:
    """Outputs indexed like the input points.

    core:            uint8 [n], 1 for core points (Sec. 2)
    labels:          int32 [n], cluster name (smallest core index of the cluster)
                     for core points, smallest cluster of a border point, -1 noise
    border_offsets:  int64 [n+1] CSR offsets of the border sets (None if not asked)
    border_ids:      int32 [K] ascending cluster names of each non-core point
    stats:           counters of the run
    """
    core: "object"
    labels: "object"
    border_offsets: "object" = None
    border_ids: "object" = None
    stats: dict | None = None


def _torch():
    import torch
    return torch


def _instances(instances, N):
    arr = (_lib.Instance * len(instances))()
    row = 0
    for k, (n, d, eps, mp) in enumerate(instances):
        arr[k].row0, arr[k].n, arr[k].d = row, int(n), int(d)
        arr[k].reserved, arr[k].eps, arr[k].min_pts = 0, float(eps), int(mp)
        row += int(n)
    if row != N:
        raise ValueError("instance sizes must add up to the number of rows")
    return arr


class DBSCAN:
    """A reusable context (device workspace sized for max_points x max_dim)."""

    def __init__(self, max_points: int, max_dim: int, precision: str = "fp32",
                 schedule: str = "size", collect_stats: bool = False, max_iters: int | None = None,
                 cell_bounds: bool = True, graph: bool = True, rho: float = 0.0):
        self.lib = _lib.load()
        self.ctx = ctypes.c_void_p()
        _lib.check(self.lib.dbscan_create(ctypes.byref(self.ctx), int(max_points), int(max_dim)),
                   "dbscan_create")
        self.max_points, self.max_dim = int(max_points), int(max_dim)
        prec = {"fp32": _lib.PREC_FP32_RECHECK, "fp64": _lib.PREC_FP64}[precision]
        sched = {"size": _lib.SCHED_SIZE, "none": _lib.SCHED_NONE, "learned": _lib.SCHED_LEARNED}[schedule]
        self.set_option(_lib.OPT_PRECISION, prec)
        self.set_option(_lib.OPT_SCHEDULE, sched)
        self.set_option(_lib.OPT_COLLECT_STATS, int(bool(collect_stats)))
        self.set_option(_lib.OPT_CELL_BOUNDS, int(bool(cell_bounds)))
        self.set_option(_lib.OPT_BATCH_GRAPH, int(bool(graph)))
        if max_iters is not None:
            self.set_option(_lib.OPT_MAX_ITERS, int(max_iters))
        if rho:
            self.set_approx(rho)

    def set_approx(self, rho: float) -> None:
        """rho-approximate connectivity for the following runs (0 = exact DBSCAN)."""
        _lib.check(self.lib.dbscan_set_approx(self.ctx, float(rho)), "dbscan_set_approx")

    def set_option(self, option: int, value: int) -> None:
        _lib.check(self.lib.dbscan_set_option(self.ctx, option, int(value)), "dbscan_set_option")

    def close(self) -> None:
        if self.ctx:
            self.lib.dbscan_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- autotuner
    def get_option(self, option: int) -> int:
        v = ctypes.c_int64(0)
        _lib.check(self.lib.dbscan_get_option(self.ctx, option, ctypes.byref(v)), "dbscan_get_option")
        return int(v.value)

    def tuning(self) -> dict:
        """The tunable options as set now."""
        return {"schedule": self.get_option(_lib.OPT_SCHEDULE), "cell_bounds": self.get_option(_lib.OPT_CELL_BOUNDS),
                "connect_waves": self.get_option(_lib.OPT_CONNECT_WAVES),
                "connect_cells": self.get_option(_lib.OPT_CONNECT_CELLS),
                "blocks_per_sm": self.get_option(_lib.OPT_BLOCKS_PER_SM),
                "small_cells": self.get_option(_lib.OPT_SMALL_CELLS),
                "pair_boxes": self.get_option(_lib.OPT_PAIR_BOXES),
                "quadtree": self.get_option(_lib.OPT_QUADTREE)}

    def set_tuning(self, t: dict) -> None:
        for key, opt in (("schedule", _lib.OPT_SCHEDULE), ("cell_bounds", _lib.OPT_CELL_BOUNDS),
                         ("connect_waves", _lib.OPT_CONNECT_WAVES), ("connect_cells", _lib.OPT_CONNECT_CELLS),
                         ("blocks_per_sm", _lib.OPT_BLOCKS_PER_SM), ("small_cells", _lib.OPT_SMALL_CELLS),
                         ("pair_boxes", _lib.OPT_PAIR_BOXES), ("quadtree", _lib.OPT_QUADTREE)):
            if key in t:
                self.set_option(opt, int(t[key]))

    def autotune(self, points, eps: float, min_pts: int, reps: int = 3, stream=None) -> dict:
        """dbscan_autotune on a CUDA tensor [n, d]; the choice stays set in the context."""
        torch = _torch()
        pts = points.contiguous()
        n, d = pts.shape
        s = stream if stream is not None else torch.cuda.current_stream(pts.device)
        out = _lib.Tuning()
        dtype = _lib.F32 if pts.dtype == torch.float32 else _lib.F64
        _lib.check(self.lib.dbscan_autotune(self.ctx, pts.data_ptr(), n, d, dtype, float(eps), int(min_pts),
                                            int(reps), ctypes.byref(out), s.cuda_stream), "dbscan_autotune")
        return out.as_dict()

    def autotune_batch(self, points, instances, reps: int = 3, stream=None) -> dict:
        """dbscan_autotune_batch; arguments as for run_batch."""
        torch = _torch()
        pts = points.contiguous()
        N, ld = pts.shape
        arr = _instances(instances, N)
        s = stream if stream is not None else torch.cuda.current_stream(pts.device)
        out = _lib.Tuning()
        dtype = _lib.F32 if pts.dtype == torch.float32 else _lib.F64
        _lib.check(self.lib.dbscan_autotune_batch(self.ctx, arr, len(instances), pts.data_ptr(), ld, dtype,
                                                  int(reps), ctypes.byref(out), s.cuda_stream),
                   "dbscan_autotune_batch")
        return out.as_dict()

    # ---- learned pair scheduler
    def enable_pair_log(self, capacity: int) -> None:
        """Log (features, outcome) of every pair the next runs test (0 = off)."""
        self.set_option(_lib.OPT_PAIR_LOG, int(capacity))

    def pair_log(self):
        """The records of the last logging run: (features [k, 6] f32, labels [k] u8) on the GPU."""
        torch = _torch()
        k = ctypes.c_int64(0)
        k0 = ctypes.c_int64(0)
        st = self.lib.dbscan_get_pair_log(self.ctx, None, None, 0, ctypes.byref(k0))
        if st not in (_lib.OK, 5):
            _lib.check(st, "dbscan_get_pair_log")
        n = int(k0.value)
        feat = torch.empty((max(n, 1), 6), dtype=torch.float32, device="cuda")
        lab = torch.empty(max(n, 1), dtype=torch.uint8, device="cuda")
        if n:
            _lib.check(self.lib.dbscan_get_pair_log(self.ctx, feat.data_ptr(), lab.data_ptr(), n, ctypes.byref(k)),
                       "dbscan_get_pair_log")
        return feat[:n], lab[:n]

    def train_scheduler(self, epochs: int = 20, batch: int = 4096, lr: float = 3e-3, seed: int = 0) -> list:
        """Fit the scheduler network to the last logging run; returns the loss per epoch."""
        import numpy as np
        losses = np.zeros(epochs, dtype=np.float32)
        _lib.check(self.lib.dbscan_train_scheduler(self.ctx, int(epochs), int(batch), float(lr), int(seed),
                                                   losses.ctypes.data), "dbscan_train_scheduler")
        return losses.tolist()

    def scheduler_weights(self):
        import numpy as np
        w = np.zeros(_lib.MLP_PARAMS, dtype=np.float32)
        _lib.check(self.lib.dbscan_scheduler_weights(self.ctx, w.ctypes.data, w.size, 0), "dbscan_scheduler_weights")
        return w

    def set_scheduler_weights(self, w) -> None:
        import numpy as np
        w = np.ascontiguousarray(np.asarray(w, dtype=np.float32))
        _lib.check(self.lib.dbscan_scheduler_weights(self.ctx, w.ctypes.data, w.size, 1), "dbscan_scheduler_weights")

    def scheduler_loss_grad(self, feat, lab):
        """Mean BCE loss and gradient of the network on CUDA tensors feat [n, 6] f32, lab [n] u8."""
        import numpy as np
        g = np.zeros(_lib.MLP_PARAMS, dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        feat, lab = feat.contiguous(), lab.contiguous()
        _lib.check(self.lib.dbscan_scheduler_loss_grad(self.ctx, feat.data_ptr(), lab.data_ptr(), feat.shape[0],
                                                       loss.ctypes.data, g.ctypes.data), "dbscan_scheduler_loss_grad")
        return float(loss[0]), g

    def link_witnesses(self, stream=None):
        """The link witnesses of the last run (made with DBSCAN_OPT_WITNESS on):
        (rep int32 [n], links int32 [k, 2]) on the GPU, see dbscan_link_witnesses."""
        torch = _torch()
        s = stream if stream is not None else torch.cuda.current_stream()
        k = ctypes.c_int64(0)
        st = self.lib.dbscan_link_witnesses(self.ctx, None, None, 0, ctypes.byref(k), s.cuda_stream)
        if st not in (_lib.OK, 5):
            _lib.check(st, "dbscan_link_witnesses")
        n = int(self.stats()["n"])
        rep = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
        links = torch.empty((max(int(k.value), 1), 2), dtype=torch.int32, device="cuda")
        _lib.check(self.lib.dbscan_link_witnesses(self.ctx, rep.data_ptr(), links.data_ptr(), int(k.value),
                                                  ctypes.byref(k), s.cuda_stream), "dbscan_link_witnesses")
        return rep[:n], links[: int(k.value)]

    def stats(self) -> dict:
        st = Stats()
        _lib.check(self.lib.dbscan_get_stats(self.ctx, ctypes.byref(st)), "dbscan_get_stats")
        return st.as_dict()

    def run(self, points, eps: float, min_pts: int, border: bool = True, out=None, stream=None) -> Result:
        """Cluster a CUDA tensor [n, d] of float32 or float64 on the current stream.

        ``out`` may supply preallocated (core u8[n], labels i32[n], offsets i64[n+1])."""
        torch = _torch()
        if not (isinstance(points, torch.Tensor) and points.is_cuda and points.dim() == 2):
            raise ValueError("points must be a CUDA tensor [n, d]")
        if points.dtype not in (torch.float32, torch.float64):
            raise ValueError("points must be float32 or float64")
        pts = points.contiguous()
        n, d = pts.shape
        dev = pts.device
        if out is None:
            core = torch.empty(n, dtype=torch.uint8, device=dev)
            labels = torch.empty(n, dtype=torch.int32, device=dev)
            offs = torch.empty(n + 1, dtype=torch.int64, device=dev) if border else None
        else:
            core, labels, offs = out
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        k = ctypes.c_int64(0)
        dtype = _lib.F32 if pts.dtype == torch.float32 else _lib.F64
        st = self.lib.dbscan_run(self.ctx, pts.data_ptr(), n, d, dtype, float(eps), int(min_pts),
                                 core.data_ptr(), labels.data_ptr(),
                                 offs.data_ptr() if offs is not None else None,
                                 ctypes.byref(k), s.cuda_stream)
        _lib.check(st, "dbscan_run")
        ids = None
        if border:
            ids = torch.empty(max(int(k.value), 1), dtype=torch.int32, device=dev)
            _lib.check(self.lib.dbscan_border_ids(self.ctx, ids.data_ptr(), ids.numel(), s.cuda_stream),
                       "dbscan_border_ids")
            ids = ids[: int(k.value)]
        return Result(core, labels, offs, ids, self.stats())

    def run_batch(self, points, instances, border: bool = True, out=None, stream=None) -> Result:
        """Cluster independent instances stored one after another in a CUDA
        tensor [N, ld] (float32 or float64).  ``instances`` lists (n, d, eps,
        min_pts) in row order; cluster names in the outputs are local to each
        instance (smallest core index counted from the instance's first row)."""
        torch = _torch()
        if not (isinstance(points, torch.Tensor) and points.is_cuda and points.dim() == 2):
            raise ValueError("points must be a CUDA tensor [N, ld]")
        pts = points.contiguous()
        N, ld = pts.shape
        arr = _instances(instances, N)
        dev = pts.device
        if out is None:
            core = torch.empty(N, dtype=torch.uint8, device=dev)
            labels = torch.empty(N, dtype=torch.int32, device=dev)
            offs = torch.empty(N + 1, dtype=torch.int64, device=dev) if border else None
        else:
            core, labels, offs = out
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        k = ctypes.c_int64(0)
        dtype = _lib.F32 if pts.dtype == torch.float32 else _lib.F64
        _lib.check(self.lib.dbscan_run_batch(self.ctx, arr, len(instances), pts.data_ptr(), ld, dtype,
                                             core.data_ptr(), labels.data_ptr(),
                                             offs.data_ptr() if offs is not None else None,
                                             ctypes.byref(k), s.cuda_stream), "dbscan_run_batch")
        ids = None
        if border:
            ids = torch.empty(max(int(k.value), 1), dtype=torch.int32, device=dev)
            _lib.check(self.lib.dbscan_border_ids(self.ctx, ids.data_ptr(), ids.numel(), s.cuda_stream),
                       "dbscan_border_ids")
            ids = ids[: int(k.value)]
        return Result(core, labels, offs, ids, self.stats())

    def run_host(self, points, eps: float, min_pts: int, core=None, labels=None, border=None, stream=None):
        """Cluster host memory (numpy array or CPU tensor, ideally pinned) through
        dbscan_run_host: the copies to and from the device are part of the call.
        ``border`` may be (offsets int64 [n+1], ids int32 [cap]) host tensors for
        the border sets; returns (core, labels, number of border ids)."""
        torch = _torch()
        pts = self._host_points(points)
        n, d = pts.shape
        core = torch.empty(n, dtype=torch.uint8) if core is None else core
        labels = torch.empty(n, dtype=torch.int32) if labels is None else labels
        s = stream if stream is not None else torch.cuda.current_stream()
        off, ids = border if border is not None else (None, None)
        k = ctypes.c_int64(0)
        dtype = _lib.F32 if pts.dtype == torch.float32 else _lib.F64
        _lib.check(self.lib.dbscan_run_host(self.ctx, pts.data_ptr(), n, d, dtype, float(eps), int(min_pts),
                                            core.data_ptr(), labels.data_ptr(),
                                            off.data_ptr() if off is not None else None,
                                            ids.data_ptr() if ids is not None else None,
                                            ids.numel() if ids is not None else 0, ctypes.byref(k), s.cuda_stream),
                   "dbscan_run_host")
        return core, labels, int(k.value)

    def run_batch_host(self, points, instances, core=None, labels=None, border=None, stream=None):
        """dbscan_run_batch_host: run_batch on host memory [N, ld]; returns
        (core, labels, number of border ids)."""
        torch = _torch()
        pts = self._host_points(points)
        N, ld = pts.shape
        arr = _instances(instances, N)
        core = torch.empty(N, dtype=torch.uint8) if core is None else core
        labels = torch.empty(N, dtype=torch.int32) if labels is None else labels
        s = stream if stream is not None else torch.cuda.current_stream()
        off, ids = border if border is not None else (None, None)
        k = ctypes.c_int64(0)
        dtype = _lib.F32 if pts.dtype == torch.float32 else _lib.F64
        _lib.check(self.lib.dbscan_run_batch_host(self.ctx, arr, len(instances), pts.data_ptr(), ld, dtype,
                                                  core.data_ptr(), labels.data_ptr(),
                                                  off.data_ptr() if off is not None else None,
                                                  ids.data_ptr() if ids is not None else None,
                                                  ids.numel() if ids is not None else 0, ctypes.byref(k),
                                                  s.cuda_stream), "dbscan_run_batch_host")
        return core, labels, int(k.value)

    def run_slabs(self, points, eps: float, min_pts: int, slabs: int = 0, border: bool = True, out=None,
                  ids=None, stream=None):
        """dbscan_run_slabs: one instance larger than this context's max_points,
        run slab by slab along its widest dimension and merged exactly.
        ``points`` is host memory (numpy array or CPU tensor) or a CUDA tensor;
        ``slabs`` = 0 picks the fewest that fit.  ``out`` may be (core uint8
        [n], labels int32 [n], offsets int64 [n+1]) tensors in host or device
        memory (default: new pinned host tensors); ``ids`` an int32 tensor for
        the border ids, used when large enough.  Returns (Result, stats dict)."""
        torch = _torch()
        import numpy as np
        if isinstance(points, np.ndarray):
            points = torch.from_numpy(np.ascontiguousarray(points))
        pts = points.contiguous()
        if pts.dtype not in (torch.float32, torch.float64) or pts.dim() != 2:
            raise ValueError("points must be float32/float64 [n, d]")
        n, d = pts.shape
        pin = torch.cuda.is_available()
        if out is None:
            core = torch.empty(n, dtype=torch.uint8, pin_memory=pin)
            labels = torch.empty(n, dtype=torch.int32, pin_memory=pin)
            off = torch.empty(n + 1, dtype=torch.int64, pin_memory=pin) if border else None
        else:
            core, labels, off = out
            if not border:
                off = None
        s = stream if stream is not None else torch.cuda.current_stream()
        k = ctypes.c_int64(0)
        st = _lib.SlabStats()
        dtype = _lib.F32 if pts.dtype == torch.float32 else _lib.F64
        _lib.check(self.lib.dbscan_run_slabs(self.ctx, pts.data_ptr(), n, d, dtype, float(eps), int(min_pts),
                                             int(slabs), core.data_ptr(), labels.data_ptr(),
                                             off.data_ptr() if off is not None else None, ctypes.byref(k),
                                             ctypes.byref(st), s.cuda_stream), "dbscan_run_slabs")
        res_ids = None
        if border:
            K = int(k.value)
            if ids is not None and ids.numel() >= K:
                res_ids = ids[:K]
            else:
                res_ids = torch.empty(K, dtype=torch.int32, pin_memory=pin and K > 0)
            _lib.check(self.lib.dbscan_slab_border_ids(self.ctx, res_ids.data_ptr() if K > 0 else None,
                                                       res_ids.numel(), s.cuda_stream), "dbscan_slab_border_ids")
        return Result(core, labels, off, res_ids), st.as_dict()

    @staticmethod
    def _host_points(points):
        torch = _torch()
        import numpy as np
        pts = torch.from_numpy(np.ascontiguousarray(points)) if isinstance(points, np.ndarray) else points.contiguous()
        if pts.dtype not in (torch.float32, torch.float64) or pts.dim() != 2 or pts.is_cuda:
            raise ValueError("points must be host float32/float64 [n, d]")
        return pts


def dbscan(points, eps: float, min_pts: int, precision: str = "fp32", schedule: str = "size",
           border: bool = True, collect_stats: bool = False, cell_bounds: bool = True, rho: float = 0.0) -> Result:
    """One-shot DBSCAN of a CUDA tensor [n, d] (float32 or float64): exact, or
    rho-approximate when rho > 0."""
    n, d = points.shape
    ctx = DBSCAN(max(int(n), 1), int(d), precision=precision, schedule=schedule,
                 collect_stats=collect_stats, cell_bounds=cell_bounds, rho=rho)
    try:
        return ctx.run(points, eps, min_pts, border=border)
    finally:
        ctx.close()
