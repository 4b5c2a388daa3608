"""ctypes binding of the C ABI in include/dbscan_gb300.h.

Argument marshalling only: every step of the clustering runs in the CUDA
library.  If the shared library is missing this module raises; there is no
other implementation to fall back to.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "libdbscan_gb300.so"

OK = 0
STATUS = {
    0: "DBSCAN_OK", 1: "DBSCAN_ERR_INVALID_ARG", 2: "DBSCAN_ERR_UNSUPPORTED_DIM",
    3: "DBSCAN_ERR_OOM", 4: "DBSCAN_ERR_KEY_OVERFLOW", 5: "DBSCAN_ERR_CAPACITY",
    6: "DBSCAN_ERR_CUDA", 7: "DBSCAN_ERR_DEVICE_TIMEOUT", 8: "DBSCAN_ERR_STATE",
}
F32, F64 = 0, 1
OPT_PRECISION, OPT_SCHEDULE, OPT_COLLECT_STATS, OPT_MAX_ITERS, OPT_PHASE_TIMING, OPT_CELL_BOUNDS = 0, 1, 2, 3, 4, 5
OPT_BATCH_GRAPH, OPT_PAIR_LOG = 6, 7
OPT_CONNECT_CELLS, OPT_CONNECT_WAVES, OPT_BLOCKS_PER_SM, OPT_SMALL_CELLS, OPT_PAIR_BOXES = 8, 9, 10, 11, 12
OPT_WITNESS, OPT_QUADTREE, OPT_SLAB_STAGE, OPT_NVTX = 13, 14, 15, 16
MLP_PARAMS = 1313
PREC_FP64, PREC_FP32_RECHECK = 0, 1
SCHED_SIZE, SCHED_NONE, SCHED_LEARNED = 0, 1, 2

# Every symbol the header declares, with its ctypes signature.
_P, _I64, _I32, _D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double


class Stats(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64), ("d", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("key_bits", ctypes.c_int32), ("radix_passes", ctypes.c_int32),
        ("num_cells", ctypes.c_int64), ("num_core_cells", ctypes.c_int64),
        ("num_neighbor_entries", ctypes.c_int64), ("num_candidate_pairs", ctypes.c_int64),
        ("num_pairs_tested", ctypes.c_int64), ("num_pairs_skipped", ctypes.c_int64),
        ("num_pairs_connected", ctypes.c_int64), ("num_pairs_box_decided", ctypes.c_int64),
        ("num_pairs_listed", ctypes.c_int64),
        ("num_core_points", ctypes.c_int64),
        ("num_border_points", ctypes.c_int64), ("num_noise_points", ctypes.c_int64),
        ("num_border_memberships", ctypes.c_int64), ("band_rechecks", ctypes.c_int64),
        ("distance_evals", ctypes.c_int64), ("distance_evals_phase", ctypes.c_int64 * 3), ("band_lo", ctypes.c_float), ("band_hi", ctypes.c_float),
        ("kernel_launches", ctypes.c_int64), ("phase_ms", ctypes.c_float * 9),
        ("markcore_pair_bound", ctypes.c_int64),
        ("schedule_used", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("rho", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        out = {k: getattr(self, k) for k, _ in self._fields_}
        out["phase_ms"] = list(self.phase_ms)
        out["distance_evals_phase"] = list(self.distance_evals_phase)
        return out


class Tuning(ctypes.Structure):
    """dbscan_tuning."""
    _fields_ = [("schedule", ctypes.c_int32), ("cell_bounds", ctypes.c_int32), ("connect_waves", ctypes.c_int32),
                ("connect_cells", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32), ("small_cells", ctypes.c_int32),
                ("pair_boxes", ctypes.c_int32), ("quadtree", ctypes.c_int32),
                ("trials", ctypes.c_int32),
                ("best_ms", ctypes.c_float), ("default_ms", ctypes.c_float)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class Instance(ctypes.Structure):
    _fields_ = [("row0", ctypes.c_int64), ("n", ctypes.c_int64), ("d", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("eps", ctypes.c_double), ("min_pts", ctypes.c_int64)]


class SlabStats(ctypes.Structure):
    """dbscan_slab_stats."""
    _fields_ = [("slabs", ctypes.c_int32), ("axis", ctypes.c_int32), ("max_slab_points", ctypes.c_int64),
                ("halo_points", ctypes.c_int64), ("border_pairs", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("ms", ctypes.c_double * 5)]

    def as_dict(self) -> dict:
        out = {name: getattr(self, name) for name, _ in self._fields_}
        out["ms"] = list(self.ms)
        return out


SIGNATURES = {
    "dbscan_create": (_I32, [ctypes.POINTER(_P), _I64, _I32]),
    "dbscan_destroy": (None, [_P]),
    "dbscan_set_option": (_I32, [_P, _I32, _I64]),
    "dbscan_run": (_I32, [_P, _P, _I64, _I32, _I32, _D, _I64, _P, _P, _P, ctypes.POINTER(_I64), _P]),
    "dbscan_border_ids": (_I32, [_P, _P, _I64, _P]),
    "dbscan_link_witnesses": (_I32, [_P, _P, _P, _I64, ctypes.POINTER(_I64), _P]),
    "dbscan_run_host": (_I32, [_P, _P, _I64, _I32, _I32, _D, _I64, _P, _P, _P, _P, _I64, ctypes.POINTER(_I64), _P]),
    "dbscan_run_batch_host": (_I32, [_P, ctypes.POINTER(Instance), _I32, _P, _I32, _I32, _P, _P, _P, _P, _I64,
                                     ctypes.POINTER(_I64), _P]),
    "dbscan_run_slabs": (_I32, [_P, _P, _I64, _I32, _I32, _D, _I64, _I32, _P, _P, _P, ctypes.POINTER(_I64),
                                ctypes.POINTER(SlabStats), _P]),
    "dbscan_slab_border_ids": (_I32, [_P, _P, _I64, _P]),
    "dbscan_run_static": (_I32, [_P, _I64, _I32, _I32, _D, _I64, _P, _P, _P]),
    "dbscan_run_batch": (_I32, [_P, ctypes.POINTER(Instance), _I32, _P, _I32, _I32, _P, _P, _P,
                                ctypes.POINTER(_I64), _P]),
    "dbscan_get_stats": (_I32, [_P, ctypes.POINTER(Stats)]),
    "dbscan_set_approx": (_I32, [_P, _D]),
    "dbscan_train_scheduler": (_I32, [_P, _I32, _I32, ctypes.c_float, ctypes.c_uint64, _P]),
    "dbscan_scheduler_weights": (_I32, [_P, _P, _I32, _I32]),
    "dbscan_scheduler_loss_grad": (_I32, [_P, _P, _P, _I64, _P, _P]),
    "dbscan_get_pair_log": (_I32, [_P, _P, _P, _I64, ctypes.POINTER(_I64)]),
    "dbscan_get_option": (_I32, [_P, _I32, ctypes.POINTER(_I64)]),
    "dbscan_autotune": (_I32, [_P, _P, _I64, _I32, _I32, ctypes.c_double, _I64, _I32, _P, _P]),
    "dbscan_autotune_batch": (_I32, [_P, ctypes.POINTER(Instance), _I32, _P, _I32, _I32, _I32, _P, _P]),
    "dbscan_status_string": (ctypes.c_char_p, [_I32]),
    "dbscan_version": (_I32, []),
}

_lib = None


def load(path: Path | str | None = None) -> ctypes.CDLL:
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = Path(path) if path else LIB_PATH
    if not p.exists():
        raise RuntimeError(f"CUDA library {p.name} is not built; call paper_1912_06255_gb300.build.build()")
    lib = ctypes.CDLL(str(p))
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


class DbscanError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}")


def check(status: int, where: str) -> None:
    if status != OK:
        raise DbscanError(status, where)
