"""CPU oracle for exact Euclidean DBSCAN (Sec. 2 definition, FP64).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The CUDA library never imports or calls
this package, and this package imports nothing from the library.

The arithmetic lives in ``dbscan_oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off`` so that no multiply-add is fused); this module builds it
with gcc, loads it with ctypes and marshals numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "dbscan_oracle.c"
_LIB = _HERE / "_build" / "liboracle.so"
_lib = None


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (OpenMP, -O2, no FP contraction)."""
    if _LIB.exists() and not force and _LIB.stat().st_mtime >= _SRC.stat().st_mtime:
        return _LIB
    _LIB.parent.mkdir(parents=True, exist_ok=True)
    tmp = _LIB.with_suffix(f".so.{os.getpid()}")
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-std=c11", str(_SRC), "-o", str(tmp), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(str(_LIB))
        P = ctypes.c_void_p
        i64, i32 = ctypes.c_int64, ctypes.c_int
        lib.oracle_dbscan.argtypes = [P, i64, i32, ctypes.c_double, i64, i32, P, P, P,
                                      ctypes.POINTER(ctypes.c_void_p)]
        lib.oracle_dbscan.restype = i32
        lib.oracle_sample_counts.argtypes = [P, i64, i32, ctypes.c_double, P, i64, i32, P]
        lib.oracle_sample_counts.restype = i32
        lib.oracle_neighbors.argtypes = [P, i64, i32, ctypes.c_double, i64, P, i64]
        lib.oracle_neighbors.restype = i64
        lib.oracle_within_pairs.argtypes = [P, i64, i32, ctypes.c_double, P, i64, i32, P]
        lib.oracle_within_pairs.restype = i32
        lib.oracle_num_threads.restype = i32
        lib.oracle_free.argtypes = [P]
        _lib = lib
    return _lib


def _as_f64(points) -> np.ndarray:
    X = np.ascontiguousarray(np.asarray(points, dtype=np.float64))
    if X.ndim != 2:
        raise ValueError("points must be [n, d]")
    return X


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def dbscan(points, eps: float, min_pts: int, threads: int = 0):
    """Exact DBSCAN of ``points`` [n, d] (widened exactly to FP64).

    Returns ``(core u8[n], labels i32[n], border_off i64[n+1], border_ids i32[K])``:
    labels name clusters by their smallest core index; a border point's label
    is the smallest name in its set; noise is -1.  ``border_off``/``border_ids``
    hold the sorted sets of the non-core points (core points: empty entry).
    """
    lib = _load()
    X = _as_f64(points)
    n, d = X.shape
    core = np.zeros(n, np.uint8)
    labels = np.zeros(n, np.int32)
    off = np.zeros(n + 1, np.int64)
    ids_ptr = ctypes.c_void_p()
    rc = lib.oracle_dbscan(X.ctypes.data, n, d, float(eps), int(min_pts), int(threads),
                           core.ctypes.data, labels.ctypes.data, off.ctypes.data,
                           ctypes.byref(ids_ptr))
    if rc != 0:
        raise RuntimeError(f"oracle_dbscan failed ({rc})")
    k = int(off[n])
    ids = np.ctypeslib.as_array(ctypes.cast(ids_ptr, ctypes.POINTER(ctypes.c_int32)),
                                shape=(max(k, 1),))[:k].copy()
    lib.oracle_free(ids_ptr)
    return core, labels, off, ids


def sample_counts(points, eps: float, samples, threads: int = 0) -> np.ndarray:
    """|{q : within(p, q)}| for each sampled index p, by a scan over all points."""
    lib = _load()
    X = _as_f64(points)
    s = np.ascontiguousarray(np.asarray(samples, dtype=np.int64))
    out = np.zeros(s.shape[0], np.int64)
    rc = lib.oracle_sample_counts(X.ctypes.data, X.shape[0], X.shape[1], float(eps),
                                  s.ctypes.data, s.shape[0], int(threads), out.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"oracle_sample_counts failed ({rc})")
    return out


def neighbors(points, eps: float, p: int) -> np.ndarray:
    """Indices q (ascending) with within(points[p], q), by a scan over all points."""
    lib = _load()
    X = _as_f64(points)
    cap = 1024
    while True:
        out = np.zeros(cap, np.int64)
        c = lib.oracle_neighbors(X.ctypes.data, X.shape[0], X.shape[1], float(eps), int(p),
                                 out.ctypes.data, cap)
        if c < 0:
            raise RuntimeError("oracle_neighbors: bad arguments")
        if c <= cap:
            return out[:c]
        cap = int(c)


def within_pairs(points, eps: float, pairs, threads: int = 0) -> np.ndarray:
    """within(points[i], points[j]) (Sec. 2, FP64) for each row (i, j) of ``pairs`` [k, 2]."""
    lib = _load()
    X = _as_f64(points)
    pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int64).reshape(-1, 2))
    out = np.zeros(pr.shape[0], np.uint8)
    rc = lib.oracle_within_pairs(X.ctypes.data, X.shape[0], X.shape[1], float(eps), pr.ctypes.data,
                                 pr.shape[0], int(threads), out.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"oracle_within_pairs failed ({rc})")
    return out.astype(bool)
