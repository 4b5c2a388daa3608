"""A persistent table of autotuned settings, keyed by workload shape.

``DBSCAN.autotune`` / ``autotune_batch`` search the settings on the GPU (the
search itself is in the library); this module stores their choices so later
runs of the same kind of workload start from them: the key is the kind
(single run or batch), the dimension, the point count rounded up to a power
of two, the element type and the precision mode.
"""
from __future__ import annotations

import json
import math
import os
from pathlib import Path

FIELDS = ("schedule", "cell_bounds", "connect_waves", "connect_cells", "blocks_per_sm", "small_cells",
          "pair_boxes")


def key(kind: str, n: int, d: int, dtype: str, precision: str) -> str:
    if kind not in ("single", "batch"):
        raise ValueError("kind is 'single' or 'batch'")
    bucket = max(0, math.ceil(math.log2(max(int(n), 1))))
    return f"{kind}/d{int(d)}/n2^{bucket}/{dtype}/{precision}"


def load(path) -> dict:
    p = Path(path)
    if not p.exists():
        return {}
    with open(p) as f:
        table = json.load(f)
    return {k: {f: int(v[f]) for f in FIELDS if f in v} for k, v in table.items()}


def save(path, table: dict) -> None:
    p = Path(path)
    tmp = p.with_suffix(p.suffix + f".{os.getpid()}")
    with open(tmp, "w") as f:
        json.dump({k: {f: int(v[f]) for f in FIELDS if f in v} for k, v in sorted(table.items())}, f, indent=1)
    os.replace(tmp, p)


def record(table: dict, k: str, choice: dict) -> dict:
    table[k] = {f: int(choice[f]) for f in FIELDS}
    return table


def lookup(table: dict, k: str) -> dict | None:
    return table.get(k)
