"""Host logic of the tuning table (no GPU)."""
from paper_1912_06255_gb300 import tuning


def test_key_buckets():
    assert tuning.key("single", 2_000_000, 3, "f32", "fp32") == "single/d3/n2^21/f32/fp32"
    assert tuning.key("single", 2 ** 21, 3, "f32", "fp32") == "single/d3/n2^21/f32/fp32"
    assert tuning.key("single", 2 ** 21 + 1, 3, "f32", "fp32") == "single/d3/n2^22/f32/fp32"
    assert tuning.key("batch", 1, 2, "f64", "fp64") == "batch/d2/n2^0/f64/fp64"


def test_roundtrip(tmp_path):
    t = {}
    choice = {"schedule": 1, "cell_bounds": 1, "connect_waves": 2, "connect_cells": 8, "blocks_per_sm": 0,
              "small_cells": 128, "pair_boxes": 0, "trials": 11, "best_ms": 1.5}
    k = tuning.key("single", 1000, 5, "f32", "fp32")
    tuning.record(t, k, choice)
    p = tmp_path / "tune.json"
    tuning.save(p, t)
    back = tuning.load(p)
    assert back == {k: {f: choice[f] for f in tuning.FIELDS}}
    assert tuning.lookup(back, k)["connect_cells"] == 8
    assert tuning.lookup(back, "missing") is None
    assert tuning.load(tmp_path / "absent.json") == {}
