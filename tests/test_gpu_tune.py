"""Runtime knobs of the persistent kernels and the autotuner on the GPU.

No knob may change the result (it only orders or groups exact tests); the
autotuner keeps the fastest of the settings it timed, starting with the one
the context had.
"""
import numpy as np
import pytest

import oracle
from paper_1912_06255_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1912_06255_gb300 import DBSCAN, DbscanError, _lib  # noqa: E402


def _check(ctx, X, eps, mp):
    r = ctx.run(torch.from_numpy(X).cuda(), eps, mp)
    exp = oracle.dbscan(X, eps, mp)
    assert np.array_equal(r.core.cpu().numpy(), exp[0])
    assert np.array_equal(r.labels.cpu().numpy(), exp[1])
    assert np.array_equal(r.border_offsets.cpu().numpy(), exp[2])
    assert np.array_equal(r.border_ids.cpu().numpy(), exp[3])
    return ctx.stats()


@pytest.mark.parametrize("cells", [1, 2, 4, 8])
@pytest.mark.parametrize("waves", [1, 2])
@pytest.mark.parametrize("blocks", [0, 1, 3])
@pytest.mark.parametrize("small", [0, 1 << 30])
@pytest.mark.parametrize("pair_boxes", [0, 1])
def test_knobs_keep_the_result(cells, waves, blocks, small, pair_boxes):
    X = synth.random_small(55, 15000, 3, dtype=np.float32)
    ctx = DBSCAN(len(X), 3)
    ctx.set_tuning({"connect_cells": cells, "connect_waves": waves, "blocks_per_sm": blocks, "small_cells": small,
                    "pair_boxes": pair_boxes})
    assert ctx.tuning()["connect_cells"] == cells and ctx.tuning()["connect_waves"] == waves
    st = _check(ctx, X, 0.25, 10)
    assert st["num_pairs_tested"] + st["num_pairs_skipped"] + st["num_pairs_box_decided"] == st["num_candidate_pairs"]


def test_knob_validation():
    ctx = DBSCAN(100, 3)
    for opt, bad in ((_lib.OPT_CONNECT_CELLS, 3), (_lib.OPT_CONNECT_WAVES, 0), (_lib.OPT_BLOCKS_PER_SM, -1),
                     (_lib.OPT_BLOCKS_PER_SM, 33), (_lib.OPT_SMALL_CELLS, -1), (_lib.OPT_PAIR_BOXES, 2)):
        with pytest.raises(DbscanError):
            ctx.set_option(opt, bad)
    with pytest.raises(DbscanError):
        ctx.get_option(99)


@pytest.mark.parametrize("d", [3, 6])
def test_autotune_single(d):
    X = synth.random_small(66 + d, 40000, d, dtype=np.float32)
    eps = 0.25 if d == 3 else 0.9
    ctx = DBSCAN(len(X), d)
    t = ctx.autotune(torch.from_numpy(X).cuda(), eps, 10, reps=2)
    assert t["trials"] >= 10 and 0 < t["best_ms"] <= t["default_ms"]
    assert t["connect_cells"] in (1, 2, 4, 8) and t["connect_waves"] in (1, 2) and t["schedule"] in (0, 1, 2)
    assert ctx.tuning() == {k: t[k] for k in ("schedule", "cell_bounds", "connect_waves", "connect_cells",
                                                "blocks_per_sm", "small_cells", "pair_boxes", "quadtree")}
    assert t["quadtree"] in ((0, 2) if d >= 5 else (0,))  # the quadtree knob is tried for d >= 5 only
    _check(ctx, X, eps, 10)


def test_autotune_batch():
    B = synth.batch_256(seed=77, count=12, lo=1e3, hi=3e4)
    N = sum(len(b.points) for b in B)
    P = np.zeros((N, 3), np.float32)
    row = 0
    for b in B:
        P[row:row + len(b.points), :b.points.shape[1]] = b.points
        row += len(b.points)
    inst = [(len(b.points), b.points.shape[1], b.eps, b.min_pts) for b in B]
    ctx = DBSCAN(N, 3)
    X = torch.from_numpy(P).cuda()
    t = ctx.autotune_batch(X, inst, reps=2)
    assert t["trials"] >= 10 and t["best_ms"] <= t["default_ms"]
    r = ctx.run_batch(X, inst)
    core, labels = r.core.cpu().numpy(), r.labels.cpu().numpy()
    row = 0
    for b in B:
        n = len(b.points)
        exp = oracle.dbscan(b.points, b.eps, b.min_pts)
        assert np.array_equal(core[row:row + n], exp[0]) and np.array_equal(labels[row:row + n], exp[1])
        row += n


@pytest.mark.parametrize("d", [2, 4, 6])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("pair_boxes", [0, 1])
def test_small_cells_kernel_all_dims(d, precision, pair_boxes):
    """MarkCore's thread-per-point path on sparse inputs (few points per cell),
    with and without the core-point box decisions."""
    X = synth.random_small(90 + d, 12000, d, dtype=np.float32, clustered=False)
    ctx = DBSCAN(len(X), d, precision=precision)
    ctx.set_tuning({"small_cells": 1 << 30, "pair_boxes": pair_boxes})
    cases = {2: ((0.04, 3), (0.08, 6)), 4: ((0.4, 3), (1.0, 6)), 6: ((1.5, 3), (2.5, 6))}[d]
    for eps, mp in cases:
        _check(ctx, X, eps, mp)


def _twelve_chains():
    """A point p at the origin and 12 chains of 20 points along the icosahedron
    directions: each chain's first point at 0.99 (within eps = 1 of p, and
    1.04 from the next chain's), the rest in [1.05, 1.5].  With minPts 14 the
    chain points are core, p (13 points within eps) is not, and p joins 12
    clusters."""
    phi = (1 + 5 ** 0.5) / 2
    v = []
    for a in (-1, 1):
        for b in (-phi, phi):
            v += [(0, a, b), (a, b, 0), (b, 0, a)]
    v = np.array(v, dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    pts = [np.zeros(3)]
    for u in v:
        pts.append(0.99 * u)
        for r in np.linspace(1.05, 1.5, 19):
            pts.append(r * u)
    return np.array(pts) + 10.0


@pytest.mark.parametrize("small", [0, 1 << 30])
def test_border_point_in_twelve_clusters(small):
    """More clusters per border point than the thread-per-point border kernel
    keeps (8): the point goes to the warp kernel, with the same result."""
    X = _twelve_chains()
    exp = oracle.dbscan(X, 1.0, 14)
    assert exp[0][0] == 0 and exp[2][1] - exp[2][0] == 12  # p is a border point of 12 clusters
    ctx = DBSCAN(len(X), 3, precision="fp64")
    ctx.set_tuning({"small_cells": small})
    _check(ctx, X, 1.0, 14)
