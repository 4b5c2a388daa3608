"""Repeated runs on one context give the exact result every time.

The cell union-find is lock-free and the points of a cell land in a different
order on every run (the semisort's atomic ranks), so a race in the
connectivity or labelling kernels shows up as a run that differs from the
oracle.  Each case repeats the same input many times and compares every run.
"""
import numpy as np
import pytest

import oracle
from paper_1912_06255_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1912_06255_gb300 import DBSCAN  # noqa: E402


@pytest.mark.parametrize("tuning", [{}, {"connect_waves": 1, "connect_cells": 8, "small_cells": 1 << 30}])
def test_repeated_single_runs(tuning):
    """A 2D blob-and-noise set of 200k points (many cells, many clusters), 12 runs."""
    I = synth.batch_256(seed=31, count=1, lo=2e5, hi=2e5)[0]
    exp = oracle.dbscan(I.points, I.eps, I.min_pts)
    ctx = DBSCAN(len(I.points), 2)
    ctx.set_tuning(tuning)
    X = torch.from_numpy(I.points).cuda()
    for r in range(12):
        res = ctx.run(X, I.eps, I.min_pts)
        assert np.array_equal(res.core.cpu().numpy(), exp[0]), r
        assert np.array_equal(res.labels.cpu().numpy(), exp[1]), r
        assert np.array_equal(res.border_ids.cpu().numpy(), exp[3]), r


def test_repeated_batches():
    """24 instances of the batch family (1e3 to 1e5 points each), 8 replays of the graph."""
    B = synth.batch_256(seed=77, count=24, lo=1e3, hi=1e5)
    n = sum(len(b.points) for b in B)
    P = np.zeros((n, 3), np.float32)
    exp_core, exp_lab = np.zeros(n, np.uint8), np.zeros(n, np.int32)
    row = 0
    for b in B:
        k = len(b.points)
        P[row:row + k, :b.points.shape[1]] = b.points
        e = oracle.dbscan(b.points, b.eps, b.min_pts)
        exp_core[row:row + k], exp_lab[row:row + k] = e[0], e[1]
        row += k
    inst = [(len(b.points), b.points.shape[1], b.eps, b.min_pts) for b in B]
    ctx = DBSCAN(n, 3)
    ctx.set_tuning({"connect_waves": 1, "connect_cells": 8, "small_cells": 1 << 30})
    X = torch.from_numpy(P).cuda()
    for r in range(8):
        res = ctx.run_batch(X, inst)
        assert np.array_equal(res.core.cpu().numpy(), exp_core), r
        assert np.array_equal(res.labels.cpu().numpy(), exp_lab), r
