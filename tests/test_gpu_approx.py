"""rho-approximate DBSCAN (Sec. 2, after Gan and Tao) on the GPU.

The approximate problem has many valid answers, so each GPU result is checked
by ``oracle.approx.check_approx``: exact core flags, every eps-connected group
of core points inside one cluster, every cluster connected within eps(1+rho),
canonical names and exact border sets.  rho = 0 must reproduce the exact
oracle bit for bit, and a gap between eps and eps(1+rho) must be bridged.
"""
import numpy as np
import pytest

import oracle
from oracle.approx import check_approx
from paper_1912_06255_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1912_06255_gb300 import DBSCAN, DbscanError, dbscan  # noqa: E402


def _run(X, eps, mp, rho, **kw):
    r = dbscan(torch.from_numpy(np.ascontiguousarray(X)).cuda(), eps, mp, rho=rho, **kw)
    torch.cuda.synchronize()
    return (r.core.cpu().numpy(), r.labels.cpu().numpy(), r.border_offsets.cpu().numpy(),
            r.border_ids.cpu().numpy(), r.stats)


@pytest.mark.parametrize("d", [2, 3, 5])
@pytest.mark.parametrize("rho", [0.0, 0.01, 0.1, 0.5])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_random_inputs_are_valid(d, rho, precision):
    X = synth.random_small(400 + d, 2000, d, dtype=np.float32)
    for eps, mp in ((0.25 if d < 5 else 0.7, 5), (0.4 if d < 5 else 1.0, 15)):
        core, labels, off, ids, st = _run(X, eps, mp, rho, precision=precision)
        assert st["rho"] == rho
        check_approx(X, eps, mp, rho, core, labels, off, ids)
        if rho == 0.0:
            exp = oracle.dbscan(X, eps, mp)
            for g, e in zip((core, labels, off, ids), exp):
                assert np.array_equal(g, e)


@pytest.mark.parametrize("schedule", ["size", "none", "learned"])
@pytest.mark.parametrize("cell_bounds", [True, False])
def test_schedules_and_boxes(schedule, cell_bounds):
    X = synth.random_small(77, 3000, 3, dtype=np.float32)
    core, labels, off, ids, _ = _run(X, 0.3, 8, 0.2, schedule=schedule, cell_bounds=cell_bounds)
    check_approx(X, 0.3, 8, 0.2, core, labels, off, ids)


def _two_blobs(gap, d=2):
    """Two lines of core points along x whose closest pair is `gap` apart."""
    t = np.arange(40) * 0.1
    a = np.zeros((40, d))
    a[:, 0] = t
    b = a.copy()
    b[:, 0] += t[-1] + gap
    return np.concatenate([a, b])


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_gap_inside_the_relaxation_is_bridged(dtype):
    """Core points 1.05 eps apart: two clusters exactly, one with rho = 0.1,
    two again with rho = 0.01 (the gap is beyond eps(1 + rho))."""
    X = _two_blobs(1.05).astype(dtype)
    eps, mp = 1.0, 5
    exact = _run(X, eps, mp, 0.0)
    assert len(np.unique(exact[1])) == 2
    wide = _run(X, eps, mp, 0.1)
    check_approx(X, eps, mp, 0.1, *wide[:4])
    assert len(np.unique(wide[1])) == 1
    narrow = _run(X, eps, mp, 0.01)
    assert np.array_equal(narrow[1], exact[1])


def test_lattice_exact_eps_approx():
    """Axis neighbours at exactly eps and diagonals at sqrt(2) eps: with
    rho = 0.5 the diagonals of the interior are within eps(1 + rho)."""
    g = np.stack(np.meshgrid(np.arange(9), np.arange(9), indexing="ij"), -1).reshape(-1, 2) * 0.75
    X = g.astype(np.float32)
    for rho in (0.0, 0.5):
        core, labels, off, ids, st = _run(X, 0.75, 5, rho)
        check_approx(X, 0.75, 5, rho, core, labels, off, ids)
        assert st["band_rechecks"] > 0


def test_batch_approx():
    parts = [synth.random_small(31 + k, 1500 + 400 * k, 2 + k % 2, dtype=np.float32) for k in range(4)]
    params = [(0.25, 6), (0.3, 8), (0.2, 4), (0.35, 10)]
    P = np.zeros((sum(len(q) for q in parts), 3), np.float32)
    row = 0
    for q in parts:
        P[row:row + len(q), :q.shape[1]] = q
        row += len(q)
    ctx = DBSCAN(len(P), 3, rho=0.15)
    r = ctx.run_batch(torch.from_numpy(P).cuda(), [(len(q), q.shape[1], e, m) for q, (e, m) in zip(parts, params)])
    core, labels = r.core.cpu().numpy(), r.labels.cpu().numpy()
    off, ids = r.border_offsets.cpu().numpy(), r.border_ids.cpu().numpy()
    row = 0
    for q, (e, m) in zip(parts, params):
        n = len(q)
        check_approx(q, e, m, 0.15, core[row:row + n], labels[row:row + n],
                     off[row:row + n + 1] - off[row], ids[off[row]:off[row + n]])
        row += n


def test_invalid_rho():
    ctx = DBSCAN(100, 2)
    for bad in (-0.1, float("nan"), float("inf")):
        with pytest.raises(DbscanError) as e:
            ctx.set_approx(bad)
        assert e.value.status == 1
