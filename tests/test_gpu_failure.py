"""Failure paths on the GPU, made without faulting it.

A bounded device wait is made to run out by lowering DBSCAN_OPT_MAX_ITERS to 1:
every union-find walk longer than one step gives up (so do look-backs of the
key sort that find a tile unpublished).  The run must report
DBSCAN_ERR_DEVICE_TIMEOUT, every later kernel must leave at entry instead of
using the incomplete data, and the next run on the same context, with the
limit restored, must match the oracle.  Allocation failures are injected on
the host (DBSCAN_FAULT=alloc): the calls that need a new buffer return
DBSCAN_ERR_OOM and the context keeps working for the rest.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1912_06255_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1912_06255_gb300 import DBSCAN, DbscanError, _lib  # noqa: E402


def _same(r, exp):
    for g, e in zip((r.core, r.labels, r.border_offsets, r.border_ids), exp):
        assert np.array_equal(g.cpu().numpy(), e)


@pytest.mark.parametrize("which", ["3d", "2d-fp64", "5d", "7d"])
def test_timeout_is_reported_and_the_context_recovers(which):
    if which == "3d":
        I = synth.spreader_3d_2m(n=200_003)
        X, eps, mp, d = I.points, I.eps, I.min_pts, 3
    elif which == "2d-fp64":
        I = synth.blobs_2d_20k()
        X, eps, mp, d = I.points, I.eps, I.min_pts, 2
    elif which == "5d":
        I = synth.spreader_5d_10m(n=100_000, eps=800.0)
        X, eps, mp, d = I.points, I.eps, I.min_pts, 5
    else:
        I = synth.spreader_7d_10m(n=100_000, eps=1000.0)
        X, eps, mp, d = I.points, I.eps, I.min_pts, 7
    exp = oracle.dbscan(X, eps, mp)
    t = torch.from_numpy(X).cuda()
    ctx = DBSCAN(len(X), d)
    _same(ctx.run(t, eps, mp), exp)
    ctx.set_option(_lib.OPT_MAX_ITERS, 1)
    for _ in range(2):
        with pytest.raises(DbscanError) as e:
            ctx.run(t, eps, mp)
        assert e.value.status == 7  # DBSCAN_ERR_DEVICE_TIMEOUT
    ctx.set_option(_lib.OPT_MAX_ITERS, 1 << 22)
    _same(ctx.run(t, eps, mp), exp)
    _same(ctx.run(t, eps, mp), exp)


def test_timeout_in_a_batch_graph():
    parts = [synth.spreader_3d_2m(n=60_000 + 7 * k, seed=1001 + k).points for k in range(3)]
    P = np.concatenate(parts).astype(np.float32)
    inst = [(len(q), 3, 100.0, 100) for q in parts]
    ctx = DBSCAN(len(P), 3)
    t = torch.from_numpy(P).cuda()
    r = ctx.run_batch(t, inst)
    ctx.set_option(_lib.OPT_MAX_ITERS, 1)
    with pytest.raises(DbscanError) as e:
        ctx.run_batch(t, inst)
    assert e.value.status == 7
    ctx.set_option(_lib.OPT_MAX_ITERS, 1 << 22)
    r2 = ctx.run_batch(t, inst)
    row = 0
    for q in parts:
        ec, el, _, _ = oracle.dbscan(q, 100.0, 100)
        assert np.array_equal(r2.core.cpu().numpy()[row:row + len(q)], ec)
        assert np.array_equal(r2.labels.cpu().numpy()[row:row + len(q)], el)
        row += len(q)
    assert torch.equal(r.labels, r2.labels)


def test_injected_allocation_failures():
    X3 = synth.random_small(3, 4000, 3, dtype=np.float32)
    X5 = synth.random_small(5, 4000, 5, dtype=np.float32)
    os.environ["DBSCAN_FAULT"] = "alloc"
    try:
        ctx = DBSCAN(len(X3), 5)  # the workspace itself is allocated at creation
    finally:
        del os.environ["DBSCAN_FAULT"]
    exp3 = oracle.dbscan(X3, 0.3, 8)
    _same(ctx.run(torch.from_numpy(X3).cuda(), 0.3, 8), exp3)
    with pytest.raises(DbscanError) as e:  # the tree buffers of d >= 5 are allocated at the first such run
        ctx.run(torch.from_numpy(X5).cuda(), 0.8, 8)
    assert e.value.status == 3
    with pytest.raises(DbscanError) as e:
        ctx.run_host(X3, 0.3, 8)
    assert e.value.status == 3
    with pytest.raises(DbscanError) as e:
        ctx.set_option(_lib.OPT_WITNESS, 1)
    assert e.value.status == 3
    with pytest.raises(DbscanError) as e:
        ctx.set_option(1, 2)  # the learned schedule's pair list
        ctx.run(torch.from_numpy(X3).cuda(), 0.3, 8)
    assert e.value.status == 3
    ctx.set_option(1, 0)
    _same(ctx.run(torch.from_numpy(X3).cuda(), 0.3, 8), exp3)  # still usable
    os.environ["DBSCAN_FAULT"] = "create"
    try:
        with pytest.raises(DbscanError) as e:
            DBSCAN(100, 3)
        assert e.value.status == 3
    finally:
        del os.environ["DBSCAN_FAULT"]
