"""Batched runs (many independent instances in one pass) against the oracle.

Each instance of a batch must come out exactly as if clustered alone: core
flags, labels (named by the smallest core index within the instance) and
border sets, bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_1912_06255_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1912_06255_gb300 import DBSCAN, _lib  # noqa: E402
from _certify import check_links  # noqa: E402


def _instances(seed, count, lo, hi, dtype=np.float32):
    """Blob-plus-noise instances like the 256-instance workload, smaller."""
    rng = np.random.default_rng(seed)
    parts, desc = [], []
    for i in range(count):
        d = 2 if i % 2 == 0 else 3
        n = int(round(np.exp(rng.uniform(np.log(lo), np.log(hi))))) if i % 7 else [0, 1, 2][i % 3]
        X = synth.gaussian_blobs(rng, n, d, max(1, n // 300), 10.0 * (n / 2000 + 0.1) ** (1 / d), 1.0, 0.1) \
            if n > 0 else np.zeros((0, d))
        eps = float(rng.uniform(0.2, 1.0))
        mp = int(rng.integers(2, 20))
        pad = np.zeros((n, 3), dtype=np.float64)
        pad[:, :d] = X
        # the unused third column of 2D instances holds garbage on purpose
        if d == 2 and n:
            pad[:, 2] = rng.normal(size=n) * 1e3
        parts.append(pad)
        desc.append((n, d, eps, mp, X))
    return np.concatenate(parts, 0).astype(dtype), desc


def _check(res, desc):
    core = res.core.cpu().numpy()
    labels = res.labels.cpu().numpy()
    off = res.border_offsets.cpu().numpy()
    ids = res.border_ids.cpu().numpy()
    row = 0
    for n, d, eps, mp, X in desc:
        ec, el, eo, ei = oracle.dbscan(X.astype(np.float64) if X.dtype != np.float32 else X, eps, mp)
        sl = slice(row, row + n)
        assert np.array_equal(core[sl], ec), (row, n, d)
        assert np.array_equal(labels[sl], el), (row, n, d)
        got_o = off[row:row + n + 1] - off[row]
        assert np.array_equal(got_o, eo), (row, n, d)
        assert np.array_equal(ids[off[row]:off[row + n]], ei), (row, n, d)
        row += n


@pytest.mark.parametrize("graph", [True, False])
def test_batch_matches_per_instance_oracle(graph):
    P, desc = _instances(11, 40, 30, 6000)
    # the oracle sees each instance's own FP32 coordinates
    desc = [(n, d, eps, mp, P[sum(x[0] for x in desc[:k]):sum(x[0] for x in desc[:k]) + n, :d])
            for k, (n, d, eps, mp, X) in enumerate(desc)]
    ctx = DBSCAN(len(P), 3, graph=graph)
    t = torch.from_numpy(P).cuda()
    inst = [(n, d, eps, mp) for n, d, eps, mp, _ in desc]
    r1 = ctx.run_batch(t, inst)
    _check(r1, desc)
    # a second call replays the captured graph
    r2 = ctx.run_batch(t, inst)
    _check(r2, desc)
    # new coordinates in the same buffer, same graph
    P2 = P.copy()
    P2[:, :2] *= 1.5
    t.copy_(torch.from_numpy(P2))
    desc2 = [(n, d, eps, mp, X * np.array([1.5, 1.5, 1.0][:d], dtype=np.float32)) for n, d, eps, mp, X in desc]
    r3 = ctx.run_batch(t, inst)
    _check(r3, desc2)


def test_batch_fp64_input():
    P, desc = _instances(12, 12, 50, 3000, dtype=np.float64)
    desc = [(n, d, eps, mp, P[sum(x[0] for x in desc[:k]):sum(x[0] for x in desc[:k]) + n, :d])
            for k, (n, d, eps, mp, X) in enumerate(desc)]
    ctx = DBSCAN(len(P), 3)
    r = ctx.run_batch(torch.from_numpy(P).cuda(), [(n, d, eps, mp) for n, d, eps, mp, _ in desc])
    _check(r, desc)
    assert r.stats["precision"] == 0  # FP64 input batches decide in FP64


def test_batch_of_one_equals_single_run():
    I = synth.blobs_2d_20k()
    X = I.points.astype(np.float32)
    ctx = DBSCAN(len(X), 2)
    t = torch.from_numpy(X).cuda()
    a = ctx.run(t, I.eps, I.min_pts)
    b = ctx.run_batch(t, [(len(X), 2, I.eps, I.min_pts)])
    for u, v in ((a.core, b.core), (a.labels, b.labels), (a.border_offsets, b.border_offsets),
                 (a.border_ids, b.border_ids)):
        assert torch.equal(u, v)


@pytest.fixture(scope="module")
def batch_full():
    """The full 256-instance batch (about 36M points) and the oracle run of
    every instance (once)."""
    B = synth.batch_256()
    N = sum(len(b.points) for b in B)
    P = np.zeros((N, 3), np.float32)
    rows, row = [], 0
    for b in B:
        P[row:row + len(b.points), :b.points.shape[1]] = b.points
        rows.append(row)
        row += len(b.points)
    exp = [oracle.dbscan(b.points, b.eps, b.min_pts) for b in B]
    return B, P, rows, exp


def _check_all(B, rows, exp, r, tag):
    core, labels = r.core.cpu().numpy(), r.labels.cpu().numpy()
    off, ids = r.border_offsets.cpu().numpy(), r.border_ids.cpu().numpy()
    for i, b in enumerate(B):
        r0, n = rows[i], len(b.points)
        ec, el, eo, ei = exp[i]
        assert np.array_equal(core[r0:r0 + n], ec), (tag, i)
        assert np.array_equal(labels[r0:r0 + n], el), (tag, i)
        assert np.array_equal(off[r0:r0 + n + 1] - off[r0], eo), (tag, i)
        assert np.array_equal(ids[off[r0]:off[r0 + n]], ei), (tag, i)


# the defaults, the setting the benchmark's autotuner has picked on this family
# (size order, thread-per-point MarkCore and ClusterBorder for all small cells)
# and list order with one wave
BATCH_SETTINGS = {
    "default": {},
    "size-smallcells-all": {"schedule": 0, "small_cells": 1 << 30},
    "list-1wave-8cells-smallcells128": {"schedule": 1, "connect_waves": 1, "connect_cells": 8, "small_cells": 128},
}


@pytest.mark.slow
def test_batch256_full_size_all_instances(batch_full):
    """The full 256-instance batch (one replayed CUDA graph) against the oracle
    run of every instance, element by element, in each setting above, in the
    autotuner's own choice on the held-out batch (seed 2003, 48 instances) as
    the benchmark runs it, and with link certificates."""
    B, P, rows, exp = batch_full
    ctx = DBSCAN(len(P), 3)
    t = torch.from_numpy(P).cuda()
    inst = [(len(b.points), b.points.shape[1], b.eps, b.min_pts) for b in B]
    for tag, setting in BATCH_SETTINGS.items():
        ctx.set_tuning(setting)
        _check_all(B, rows, exp, ctx.run_batch(t, inst), tag)
    H = synth.batch_256(seed=2003, count=48)
    NH = sum(len(b.points) for b in H)
    PH = np.zeros((NH, 3), np.float32)
    row = 0
    for b in H:
        PH[row:row + len(b.points), :b.points.shape[1]] = b.points
        row += len(b.points)
    ctx.set_tuning(BATCH_SETTINGS["default"] | {"schedule": 0, "connect_waves": 2, "connect_cells": 4,
                                                "blocks_per_sm": 0, "small_cells": 0, "pair_boxes": 1})
    choice = ctx.autotune_batch(torch.from_numpy(PH).cuda(),
                                [(len(b.points), b.points.shape[1], b.eps, b.min_pts) for b in H], reps=2)
    ctx.set_option(_lib.OPT_WITNESS, 1)
    r = ctx.run_batch(t, inst)
    _check_all(B, rows, exp, r, f"autotuned {choice}")
    rep, links = ctx.link_witnesses()
    rep, links = rep.cpu().numpy(), links.cpu().numpy()
    # links stay inside their instance; certify every instance on its own rows
    inst_of = np.searchsorted(np.asarray(rows), links[:, 0], side="right") - 1
    assert np.array_equal(inst_of, np.searchsorted(np.asarray(rows), links[:, 1], side="right") - 1)
    for i, b in enumerate(B):
        r0, n = rows[i], len(b.points)
        rr = rep[r0:r0 + n].astype(np.int64)
        rr[rr >= 0] -= r0
        check_links(b.points, b.eps, exp[i][0], exp[i][1], rr, links[inst_of == i].astype(np.int64) - r0)


def test_batch_key_width_of_lower_dimensional_instances():
    """A 2D instance inside a 3D batch interleaves three coordinates into its
    cell key (the third is zero), so it needs 3 x bits key bits: 2^19 cells in
    a dimension fit beside the instance id, 2^22 do not (KEY_OVERFLOW instead
    of a key that runs into the instance bits)."""
    from paper_1912_06255_gb300 import DbscanError
    small = synth.random_small(5, 500, 3, dtype=np.float32)
    for far, ok in ((3.0e5, True), (1.5e6, False)):
        wide = np.array([[0.0, 0.0], [far, 0.0], [0.1, 0.1], [far, 0.3]], np.float32)
        P = np.zeros((len(small) + len(wide), 3), np.float32)
        P[:len(small)] = small
        P[len(small):, :2] = wide
        ctx = DBSCAN(len(P), 3)
        inst = [(len(small), 3, 0.3, 5), (len(wide), 2, 1.0, 2)]
        if not ok:
            with pytest.raises(DbscanError) as e:
                ctx.run_batch(torch.from_numpy(P).cuda(), inst)
            assert e.value.status == 4
            continue
        r = ctx.run_batch(torch.from_numpy(P).cuda(), inst)
        ec, el, _, _ = oracle.dbscan(wide, 1.0, 2)
        assert np.array_equal(r.core.cpu().numpy()[len(small):], ec)
        assert np.array_equal(r.labels.cpu().numpy()[len(small):], el)
        ec, el, _, _ = oracle.dbscan(small, 0.3, 5)
        assert np.array_equal(r.labels.cpu().numpy()[:len(small)], el)
