"""Parity of the CUDA library with the CPU oracle, element by element.

Every case compares core flags, labels and the border-set CSR bit for bit
(the result of exact DBSCAN is unique, Sec. 2, and both sides name clusters by
their smallest core index).  Inputs are seeded; the oracle runs on the CPU.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1912_06255_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1912_06255_gb300 import DBSCAN, DbscanError, _lib, dbscan  # noqa: E402
from _certify import check_links  # noqa: E402


def _run(X, eps, mp, **kw):
    t = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    r = dbscan(t, eps, mp, **kw)
    torch.cuda.synchronize()
    return (r.core.cpu().numpy(), r.labels.cpu().numpy(), r.border_offsets.cpu().numpy(),
            r.border_ids.cpu().numpy(), r.stats)


def _assert_same(X, eps, mp, **kw):
    got = _run(X, eps, mp, **kw)
    exp = oracle.dbscan(X, eps, mp)
    names = ("core", "labels", "border_offsets", "border_ids")
    for name, g, e in zip(names, got[:4], exp):
        if not np.array_equal(g, e):
            bad = np.flatnonzero(g != e)[:10] if g.shape == e.shape else "shape"
            raise AssertionError(f"{name} differs at {bad} (n={len(X)}, eps={eps}, minPts={mp}, {kw})")
    return got[4]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_hand_example(precision, dtype):
    import json, os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "two_plus_2d.json")))
    X = np.array(g["points"], dtype=dtype)
    core, labels, off, ids, _ = _run(X, g["eps"], g["min_pts"], precision=precision)
    assert core.tolist() == g["core"] and labels.tolist() == g["labels"]
    sets = [ids[off[i]:off[i + 1]].tolist() for i in range(len(X))]
    assert sets == g["border_sets"]


@pytest.mark.parametrize("d", [1, 2, 3, 4])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_lattice_exact_eps(d, precision, dtype):
    """Every axis neighbour sits at exactly eps: the FP32 band must send those
    pairs to the FP64 recheck and keep them."""
    L = {1: 40, 2: 12, 3: 7, 4: 5}[d]
    grid = np.stack(np.meshgrid(*[np.arange(L)] * d, indexing="ij"), -1).reshape(-1, d)
    X = (grid * 0.75 + 3.0).astype(dtype)
    st = _assert_same(X, 0.75, 2 * d + 1, precision=precision)
    if precision == "fp32":
        assert st["band_rechecks"] > 0


@pytest.mark.parametrize("d", [1, 2, 3, 4])
@pytest.mark.parametrize("seed", [0, 1])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_random_mixed(d, seed, precision, dtype):
    X = synth.random_small(300 + 10 * seed + d, 5000 + 777 * seed, d, dtype=dtype)
    for eps, mp in ((0.15, 4), (0.3, 12), (0.6, 40)):
        _assert_same(X, eps, mp, precision=precision)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_dyadic_translation(precision, dtype):
    """Points on a 2^-4 grid, moved by multiples of 2^10: the coordinates stay
    exact in both storage types, so every run matches the oracle (and each
    other); larger coordinates widen the FP32 band for FP64 input."""
    rng = np.random.default_rng(17)
    X = rng.integers(0, 400, (6000, 3)).astype(np.float64) / 16.0  # 2k core, 300 clusters, 2k noise
    for t in (0.0, 1024.0, -3072.0):
        _assert_same((X + t).astype(dtype), 1.25, 5, precision=precision)


@pytest.mark.parametrize("cell_bounds", [True, False])
@pytest.mark.parametrize("schedule", ["size", "none"])
def test_schedules_agree(schedule, cell_bounds):
    X = synth.random_small(77, 20000, 3, dtype=np.float32)
    st = _assert_same(X, 0.25, 10, schedule=schedule, cell_bounds=cell_bounds)
    assert (st["num_pairs_tested"] + st["num_pairs_skipped"] + st["num_pairs_box_decided"]
            == st["num_candidate_pairs"])
    if not cell_bounds:
        assert st["num_pairs_box_decided"] == 0


@pytest.mark.parametrize("d", [2, 3, 4])
def test_cell_bounds_off_matches(d):
    """Point-by-point tests without the box shortcuts give the same result."""
    X = synth.random_small(500 + d, 6000, d, dtype=np.float32)
    for eps, mp in ((0.2, 5), (0.5, 30)):
        _assert_same(X, eps, mp, cell_bounds=False)


def test_blobs_2d_20k_fp64():
    """Gaussian blobs in 2D, FP64 input, eps 0.5, minPts 10."""
    I = synth.blobs_2d_20k()
    for precision in ("fp64", "fp32"):
        _assert_same(I.points, I.eps, I.min_pts, precision=precision)


def test_spreader_3d_scaled():
    """The 3D seed-spreader workload at 1/10 size (several tiles, ragged tail)."""
    I = synth.spreader_3d_2m(n=200_003)
    st = _assert_same(I.points, I.eps, I.min_pts)
    assert st["num_cells"] > 1000 and st["num_pairs_tested"] > 0


@pytest.fixture(scope="module")
def c1_full():
    """The full 2,000,000-point 3D workload and its full oracle run (once)."""
    I = synth.spreader_3d_2m()
    return I, oracle.dbscan(I.points, I.eps, I.min_pts)


def _check_full(ctx, I, exp, tag):
    r = ctx.run(torch.from_numpy(I.points).cuda(), I.eps, I.min_pts, border=True)
    torch.cuda.synchronize()
    for name, g, e in zip(("core", "labels", "border_offsets", "border_ids"),
                          (r.core, r.labels, r.border_offsets, r.border_ids), exp):
        g = g.cpu().numpy()
        if not np.array_equal(g, e):
            bad = np.flatnonzero(g != e)[:10] if g.shape == e.shape else "shape"
            raise AssertionError(f"{tag}: {name} differs at {bad}")
    return r


# Settings the benchmark's autotuner has chosen on this workload (list order, one
# wave, 8 cells per work item), the defaults, and the other corners of the knobs.
C1_SETTINGS = {
    "default": {},
    "list-1wave-8cells": {"schedule": 1, "connect_waves": 1, "connect_cells": 8},
    "list-2waves-4cells": {"schedule": 1, "connect_waves": 2, "connect_cells": 4},
    "size-1wave-1cell-2bps": {"schedule": 0, "connect_waves": 1, "connect_cells": 1, "blocks_per_sm": 2},
    "small-cells-no-pairboxes": {"small_cells": 1 << 30, "pair_boxes": 0},
    "no-cell-bounds": {"cell_bounds": 0},
}


@pytest.mark.slow
@pytest.mark.parametrize("setting", sorted(C1_SETTINGS))
def test_spreader_3d_full_size(c1_full, setting):
    """The full 2,000,000-point 3D workload (FP32 input, FP32 band + FP64
    recheck) against the full oracle run, in each setting the benchmark can
    time."""
    I, exp = c1_full
    ctx = DBSCAN(len(I.points), 3)
    ctx.set_tuning(C1_SETTINGS[setting])
    _check_full(ctx, I, exp, setting)


@pytest.mark.slow
def test_spreader_3d_full_size_as_benchmarked(c1_full):
    """The benchmark's own procedure on the full 3D workload: log and train the
    pair scheduler on the held-out input (seed 2001), autotune there, then run
    the chosen setting and the learned schedule on the timed input; both
    against the full oracle run, the learned one with its link certificate."""
    I, exp = c1_full
    H = synth.spreader_3d_2m(seed=2001)
    ctx = DBSCAN(len(I.points), 3)
    ctx.enable_pair_log(1 << 24)
    ctx.run(torch.from_numpy(H.points).cuda(), H.eps, H.min_pts, border=False)
    ctx.train_scheduler(epochs=30, batch=4096, lr=3e-3, seed=1)
    ctx.enable_pair_log(0)
    choice = ctx.autotune(torch.from_numpy(H.points).cuda(), H.eps, H.min_pts, reps=2)
    _check_full(ctx, I, exp, f"autotuned {choice}")
    ctx.set_option(1, 2)  # the learned schedule
    ctx.set_option(_lib.OPT_WITNESS, 1)
    r = _check_full(ctx, I, exp, "learned")
    rep, links = ctx.link_witnesses()
    check_links(I.points, I.eps, exp[0], exp[1], rep.cpu().numpy(), links.cpu().numpy(),
                num_core_cells=r.stats["num_core_cells"])


def test_edge_cases():
    rng = np.random.default_rng(5)
    # empty
    ctx = DBSCAN(100, 3)
    r = ctx.run(torch.zeros((0, 3), device="cuda"), 1.0, 3)
    assert r.core.numel() == 0 and r.border_offsets.cpu().tolist() == [0]
    # one point
    _assert_same(np.array([[1.0, 2.0]]), 0.5, 1)
    _assert_same(np.array([[1.0, 2.0]]), 0.5, 2)
    # all identical
    _assert_same(np.full((500, 3), 7.5, np.float32), 0.1, 500)
    _assert_same(np.full((500, 3), 7.5, np.float32), 0.1, 501)
    # minPts = 1 (every point core) and minPts > n (all noise)
    X = rng.random((3000, 2))
    _assert_same(X, 0.02, 1)
    _assert_same(X, 0.02, 4000)
    # eps above the diameter: one cell, one cluster
    _assert_same(X.astype(np.float32), 5.0, 100)
    # negative and large coordinates, ragged size
    Y = (rng.standard_normal((4099, 3)) * 1e4 - 5e4).astype(np.float32)
    _assert_same(Y, 900.0, 5)


def test_host_entry_point_matches_device():
    """dbscan_run_host from pinned host buffers, with and without the border
    sets (a too small ids buffer reports CAPACITY and the needed length), and
    dbscan_run_batch_host on two instances."""
    X = synth.random_small(8, 10000, 3, dtype=np.float32)
    ctx = DBSCAN(len(X), 3)
    pinned = torch.from_numpy(X).pin_memory()
    exp = oracle.dbscan(X, 0.3, 8)
    core, labels, k = ctx.run_host(pinned, 0.3, 8, core=torch.empty(len(X), dtype=torch.uint8).pin_memory(),
                                   labels=torch.empty(len(X), dtype=torch.int32).pin_memory())
    assert np.array_equal(core.numpy(), exp[0]) and np.array_equal(labels.numpy(), exp[1])
    assert k == len(exp[3]) > 0
    off = torch.empty(len(X) + 1, dtype=torch.int64).pin_memory()
    with pytest.raises(DbscanError) as e:
        ctx.run_host(pinned, 0.3, 8, border=(off, torch.empty(k - 1, dtype=torch.int32)))
    assert e.value.status == 5
    ids = torch.empty(k, dtype=torch.int32).pin_memory()
    core, labels, k2 = ctx.run_host(pinned, 0.3, 8, border=(off, ids))
    assert k2 == k and np.array_equal(off.numpy(), exp[2]) and np.array_equal(ids.numpy(), exp[3])
    assert np.array_equal(labels.numpy(), exp[1])
    # the batch form
    Y = synth.random_small(9, 4000, 2, dtype=np.float32)
    P = np.zeros((len(X) + len(Y), 3), np.float32)
    P[:len(X)] = X
    P[len(X):, :2] = Y
    bctx = DBSCAN(len(P), 3)
    boff = torch.empty(len(P) + 1, dtype=torch.int64)
    bids = torch.empty(4 * len(P), dtype=torch.int32)
    core, labels, kb = bctx.run_batch_host(P, [(len(X), 3, 0.3, 8), (len(Y), 2, 0.2, 5)], border=(boff, bids))
    ey = oracle.dbscan(Y, 0.2, 5)
    assert np.array_equal(labels.numpy()[:len(X)], exp[1]) and np.array_equal(labels.numpy()[len(X):], ey[1])
    assert kb == len(exp[3]) + len(ey[3])
    o = boff.numpy()
    assert np.array_equal(bids.numpy()[o[len(X)]:o[-1]], ey[3])


def test_invalid_arguments():
    ctx = DBSCAN(1000, 3)
    X = torch.zeros((10, 3), device="cuda")
    with pytest.raises(DbscanError) as e:
        ctx.run(X, -1.0, 3)
    assert e.value.status == 1
    with pytest.raises(DbscanError) as e:
        ctx.run(X, float("nan"), 3)
    assert e.value.status == 1
    with pytest.raises(DbscanError) as e:
        ctx.run(X, 1.0, 0)
    assert e.value.status == 1
    Xn = X.clone()
    Xn[3, 1] = float("nan")
    with pytest.raises(DbscanError) as e:
        ctx.run(Xn, 1.0, 3)
    assert e.value.status == 1
    Xi = X.clone()
    Xi[4, 0] = float("inf")
    with pytest.raises(DbscanError) as e:
        ctx.run(Xi, 1.0, 3)
    assert e.value.status == 1
    with pytest.raises(DbscanError) as e:
        ctx.run(torch.zeros((2000, 3), device="cuda"), 1.0, 3)
    assert e.value.status == 1
    with pytest.raises(DbscanError) as e:
        ctx.run(torch.zeros((10, 4), device="cuda"), 1.0, 3)
    assert e.value.status == 2
    # a grid wider than 2^30 cells in one dimension
    Xw = torch.tensor([[0.0, 0.0, 0.0], [1e12, 0.0, 0.0]], device="cuda", dtype=torch.float64)
    with pytest.raises(DbscanError) as e:
        ctx.run(Xw, 1e-3, 2)
    assert e.value.status == 4
    # the context stays usable after errors
    _ = ctx.run(torch.rand((500, 3), device="cuda"), 0.2, 3)


def test_context_reuse_and_determinism():
    X = synth.random_small(21, 8000, 2, dtype=np.float32)
    ctx = DBSCAN(len(X), 2)
    t = torch.from_numpy(X).cuda()
    a = ctx.run(t, 0.2, 6)
    b = ctx.run(t, 0.2, 6)
    for u, v in ((a.core, b.core), (a.labels, b.labels), (a.border_offsets, b.border_offsets),
                 (a.border_ids, b.border_ids)):
        assert torch.equal(u, v)
    c = ctx.run(t[:5000], 0.35, 9)
    exp = oracle.dbscan(X[:5000], 0.35, 9)
    assert np.array_equal(c.labels.cpu().numpy(), exp[1])


def test_border_ids_without_offsets_in_the_run():
    """A run that skips the border offsets still serves dbscan_border_ids (the
    offsets are scanned on demand) and reports the total set length."""
    import ctypes
    X = synth.random_small(33, 12000, 2, dtype=np.float32)
    eps, mp = 0.12, 6
    ctx = DBSCAN(len(X), 2)
    r = ctx.run(torch.from_numpy(X).cuda(), eps, mp, border=False)
    exp = oracle.dbscan(X, eps, mp)
    K = ctx.stats()["num_border_memberships"]
    assert K == len(exp[3]) and K > 0
    ids = torch.empty(K, dtype=torch.int32, device="cuda")
    st = ctx.lib.dbscan_border_ids(ctx.ctx, ids.data_ptr(), K, torch.cuda.current_stream().cuda_stream)
    assert st == 0
    assert np.array_equal(ids.cpu().numpy(), exp[3])
    assert np.array_equal(r.labels.cpu().numpy(), exp[1])


@pytest.mark.parametrize("schedule", ["size", "none", "learned"])
@pytest.mark.parametrize("cell_bounds", [True, False])
@pytest.mark.parametrize("d", [2, 3, 6])
def test_link_witnesses(schedule, cell_bounds, d):
    """Every union the run makes is recorded with a pair of core points within
    eps; with the cell representatives they certify each cluster as one
    connected graph of verified eps-edges, and the run still matches the
    oracle with the recording on."""
    X = synth.random_small(60 + d, 8000, d, dtype=np.float32)
    eps, mp = {2: (0.2, 6), 3: (0.3, 8), 6: (0.9, 10)}[d]
    ctx = DBSCAN(len(X), d, schedule=schedule, cell_bounds=cell_bounds)
    ctx.set_option(_lib.OPT_WITNESS, 1)
    r = ctx.run(torch.from_numpy(X).cuda(), eps, mp)
    exp = oracle.dbscan(X, eps, mp)
    assert np.array_equal(r.core.cpu().numpy(), exp[0]) and np.array_equal(r.labels.cpu().numpy(), exp[1])
    rep, links = ctx.link_witnesses()
    ncl = check_links(X, eps, exp[0], exp[1], rep.cpu().numpy(), links.cpu().numpy(),
                      num_core_cells=r.stats["num_core_cells"])
    assert ncl > 1
    # without the option there is nothing to export
    ctx.set_option(_lib.OPT_WITNESS, 0)
    ctx.run(torch.from_numpy(X).cuda(), eps, mp)
    with pytest.raises(DbscanError) as e:
        ctx.link_witnesses()
    assert e.value.status == 8


def test_nvtx_ranges_change_nothing():
    """NVTX phase ranges (host calls only) leave every output as it was, also
    after a failed run left a range open, and in the slab path."""
    X = synth.random_small(77, 6000, 3, dtype=np.float32)
    exp = oracle.dbscan(X, 0.3, 8)
    ctx = DBSCAN(len(X), 3)
    ctx.set_option(_lib.OPT_NVTX, 1)
    assert ctx.get_option(_lib.OPT_NVTX) == 1
    t = torch.from_numpy(X).cuda()
    ctx.set_option(_lib.OPT_MAX_ITERS, 1)
    with pytest.raises(DbscanError):
        ctx.run(t, 0.3, 8)
    ctx.set_option(_lib.OPT_MAX_ITERS, 1 << 22)
    for _ in range(2):
        r = ctx.run(t, 0.3, 8)
        for g, e in zip((r.core, r.labels, r.border_offsets, r.border_ids), exp):
            assert np.array_equal(g.cpu().numpy(), e)
    r, _ = ctx.run_slabs(X, 0.3, 8, slabs=3)
    for g, e in zip((r.core, r.labels, r.border_offsets, r.border_ids), exp):
        assert np.array_equal(g.numpy(), e)
    ctx.close()
