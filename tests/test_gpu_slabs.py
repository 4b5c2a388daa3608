"""dbscan_run_slabs: one instance run slab by slab with halos and merged.

Every case compares core flags, labels and the border-set CSR with the FP64
oracle on the whole input, element by element: the merge must reproduce the
single-run result exactly, whatever the number of slabs, the input's memory
(pageable host, pinned host, device) and the place of the cuts.  Thin slabs
(halo wider than the slab) and cuts through a point of many clusters are
included; a context too small for any slab must fail cleanly and stay usable.
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

from paper_1912_06255_gb300 import DBSCAN, DbscanError, _lib  # noqa: E402


def _same(r, exp):
    for g, e, what in zip((r.core, r.labels, r.border_offsets, r.border_ids), exp,
                          ("core", "labels", "offsets", "ids")):
        g = g.numpy() if hasattr(g, "numpy") else np.asarray(g)
        assert np.array_equal(g, e), what


def _slabs(X, eps, mp, slabs, max_points=None, precision="fp32", memory="pageable", rho=0.0, stage=1):
    n, d = X.shape
    ctx = DBSCAN(max_points or n, d, precision=precision, rho=rho)
    ctx.set_option(_lib.OPT_SLAB_STAGE, stage)
    try:
        if memory == "pinned":
            pts = torch.from_numpy(X).pin_memory()
        elif memory == "device":
            pts = torch.from_numpy(X).cuda()
        else:
            pts = X
        return ctx.run_slabs(pts, eps, mp, slabs=slabs)
    finally:
        ctx.close()


@pytest.mark.parametrize("slabs", [1, 2, 3, 7, 40])
def test_spreader_3d_slab_counts(slabs):
    I = synth.spreader_3d_2m(n=200_003)
    exp = oracle.dbscan(I.points, I.eps, I.min_pts)
    r, st = _slabs(I.points, I.eps, I.min_pts, slabs)
    _same(r, exp)
    assert st["slabs"] <= slabs and (slabs == 1 or st["slabs"] > 1)
    if slabs > 1:
        assert st["halo_points"] > 0


@pytest.mark.parametrize("memory", ["pageable", "pinned", "device"])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("stage", [1, 0])
def test_input_memory_and_precision(memory, precision, stage):
    """Host input copied to the device once (stage 1) or read in place when
    pinned and staged chunk by chunk when pageable (stage 0)."""
    I = synth.spreader_3d_2m(n=120_001)
    exp = oracle.dbscan(I.points, I.eps, I.min_pts)
    r, _ = _slabs(I.points, I.eps, I.min_pts, 4, precision=precision, memory=memory, stage=stage)
    _same(r, exp)


def test_automatic_slab_count_fits_the_context():
    I = synth.spreader_3d_2m(n=300_007)
    exp = oracle.dbscan(I.points, I.eps, I.min_pts)
    cap = 80_000
    r, st = _slabs(I.points, I.eps, I.min_pts, 0, max_points=cap)
    _same(r, exp)
    assert st["slabs"] >= 4 and st["max_slab_points"] <= cap


def test_thin_slabs_wider_halo():
    """Slabs thinner than the halo (2 eps on each side): each run sees several
    neighbouring slabs whole, still the single-run result."""
    X = synth.random_small(41, 30_000, 2, dtype=np.float64)
    eps, mp = 0.2, 10
    exp = oracle.dbscan(X, eps, mp)
    r, st = _slabs(X, eps, mp, 200)
    _same(r, exp)
    assert st["slabs"] > 50


def test_blobs_2d_fp64():
    I = synth.blobs_2d_20k()
    exp = oracle.dbscan(I.points, I.eps, I.min_pts)
    for s in (2, 5, 13):
        r, _ = _slabs(I.points, I.eps, I.min_pts, s)
        _same(r, exp)


@pytest.mark.parametrize("which", ["5d", "7d"])
def test_high_dimensions(which):
    if which == "5d":
        I = synth.spreader_5d_10m(n=100_000, eps=800.0)
    else:
        I = synth.spreader_7d_10m(n=100_000, eps=1000.0)
    exp = oracle.dbscan(I.points, I.eps, I.min_pts)
    r, st = _slabs(I.points, I.eps, I.min_pts, 3)
    _same(r, exp)
    assert st["slabs"] == 3


def _twelve_chains():
    """A point p at 10 and 12 chains of 20 points along the icosahedron
    directions, the first point of each at 0.99 (within eps = 1 of p, farther
    than eps from the next chain's first point), the rest in [1.05, 1.5]: with
    minPts 14 p is a border point of 12 clusters."""
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


@pytest.mark.parametrize("slabs", [2, 3, 4, 6])
def test_cut_through_a_border_point_of_twelve_clusters(slabs):
    X = _twelve_chains()
    exp = oracle.dbscan(X, 1.0, 14)
    assert exp[2][1] - exp[2][0] == 12
    r, _ = _slabs(X, 1.0, 14, slabs, precision="fp64")
    _same(r, exp)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_lattice_exact_eps(dtype):
    """Axis neighbours at exactly eps, cuts between lattice planes."""
    g = np.stack(np.meshgrid(np.arange(30), np.arange(12), np.arange(5), indexing="ij"), -1).reshape(-1, 3)
    X = (g * 0.75 + 3.0).astype(dtype)
    exp = oracle.dbscan(X, 0.75, 7)
    for s in (2, 5, 9):
        r, _ = _slabs(X, 0.75, 7, s)
        _same(r, exp)


def test_duplicates_and_degenerate_axes():
    """Many copies of few points, and all points sharing their coordinates on
    every axis but one."""
    rng = np.random.default_rng(5)
    X = np.repeat(rng.random((300, 3)) * 10, 7, axis=0)
    X = X[rng.permutation(len(X))]
    exp = oracle.dbscan(X, 0.8, 9)
    r, _ = _slabs(X, 0.8, 9, 6)
    _same(r, exp)
    Y = np.zeros((5000, 3))
    Y[:, 1] = np.sort(rng.random(5000)) * 50
    exp = oracle.dbscan(Y, 0.05, 4)
    r, st = _slabs(Y, 0.05, 4, 8)
    _same(r, exp)
    assert st["axis"] == 1


def test_empty_and_tiny():
    r, st = _slabs(np.zeros((0, 3), np.float32), 1.0, 3, 0, max_points=1)
    assert r.core.numel() == 0 and r.border_offsets.tolist() == [0]
    X = np.array([[0.0, 0.0], [0.5, 0.0], [5.0, 5.0]])
    exp = oracle.dbscan(X, 1.0, 2)
    r, _ = _slabs(X, 1.0, 2, 3)
    _same(r, exp)


def test_context_too_small_fails_cleanly():
    I = synth.spreader_3d_2m(n=50_000)
    ctx = DBSCAN(200, 3)
    try:
        with pytest.raises(DbscanError) as e:
            ctx.run_slabs(I.points, I.eps, I.min_pts, slabs=0)
        assert e.value.status == 5  # DBSCAN_ERR_CAPACITY: no slab count fits 200 points
        with pytest.raises(DbscanError) as e:
            ctx.run_slabs(I.points, I.eps, I.min_pts, slabs=3)
        assert e.value.status == 5
        # the context still runs what fits
        X = synth.random_small(3, 150, 3)
        r = ctx.run(torch.from_numpy(X).cuda(), 0.3, 5)
        exp = oracle.dbscan(X, 0.3, 5)
        assert np.array_equal(r.labels.cpu().numpy(), exp[1])
    finally:
        ctx.close()


def test_rho_approximate_slabs():
    """rho > 0: each slab's answer is a valid approximate answer and so is the
    merge (the core flags stay exact, every merged link is an allowed one)."""
    X = synth.random_small(61, 8000, 2, dtype=np.float32)
    eps, mp, rho = 0.25, 6, 0.2
    r, _ = _slabs(X, eps, mp, 5, rho=rho)
    check_approx(X, eps, mp, rho, r.core.numpy(), r.labels.numpy(), r.border_offsets.numpy(),
                 r.border_ids.numpy())


def test_full_size_3d_against_the_oracle():
    """The 2M-point 3D workload in 4 slabs and with an automatic count for a
    context of a quarter of its size."""
    I = synth.spreader_3d_2m()
    exp = oracle.dbscan(I.points, I.eps, I.min_pts)
    r, st = _slabs(I.points, I.eps, I.min_pts, 4, memory="pinned")
    _same(r, exp)
    r, st = _slabs(I.points, I.eps, I.min_pts, 0, max_points=len(I.points) // 4, memory="pinned", stage=0)
    _same(r, exp)
    assert st["slabs"] >= 5


def test_repeated_calls_reuse_the_context():
    A = synth.spreader_3d_2m(n=100_000, seed=7)
    B = synth.spreader_3d_2m(n=150_000, seed=8)
    ctx = DBSCAN(90_000, 3)
    try:
        for X in (A.points, B.points, A.points):
            r, _ = ctx.run_slabs(X, 100.0, 100, slabs=0)
            _same(r, oracle.dbscan(X, 100.0, 100))
    finally:
        ctx.close()


def test_timeout_and_allocation_failures_leave_the_context_usable():
    """A bounded wait that runs out inside a slab's run, and allocations that
    fail (host-side injection), end the call with their status; the same
    context then gives the exact result."""
    import os
    I = synth.spreader_3d_2m(n=60_000)
    exp = oracle.dbscan(I.points, I.eps, I.min_pts)
    ctx = DBSCAN(30_000, 3)
    try:
        ctx.set_option(_lib.OPT_MAX_ITERS, 1)
        with pytest.raises(DbscanError) as e:
            ctx.run_slabs(I.points, I.eps, I.min_pts, slabs=3)
        assert e.value.status == 7  # DBSCAN_ERR_DEVICE_TIMEOUT
        ctx.set_option(_lib.OPT_MAX_ITERS, 1 << 22)
        r, _ = ctx.run_slabs(I.points, I.eps, I.min_pts, slabs=3)
        _same(r, exp)
    finally:
        ctx.close()
    os.environ["DBSCAN_FAULT"] = "alloc"
    try:
        ctx = DBSCAN(30_000, 3)
    finally:
        del os.environ["DBSCAN_FAULT"]
    try:
        with pytest.raises(DbscanError) as e:
            ctx.run_slabs(I.points, I.eps, I.min_pts, slabs=3)
        assert e.value.status == 3  # DBSCAN_ERR_OOM: the slab buffers are allocated at the first call
        X = synth.random_small(9, 2000, 3, dtype=np.float32)
        r = ctx.run(torch.from_numpy(X).cuda(), 0.3, 8)
        assert np.array_equal(r.labels.cpu().numpy(), oracle.dbscan(X, 0.3, 8)[1])
    finally:
        ctx.close()
