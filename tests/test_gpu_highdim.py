"""Parity for 5 <= d <= 8 (cells by 128-bit key sort, neighbours by the tree
over the cells) against the CPU oracle, element by element, plus the 5D and
7D workloads at full size on sampled outputs."""
import numpy as np
import pytest

import oracle
from paper_1912_06255_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1912_06255_gb300 import DBSCAN, DbscanError, _lib, dbscan  # noqa: E402
from _certify import check_links, sampled_invariants  # noqa: E402


def _assert_same(X, eps, mp, **kw):
    t = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    r = dbscan(t, eps, mp, **kw)
    torch.cuda.synchronize()
    got = (r.core.cpu().numpy(), r.labels.cpu().numpy(), r.border_offsets.cpu().numpy(), r.border_ids.cpu().numpy())
    exp = oracle.dbscan(X, eps, mp)
    for name, g, e in zip(("core", "labels", "border_offsets", "border_ids"), got, exp):
        if not np.array_equal(g, e):
            bad = np.flatnonzero(g != e)[:10] if g.shape == e.shape else "shape"
            raise AssertionError(f"{name} differs at {bad} (n={len(X)}, d={X.shape[1]}, eps={eps}, {kw})")
    return r.stats


@pytest.mark.parametrize("d", [5, 6, 7, 8])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_random_mixed_highdim(d, precision, dtype):
    X = synth.random_small(700 + d, 6000, d, dtype=dtype)
    for eps, mp in ((0.4, 4), (0.8, 12), (1.6, 40)):
        st = _assert_same(X, eps, mp, precision=precision)
        assert st["num_neighbor_entries"] >= 0


@pytest.mark.parametrize("d", [5, 6, 7, 8])
def test_lattice_exact_eps_highdim(d):
    """Axis neighbours at exactly eps: core iff interior (count 2d+1)."""
    L = 4 if d <= 5 else 3
    grid = np.stack(np.meshgrid(*[np.arange(L)] * d, indexing="ij"), -1).reshape(-1, d)
    X = (grid * 0.75 + 3.0).astype(np.float32)
    for precision in ("fp32", "fp64"):
        st = _assert_same(X, 0.75, 2 * d + 1, precision=precision)
        if precision == "fp32":
            assert st["band_rechecks"] > 0


@pytest.mark.parametrize("schedule", ["size", "none", "learned"])
@pytest.mark.parametrize("cell_bounds", [True, False])
def test_highdim_schedules(schedule, cell_bounds):
    X = synth.random_small(91, 12000, 6, dtype=np.float32)
    st = _assert_same(X, 0.9, 10, schedule=schedule, cell_bounds=cell_bounds)
    assert (st["num_pairs_tested"] + st["num_pairs_skipped"] + st["num_pairs_box_decided"]
            == st["num_candidate_pairs"])


def test_highdim_uniform_sparse():
    """Isolated points in 5D (every cell its own, no neighbours) and a few
    duplicates; one cell; minPts 1."""
    rng = np.random.default_rng(12)
    X = (rng.random((20000, 5)) * 1e4).astype(np.float32)
    _assert_same(X, 1.0, 2)
    _assert_same(X, 1.0, 1)
    Y = np.concatenate([X[:100], X[:100], X[:50]])  # pairs and triples of identical points
    _assert_same(Y, 5.0, 3)
    _assert_same(np.full((300, 7), 2.5, np.float32), 0.1, 300)


@pytest.mark.parametrize("eps", [200.0, 400.0, 800.0])
def test_spreader_5d_scaled(eps):
    """The 5D mixed workload at 1/100 size, every eps of its sweep."""
    I = synth.spreader_5d_10m(n=100_000, eps=eps)
    st = _assert_same(I.points, I.eps, I.min_pts)
    assert st["num_cells"] > 1000


@pytest.mark.parametrize("eps", [500.0, 1000.0, 2000.0])
def test_spreader_7d_scaled(eps):
    I = synth.spreader_7d_10m(n=100_000, eps=eps)
    _assert_same(I.points, I.eps, I.min_pts)


@pytest.mark.parametrize("d", [7, 8])
def test_keys_wider_than_64_bits(d):
    """More than 64 key bits (the two-word sort): 10 bits per dimension."""
    X = synth.random_small(800 + d, 8000, d, dtype=np.float32)
    rng = np.random.default_rng(d)
    X = np.concatenate([X, X[:2000] + (rng.standard_normal((2000, d)) * 0.01).astype(np.float32)])
    eps = 10.0 * np.sqrt(d) / 700.0  # about 800 cells per dimension
    st = _assert_same(X, eps, 2)
    assert st["key_bits"] > 64
    _assert_same(X, eps * 8, 3, precision="fp64")


def test_highdim_key_overflow_and_reuse():
    ctx = DBSCAN(1000, 8)
    X = torch.zeros((10, 6), device="cuda", dtype=torch.float64)
    X[1, 0] = 1e6
    with pytest.raises(DbscanError) as e:
        ctx.run(X, 1.0, 2)  # 2.4e6 cells in one dimension > 2^15
    assert e.value.status == 4
    # the same context alternates between tree and hash paths
    for d in (3, 7, 2, 5):
        Y = synth.random_small(30 + d, 900, d, dtype=np.float32)
        r = ctx.run(torch.from_numpy(Y).cuda(), 0.5, 5)
        exp = oracle.dbscan(Y, 0.5, 5)
        assert np.array_equal(r.labels.cpu().numpy(), exp[1]), d
        assert np.array_equal(r.border_ids.cpu().numpy(), exp[3]), d


def _full_size_checked(I, d, seed):
    """One full-size run with link witnesses: sampled outputs against the
    oracle and every cluster certified as a connected graph of verified
    eps-edges."""
    ctx = DBSCAN(len(I.points), d)
    ctx.set_option(_lib.OPT_WITNESS, 1)
    r = ctx.run(torch.from_numpy(I.points).cuda(), I.eps, I.min_pts)
    core, labels = r.core.cpu().numpy(), r.labels.cpu().numpy()
    off, ids = r.border_offsets.cpu().numpy(), r.border_ids.cpu().numpy()
    rep, links = ctx.link_witnesses()
    ncl = check_links(I.points, I.eps, core, labels, rep.cpu().numpy(), links.cpu().numpy(),
                      num_core_cells=r.stats["num_core_cells"])
    rng = np.random.default_rng(seed)
    samples = np.sort(rng.choice(len(I.points), 2000, replace=False))
    sampled_invariants(I.points, I.eps, I.min_pts, core, labels, off, ids, samples)
    return ncl


@pytest.mark.slow
@pytest.mark.parametrize("eps", [200.0, 400.0, 800.0])
def test_spreader_5d_full_size_sampled(eps):
    """The 10M-point 5D mixed workload (FP32, minPts 10) on sampled outputs,
    with the link certificate."""
    assert _full_size_checked(synth.spreader_5d_10m(eps=eps), 5, 5) > 0


@pytest.mark.slow
@pytest.mark.parametrize("eps", [500.0, 1000.0, 2000.0])
def test_spreader_7d_full_size_sampled(eps):
    """The 10M-point 7D varying-density workload (FP32, minPts 100) on sampled
    outputs, with the link certificate (eps 500 needs 70-bit cell keys)."""
    assert _full_size_checked(synth.spreader_7d_10m(eps=eps), 7, 7) > 0


def test_highdim_list_buffer_grows():
    """More neighbour entries than the context's list buffer (840 per point):
    the buffer grows and the walk runs again, with the exact result.  In 7D,
    about one point per cell in a box of 5 cells a side gives each cell some
    2,500 neighbouring cells."""
    rng = np.random.default_rng(23)
    n, d = 8000, 7
    eps = 1.0
    X = rng.random((n, d)) * (eps / np.sqrt(d)) * 5.0
    ctx = DBSCAN(n, d, precision="fp64")
    for eps_run, mp in ((eps, 2), (0.8 * eps, 30)):
        r = ctx.run(torch.from_numpy(X).cuda(), eps_run, mp)
        exp = oracle.dbscan(X, eps_run, mp)
        assert np.array_equal(r.core.cpu().numpy(), exp[0])
        assert np.array_equal(r.labels.cpu().numpy(), exp[1])
        assert np.array_equal(r.border_ids.cpu().numpy(), exp[3])
        if mp == 2:
            assert ctx.stats()["num_neighbor_entries"] > 840 * n


@pytest.mark.parametrize("levels", [1, 2, 3])
@pytest.mark.parametrize("d", [5, 6, 7, 8])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_quadtree_range_counts(levels, d, dtype):
    """MarkCore's range counts through the quadtree below the cells (Sec. 5.2)
    give the exact result, with the warp kernel and with the thread-per-point
    kernel for small cells."""
    X = synth.random_small(900 + d, 12000, d, dtype=dtype)
    X = np.concatenate([X, X[:3000] + 0.01])  # denser cells, so large neighbouring cells exist
    for eps, mp in ((0.8, 12), (1.6, 60)):
        exp = oracle.dbscan(X, eps, mp)
        for small in (0, 1 << 30):
            ctx = DBSCAN(len(X), d)
            ctx.set_option(_lib.OPT_QUADTREE, levels)
            ctx.set_option(_lib.OPT_SMALL_CELLS, small)
            r = ctx.run(torch.from_numpy(X).cuda(), eps, mp)
            for g, e in zip((r.core, r.labels, r.border_offsets, r.border_ids), exp):
                assert np.array_equal(g.cpu().numpy(), e), (levels, d, eps, small)


@pytest.mark.parametrize("which,eps", [("5d", 200.0), ("5d", 800.0), ("7d", 500.0), ("7d", 1000.0), ("7d", 2000.0)])
def test_quadtree_on_the_workloads(which, eps):
    I = synth.spreader_5d_10m(n=100_000, eps=eps) if which == "5d" else synth.spreader_7d_10m(n=100_000, eps=eps)
    d = I.points.shape[1]
    exp = oracle.dbscan(I.points, I.eps, I.min_pts)
    ctx = DBSCAN(len(I.points), d)
    ctx.set_option(_lib.OPT_QUADTREE, 2)
    r = ctx.run(torch.from_numpy(I.points).cuda(), I.eps, I.min_pts)
    for g, e in zip((r.core, r.labels, r.border_offsets, r.border_ids), exp):
        assert np.array_equal(g.cpu().numpy(), e)


def test_quadtree_option_values():
    ctx = DBSCAN(100, 5)
    for bad in (-1, 4):
        with pytest.raises(DbscanError):
            ctx.set_option(_lib.OPT_QUADTREE, bad)
    ctx.set_option(_lib.OPT_QUADTREE, 3)
    assert ctx.get_option(_lib.OPT_QUADTREE) == 3
