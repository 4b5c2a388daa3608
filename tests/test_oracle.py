"""Pins for the CPU oracle: each test ties it to something other than itself.

The oracle follows the DBSCAN definition of Sec. 2.  These tests check it
against library routines (scikit-learn's DBSCAN, SciPy's single linkage and
connected components), closed forms (integer lattices), a hand-derived example,
exact-boundary cases, and the special cases the definition implies.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1912_06255_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _sets(off, ids, n):
    return [list(ids[off[i]:off[i + 1]]) for i in range(n)]


def test_hand_example_two_plus():
    """Sec. 2: a border point shared by two clusters; ties at exactly eps count."""
    g = json.load(open(os.path.join(GOLDEN, "two_plus_2d.json")))
    X = np.array(g["points"], dtype=np.float64)
    core, labels, off, ids = oracle.dbscan(X, g["eps"], g["min_pts"])
    assert core.tolist() == g["core"]
    assert labels.tolist() == g["labels"]
    assert _sets(off, ids, len(X)) == g["border_sets"]
    # Just below eps every arm detaches: no point reaches minPts.
    core2, labels2, off2, _ = oracle.dbscan(X, math.nextafter(g["eps"], 0.0), g["min_pts"])
    assert core2.sum() == 0 and (labels2 == -1).all() and off2[-1] == 0


@pytest.mark.parametrize("d", [1, 2, 3, 4])
@pytest.mark.parametrize("L", [3, 5])
def test_integer_lattice_closed_form(d, L):
    """Lattice {0..L-1}^d, eps = 1 (axis neighbours at exactly eps), minPts = 2d+1.

    A point's count is 1 + #axis neighbours inside the lattice, so the core
    points are exactly the interior ones; they form one cluster (named by the
    first interior index); a non-core point with exactly one boundary
    coordinate touches an interior point and is border; the rest is noise."""
    grid = np.stack(np.meshgrid(*[np.arange(L)] * d, indexing="ij"), -1).reshape(-1, d)
    X = grid.astype(np.float64)
    core, labels, off, ids = oracle.dbscan(X, 1.0, 2 * d + 1)
    on_edge = (grid == 0) | (grid == L - 1)
    interior = ~on_edge.any(1)
    assert (core.astype(bool) == interior).all()
    first = int(np.flatnonzero(interior)[0]) if interior.any() else -1
    border = on_edge.sum(1) == 1
    exp = np.where(interior | border, first, -1)
    assert (labels == exp).all()
    sets = _sets(off, ids, len(X))
    for i in range(len(X)):
        assert sets[i] == ([first] if border[i] else [])


def test_lattice_scaled_dyadic_invariance():
    """Scaling coordinates and eps by 2^k is exact, so the result is unchanged."""
    rng = np.random.default_rng(7)
    X = rng.integers(0, 40, (600, 3)).astype(np.float64)
    base = oracle.dbscan(X, 3.0, 6)
    for k in (-6, 5):
        sc = oracle.dbscan(X * 2.0 ** k, 3.0 * 2.0 ** k, 6)
        for a, b in zip(base, sc):
            assert np.array_equal(a, b)


def test_dyadic_translation_invariance():
    """Points on a 2^-4 grid moved by a multiple of 2^10: every coordinate
    difference is the same exact number, so the result is unchanged (a dropped
    or shifted origin term would show here)."""
    rng = np.random.default_rng(17)
    X = rng.integers(0, 160, (800, 3)).astype(np.float64) / 16.0
    base = oracle.dbscan(X, 1.25, 5)
    assert 0 < base[0].sum() < len(X) and len(np.unique(base[1][base[0] == 1])) > 1  # core, noise, clusters
    for t in ((1024.0, 0.0, 0.0), (-3072.0, 2048.0, 1024.0)):
        moved = oracle.dbscan(X + np.array(t), 1.25, 5)
        for a, b in zip(base, moved):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("pts,eps", [(((0.0, 0.0), (3.0, 4.0)), 5.0),
                                     (((1.0, 2.0, 2.0), (0.0, 0.0, 0.0)), 3.0),
                                     (((0.5,), (2.0,)), 1.5)])
def test_exact_eps_is_inclusive(pts, eps):
    """d(p,q) <= eps (Sec. 2) is inclusive: a pair at exactly eps is joined."""
    X = np.array(pts, dtype=np.float64)
    core, labels, _, _ = oracle.dbscan(X, eps, 2)
    assert core.tolist() == [1, 1] and labels.tolist() == [0, 0]
    core, labels, _, _ = oracle.dbscan(X, math.nextafter(eps, 0.0), 2)
    assert core.tolist() == [0, 0] and labels.tolist() == [-1, -1]


def test_special_cases():
    rng = np.random.default_rng(3)
    X = rng.random((300, 3))
    # minPts > n: all noise.
    core, labels, off, _ = oracle.dbscan(X, 0.2, 301)
    assert core.sum() == 0 and (labels == -1).all() and off[-1] == 0
    # eps above the diameter: one cluster named 0 (every point core).
    core, labels, off, _ = oracle.dbscan(X, 2.0, 300)
    assert core.all() and (labels == 0).all()
    # All points identical: one cell; all core iff n >= minPts.
    Y = np.full((50, 2), 1.25)
    assert oracle.dbscan(Y, 1e-3, 50)[0].all()
    assert not oracle.dbscan(Y, 1e-3, 51)[0].any()
    # Empty input.
    core, labels, off, ids = oracle.dbscan(np.zeros((0, 2)), 1.0, 3)
    assert core.size == 0 and off.tolist() == [0] and ids.size == 0


def _check_against_sklearn(X, eps, mp):
    skc = pytest.importorskip("sklearn.cluster")
    core, labels, off, ids = oracle.dbscan(X, eps, mp)
    m = skc.DBSCAN(eps=eps, min_samples=mp, algorithm="brute").fit(X)
    sk_core = np.zeros(len(X), bool)
    sk_core[m.core_sample_indices_] = True
    assert (core.astype(bool) == sk_core).all()
    # Same partition of the core points.
    ci = np.flatnonzero(sk_core)
    ours, theirs = labels[ci], m.labels_[ci]
    fwd, bwd = {}, {}
    for a, b in zip(ours, theirs):
        assert fwd.setdefault(a, b) == b and bwd.setdefault(b, a) == a
    # Each cluster is named by its smallest core index.
    for name in np.unique(ours):
        assert name == ci[ours == name].min()
    # Noise agrees; scikit-learn puts a border point in one of its clusters.
    nc = np.flatnonzero(~sk_core)
    for i in nc:
        s = ids[off[i]:off[i + 1]]
        if m.labels_[i] == -1:
            assert s.size == 0 and labels[i] == -1
        else:
            assert bwd[m.labels_[i]] in s and labels[i] == s.min()
    return core, labels


@pytest.mark.parametrize("d", [1, 2, 3, 5, 7])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_matches_sklearn(d, seed):
    X = synth.random_small(100 + seed * 10 + d, 700, d)
    # eps near the median nearest-neighbour distance times a few.
    rng = np.random.default_rng(seed)
    sub = X[rng.choice(len(X), 50, replace=False)]
    nn = np.sort(np.sqrt(((sub[:, None, :] - X[None]) ** 2).sum(-1)), 1)[:, 1]
    eps = float(np.median(nn) * (2.0 + seed))
    for mp in (1, 2, 5, 20):
        _check_against_sklearn(X, eps, mp)


def test_blobs_2d_20k_against_sklearn():
    I = synth.blobs_2d_20k()
    core, labels = _check_against_sklearn(I.points, I.eps, I.min_pts)
    assert 0 < core.sum() < len(core)


@pytest.mark.parametrize("seed", [0, 1])
def test_min_pts_one_is_single_linkage(seed):
    """minPts = 1 makes every point core; clusters become single-linkage
    components at height eps."""
    hier = pytest.importorskip("scipy.cluster.hierarchy")
    X = synth.random_small(200 + seed, 500, 3)
    eps = 0.3
    core, labels, off, _ = oracle.dbscan(X, eps, 1)
    assert core.all() and off[-1] == 0
    f = hier.fcluster(hier.linkage(X, "single"), t=eps, criterion="distance")
    fwd, bwd = {}, {}
    for a, b in zip(labels, f):
        assert fwd.setdefault(a, b) == b and bwd.setdefault(b, a) == a


def test_connected_components_library():
    """Clusters equal SciPy's connected components of the core eps-graph."""
    csg = pytest.importorskip("scipy.sparse.csgraph")
    sp = pytest.importorskip("scipy.sparse")
    X = synth.random_small(42, 800, 2)
    eps, mp = 0.25, 6
    core, labels, _, _ = oracle.dbscan(X, eps, mp)
    D2 = ((X[:, None, :] - X[None]) ** 2).sum(-1)
    A = D2 <= eps * eps
    assert ((A.sum(1) >= mp) == core.astype(bool)).all()
    ci = np.flatnonzero(core)
    ncomp, comp = csg.connected_components(sp.csr_matrix(A[np.ix_(ci, ci)]), directed=False)
    for c in range(ncomp):
        members = ci[comp == c]
        assert (labels[members] == members.min()).all()


def test_permutation_relabels_only():
    X = synth.random_small(9, 900, 3)
    eps, mp = 0.3, 5
    core, labels, off, ids = oracle.dbscan(X, eps, mp)
    perm = np.random.default_rng(1).permutation(len(X))
    core2, labels2, off2, ids2 = oracle.dbscan(X[perm], eps, mp)
    assert (core2 == core[perm]).all()
    # Map names through the permutation: new name = smallest new index.
    inv = np.argsort(perm)
    for name in np.unique(labels[core.astype(bool)]):
        members_new = inv[np.flatnonzero((labels == name) & core.astype(bool))]
        assert (labels2[members_new] == members_new.min()).all()
    # Border sets have the same sizes after relabelling.
    assert ((off2[1:] - off2[:-1]) == (off[1:] - off[:-1])[perm]).all()


def test_sample_queries_agree_with_definition():
    X = synth.random_small(5, 1000, 4)
    eps, mp = 0.4, 8
    core, labels, _, _ = oracle.dbscan(X, eps, mp)
    s = np.arange(0, 1000, 7)
    cnt = oracle.sample_counts(X, eps, s)
    assert ((cnt >= mp) == core[s].astype(bool)).all()
    D2 = ((X[s][:, None, :] - X[None]) ** 2).sum(-1)
    assert (cnt == (D2 <= eps * eps).sum(1)).all()
    nb = oracle.neighbors(X, eps, 3)
    assert nb.tolist() == np.flatnonzero(((X - X[3]) ** 2).sum(1) <= eps * eps).tolist()


def test_within_pairs_pins():
    """The pairwise predicate (used to verify link witnesses of GPU runs):
    exact-eps lattice pairs are in, their nextafter neighbours and diagonals
    out (Sec. 2 is inclusive), SciPy's distances agree away from the boundary,
    and each pair is taken in its own order (a swapped or shifted index would
    fail the neighbour check)."""
    from scipy.spatial.distance import cdist
    # 3-4-5 and 1-2-2 pairs at exactly eps; nextafter below eps is out
    X = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0], [1.0, 2.0, 2.0], [0.0, 0.0, 5.0]])
    got = oracle.within_pairs(X, 5.0, [[0, 1], [1, 0], [0, 3], [1, 3], [0, 2]])
    assert got.tolist() == [True, True, True, False, True]
    assert not oracle.within_pairs(X, math.nextafter(5.0, 0.0), [[0, 1]]).any()
    assert oracle.within_pairs(X, 3.0, [[0, 2]]).all()
    assert not oracle.within_pairs(X, math.nextafter(3.0, 0.0), [[0, 2]]).any()
    # random pairs against SciPy, skipping the 1e-9 band around eps
    rng = np.random.default_rng(41)
    for d in (1, 3, 7):
        Y = rng.random((400, d)) * 4.0
        pr = rng.integers(0, 400, (5000, 2))
        eps = 1.1
        dist = cdist(Y, Y)[pr[:, 0], pr[:, 1]]
        keep = np.abs(dist - eps) > 1e-9
        got = oracle.within_pairs(Y, eps, pr)
        assert np.array_equal(got[keep], (dist <= eps)[keep])
    # against the neighbour scan: pairs (p, q) for all q select exactly neighbors(p)
    Z = synth.random_small(6, 800, 3)
    for p in (0, 17, 799):
        pr = np.stack([np.full(800, p), np.arange(800)], 1)
        assert np.flatnonzero(oracle.within_pairs(Z, 0.35, pr)).tolist() == oracle.neighbors(Z, 0.35, p).tolist()
    with pytest.raises(RuntimeError):
        oracle.within_pairs(Z, 0.35, [[0, 800]])
