"""Checker of approximate DBSCAN results (the rho-approximate problem of Gan
and Tao, Sec. 2).  TEST INFRASTRUCTURE ONLY: like the rest of ``oracle/``, it
is called by the tests alone and shares nothing with the CUDA library.

The approximate problem keeps the DBSCAN core rule and border rule and relaxes
only the connectivity of core points: two core points within eps are
connected, two farther apart than eps(1+rho) are not connected directly, and a
pair in between may or may not be.  Clusters are the connected components of
the core points under some such choice.  The result is therefore not unique,
so this module checks a given result instead of computing one.  A clustering
of the core points is valid iff

  (a) every connected component of the eps-graph of the core points lies
      inside one cluster, and
  (b) every cluster is connected in the eps(1+rho)-graph of its own core
      points;

then the clusters are the components of the graph made of the eps-edges and
a spanning tree of each cluster in the eps(1+rho)-graph, which lies between
the two graphs, and conversely.  On top of that the checker requires the
conventions of the exact outputs: core flags equal to the exact ones, each
cluster named by its smallest core index, and each non-core point's set equal
to the sorted names of the clusters with a core point within eps of it
(labels = the smallest, -1 when empty).

Distances are the FP64 predicate of the exact oracle: sum_j (p_j - q_j)^2,
left to right, each operation rounded, against fl(r * r) with r = eps or
r = fl(eps * (1 + rho)).  Brute force over all pairs: for small cases.
"""
from __future__ import annotations

import numpy as np

__all__ = ["check_approx", "is_valid_approx"]


def _d2_matrix(X: np.ndarray) -> np.ndarray:
    """All squared distances, summed over the coordinates in order."""
    X = np.asarray(X, dtype=np.float64)
    n, d = X.shape
    s = np.zeros((n, n), dtype=np.float64)
    for j in range(d):
        t = X[:, j][:, None] - X[:, j][None, :]
        s = s + t * t
    return s


def _components(adj: np.ndarray, nodes: np.ndarray) -> list:
    """Connected components of the graph adj restricted to nodes (lists of indices)."""
    left = set(int(i) for i in nodes)
    comps = []
    while left:
        start = left.pop()
        comp, stack = [start], [start]
        while stack:
            u = stack.pop()
            nbrs = [int(v) for v in np.flatnonzero(adj[u]) if int(v) in left]
            for v in nbrs:
                left.discard(v)
                comp.append(v)
                stack.append(v)
        comps.append(sorted(comp))
    return comps


def check_approx(X, eps: float, min_pts: int, rho: float, core, labels, border_offsets=None,
                 border_ids=None) -> None:
    """Raise AssertionError naming the first rule a result breaks."""
    X = np.asarray(X, dtype=np.float64)
    n = len(X)
    core = np.asarray(core).astype(bool)
    labels = np.asarray(labels).astype(np.int64)
    assert core.shape == (n,) and labels.shape == (n,), "output shapes"
    if n == 0:
        return
    d2 = _d2_matrix(X)
    T = float(eps) * float(eps)
    r = float(eps) * (1.0 + float(rho))
    Tr = r * r
    near = d2 <= T
    # core rule: at least min_pts points within eps, the point itself included
    exact_core = near.sum(axis=1) >= int(min_pts)
    assert np.array_equal(core, exact_core), "core flags differ from the core rule"
    ci = np.flatnonzero(core)
    # (a) eps-components of the core points inside one cluster
    for comp in _components(near & core[None, :] & core[:, None], ci):
        assert len(set(labels[comp].tolist())) == 1, "an eps-connected group of core points is split"
    # (b) every cluster connected in the eps(1+rho)-graph of its core points; named by its smallest index
    wide = (d2 <= Tr) & core[None, :] & core[:, None]
    for name in np.unique(labels[ci]):
        members = ci[labels[ci] == name]
        assert name == members.min(), "a cluster is not named by its smallest core index"
        comps = _components(wide, members)
        assert len(comps) == 1, "a cluster is not connected within eps(1+rho)"
    # border rule: the clusters with a core point within eps of a non-core point
    for p in np.flatnonzero(~core):
        exp = sorted(set(labels[ci[near[p, ci]]].tolist()))
        assert labels[p] == (exp[0] if exp else -1), "a non-core label is not its smallest cluster"
        if border_offsets is not None:
            got = list(np.asarray(border_ids)[int(border_offsets[p]):int(border_offsets[p + 1])])
            assert got == exp, "a border set differs from the clusters within eps"
    if border_offsets is not None:
        off = np.asarray(border_offsets)
        assert all(off[i] == off[i + 1] for i in ci), "a core point has a border set"


def is_valid_approx(*args, **kw) -> bool:
    try:
        check_approx(*args, **kw)
    except AssertionError:
        return False
    return True
