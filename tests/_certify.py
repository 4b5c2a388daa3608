"""Checks of large GPU runs that the oracle cannot redo in full.

``check_links``: the link certificate of a run made with DBSCAN_OPT_WITNESS.
Every pair it names is verified with the oracle's FP64 predicate (Sec. 2):
the star edges (each core point to the first core point of its cell) and the
pairs recorded at each union of the union-find.  All of them must join two
points the run flagged core and carry equal labels.  The components of these
verified eps-edges must then be exactly the run's clusters: as many components
as cluster names, so no cluster is a union of two groups that no eps-path
joins (no spurious merge).

``sampled_invariants``: the core flag of sampled points by a count over all
points, equal labels of the sampled core points and their core neighbours
within eps (no split along those edges), border sets and noise, and canonical
names (the smallest core index of each cluster).
"""
import numpy as np
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components

import oracle


def check_links(X, eps, core, labels, rep, links, num_core_cells=None):
    """X [n, d] (the instance's own coordinates), outputs of one instance with
    rep and links in its own row indices."""
    n = len(X)
    core = np.asarray(core).astype(bool)
    labels = np.asarray(labels)
    rep = np.asarray(rep).astype(np.int64)
    links = np.asarray(links, dtype=np.int64).reshape(-1, 2)
    assert (rep[~core] == -1).all(), "a non-core point has a cell representative"
    idx = np.flatnonzero(core)
    r = rep[idx]
    assert ((r >= 0) & (r < n)).all() and core[r].all(), "a representative is not a core point"
    star = np.stack([idx, r], 1)
    star = star[star[:, 0] != star[:, 1]]
    if len(links):
        assert ((links >= 0) & (links < n)).all(), "a witness outside the instance"
        assert core[links].all(), "a link witness names a non-core point"
    edges = np.concatenate([star, links]) if len(links) else star
    ok = oracle.within_pairs(X, eps, edges)
    assert ok.all(), f"{int((~ok).sum())} witness pairs are farther than eps, e.g. {edges[~ok][:3].tolist()}"
    assert (labels[edges[:, 0]] == labels[edges[:, 1]]).all(), "a verified eps-edge joins two clusters"
    if len(idx) == 0:
        return 0
    g = coo_matrix((np.ones(len(edges), np.int8), (edges[:, 0], edges[:, 1])), shape=(n, n))
    _, comp = connected_components(g, directed=False)
    ncomp = len(np.unique(comp[idx]))
    ncl = len(np.unique(labels[idx]))
    assert ncomp == ncl, f"{ncl} clusters but {ncomp} components of verified eps-edges"
    if num_core_cells is not None:
        assert len(links) == num_core_cells - ncl, "one witness per union expected"
    return ncl


def sampled_invariants(X, eps, mp, core, labels, off, ids, samples, n_nbr=300):
    cnt = oracle.sample_counts(X, eps, samples)
    assert np.array_equal(core[samples], (cnt >= mp).astype(np.uint8))
    for p in samples[:n_nbr]:
        nb = oracle.neighbors(X, eps, int(p))
        cn = nb[core[nb] == 1]
        if core[p]:
            assert np.all(labels[cn] == labels[p]), p
        else:
            exp = np.unique(labels[cn])
            assert np.array_equal(ids[off[p]:off[p + 1]], exp), p
            assert labels[p] == (exp[0] if len(exp) else -1), p
    # cluster names: the smallest core index of the cluster, itself core
    cl = labels[core == 1]
    idx = np.flatnonzero(core == 1)
    first = np.full(len(X), np.iinfo(np.int64).max)
    np.minimum.at(first, cl, idx)
    names = np.unique(cl)
    assert np.array_equal(first[names], names)
