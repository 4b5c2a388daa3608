"""The link-certificate checker on the CPU: it accepts a certificate built from
the oracle's own clustering and rejects planted mistakes (a spurious merge of
two clusters, a witness pair farther than eps, a missing link, a witness on a
non-core point)."""
import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import minimum_spanning_tree

import oracle
from paper_1912_06255_gb300 import synth

from _certify import check_links


def _certificate(X, eps, mp):
    core, labels, _, _ = oracle.dbscan(X, eps, mp)
    idx = np.flatnonzero(core == 1)
    n = len(X)
    # every core-core pair, its predicate, then a spanning forest of the true eps-edges
    a, b = np.triu_indices(len(idx), 1)
    pr = np.stack([idx[a], idx[b]], 1)
    ok = oracle.within_pairs(X, eps, pr)
    e = pr[ok]
    g = coo_matrix((np.ones(len(e)), (e[:, 0], e[:, 1])), shape=(n, n))
    t = minimum_spanning_tree(g).tocoo()
    links = np.stack([t.row, t.col], 1)
    rep = np.full(n, -1, np.int64)
    rep[idx] = idx
    return core, labels, rep, links


def test_certificate_accepts_the_oracle_and_rejects_plants():
    X = synth.random_small(3, 1500, 2)
    eps, mp = 0.35, 6
    core, labels, rep, links = _certificate(X, eps, mp)
    names = np.unique(labels[core == 1])
    assert len(names) >= 3 and len(links) > 10
    assert check_links(X, eps, core, labels, rep, links) == len(names)
    # a spurious merge: two clusters under one name
    bad = labels.copy()
    bad[bad == names[1]] = names[0]
    with pytest.raises(AssertionError):
        check_links(X, eps, core, bad, rep, links)
    # a witness pair beyond eps joining two clusters
    i = np.flatnonzero(labels == names[0])[0]
    j = np.flatnonzero(labels == names[1])[0]
    with pytest.raises(AssertionError):
        check_links(X, eps, core, bad, rep, np.concatenate([links, [[i, j]]]))
    # a dropped link splits a cluster's certificate
    with pytest.raises(AssertionError):
        check_links(X, eps, core, labels, rep, links[1:])
    # a witness on a non-core point
    nc = np.flatnonzero(core == 0)[0]
    with pytest.raises(AssertionError):
        check_links(X, eps, core, labels, rep, np.concatenate([links, [[nc, i]]]))
