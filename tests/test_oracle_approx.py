"""Pins of the approximate-DBSCAN checker (Sec. 2, the rho-approximate problem).

Each case either builds a result the definition allows and expects the checker
to accept it, or plants one mistake (a split eps-group, a merge across a gap
wider than eps(1+rho), a wrong core flag, a wrong border set, a wrong name) and
expects a rejection.  The exact result must be accepted for every rho.
"""
import numpy as np
import pytest

import oracle
from oracle import approx
from paper_1912_06255_gb300 import synth


def _line(gap):
    """Two 1D groups, all core at eps 0.6 and minPts 2: A = {0, 0.5, 1.0},
    B = {1.0 + gap, 1.5 + gap}."""
    return np.array([[0.0], [0.5], [1.0], [1.0 + gap], [1.5 + gap]])


@pytest.mark.parametrize("rho", [0.0, 0.01, 0.1, 0.5])
def test_exact_result_is_valid(rho):
    for seed, d in ((3, 2), (4, 3), (5, 5)):
        X = synth.random_small(seed, 700, d)
        for eps, mp in ((0.3, 4), (0.6, 10)):
            core, labels, off, ids = oracle.dbscan(X, eps, mp)
            approx.check_approx(X, eps, mp, rho, core, labels, off, ids)


def test_merge_inside_the_slack_only():
    X = _line(0.65)  # closest cross pair 0.65: beyond eps 0.6, within 0.6 * 1.1 = 0.66
    core, labels, off, ids = oracle.dbscan(X, 0.6, 2)
    assert labels.tolist() == [0, 0, 0, 3, 3]
    merged = np.zeros(5, dtype=np.int32)
    assert approx.is_valid_approx(X, 0.6, 2, 0.1, core, labels)   # not merging is allowed
    assert approx.is_valid_approx(X, 0.6, 2, 0.1, core, merged)   # merging is allowed
    assert not approx.is_valid_approx(X, 0.6, 2, 0.05, core, merged)  # 0.63 < 0.65: not allowed
    assert not approx.is_valid_approx(X, 0.6, 2, 0.0, core, merged)   # rho = 0 is exact DBSCAN


def test_split_of_an_eps_group_is_rejected():
    X = _line(0.65)
    core, labels, _, _ = oracle.dbscan(X, 0.6, 2)
    split = labels.copy()
    split[2] = 2  # 1.0 is within eps of 0.5
    assert not approx.is_valid_approx(X, 0.6, 2, 0.5, core, split)


def test_wrong_core_flag_and_name_are_rejected():
    X = _line(0.65)
    core, labels, _, _ = oracle.dbscan(X, 0.6, 2)
    bad_core = core.copy()
    bad_core[4] = 0
    assert not approx.is_valid_approx(X, 0.6, 2, 0.1, bad_core, labels)
    renamed = labels.copy()
    renamed[3:] = 4  # not the smallest index of its cluster
    assert not approx.is_valid_approx(X, 0.6, 2, 0.1, core, renamed)


def test_border_sets_follow_the_chosen_clusters():
    """A non-core point within eps of one core point of each of two groups
    joins both clusters; if the groups are merged (allowed only when their
    closest core points are within eps(1+rho)), it joins the one."""
    A = [0.00, 0.01, 0.02, 0.03, 0.04]
    B = [2.03, 2.04, 2.05, 2.06, 2.07]
    X = np.array(A + [1.035] + B)[:, None]  # the point at 1.035 is 0.995 from 0.04 and from 2.03
    eps, mp = 1.0, 5
    core, labels, off, ids = oracle.dbscan(X, eps, mp)
    assert core.tolist() == [1] * 5 + [0] + [1] * 5
    assert labels.tolist() == [0] * 6 + [6] * 5 and ids.tolist() == [0, 6]
    approx.check_approx(X, eps, mp, 0.0, core, labels, off, ids)
    # dropping a cluster from the border set is rejected
    assert not approx.is_valid_approx(X, eps, mp, 0.0, core, labels, off, ids[:1])
    # the merged clustering: the groups are 1.99 apart
    merged = np.zeros(11, dtype=np.int32)
    moff = np.array([0] * 6 + [1] * 6, dtype=np.int64)
    mids = np.array([0], dtype=np.int32)
    assert approx.is_valid_approx(X, eps, mp, 1.0, core, merged, moff, mids)      # 1.99 <= 2.0
    assert not approx.is_valid_approx(X, eps, mp, 0.5, core, merged, moff, mids)  # 1.99 > 1.5
    # after a merge the old two-cluster border set is wrong
    assert not approx.is_valid_approx(X, eps, mp, 1.0, core, merged, off, ids)
