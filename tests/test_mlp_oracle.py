"""Pins for the FP64 gradient oracle of the scheduler network (no GPU).

The analytic backward pass must match central finite differences of the loss,
and the all-zero network has a closed-form loss and gradient."""
import math

import numpy as np

from oracle import mlp


def test_zero_network_closed_form():
    rng = np.random.default_rng(0)
    X = rng.normal(size=(50, mlp.F))
    y = (rng.random(50) < 0.3).astype(float)
    w = np.zeros(mlp.NPARAM)
    L, g = mlp.loss_grad(w, X, y)
    assert abs(L - math.log(2.0)) < 1e-15          # logit 0 everywhere
    assert abs(g[-1] - np.mean(0.5 - y)) < 1e-15    # d/db3 = mean(sigmoid(0) - y)
    assert np.all(g[:-1] == 0.0)                    # hidden units are all off


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    X = rng.normal(size=(40, mlp.F)) * 2.0
    y = (rng.random(40) < 0.5).astype(float)
    w = rng.normal(size=mlp.NPARAM) * 0.3
    _, g = mlp.loss_grad(w, X, y)
    h = 1e-6
    idx = rng.choice(mlp.NPARAM, 120, replace=False)
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (mlp.loss(wp, X, y) - mlp.loss(wm, X, y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
