"""The seeded input generators: reproducible, shaped as their recipes say.

The large 3D generator builds its points in parallel blocks and shuffles them
with a parallel bucket shuffle; its output must not depend on the number of
threads, must stay in the stated box, and must leave memory order without
spatial coherence.
"""
import numpy as np

from paper_1912_06255_gb300 import synth


def test_scaled_spreader_is_deterministic_and_thread_independent():
    a = synth.spreader_3d_scaled(300_000, seed=11, threads=1)
    b = synth.spreader_3d_scaled(300_000, seed=11, threads=5)
    c = synth.spreader_3d_scaled(300_000, seed=12, threads=5)
    assert a.points.dtype == np.float32 and a.points.shape == (300_000, 3)
    assert np.array_equal(a.points, b.points)
    assert not np.array_equal(a.points, c.points)
    assert (a.eps, a.min_pts) == (100.0, 100)


def test_scaled_spreader_fills_a_given_buffer_and_keeps_the_box():
    n = 120_000
    out = np.full((n, 3), np.nan, np.float32)
    inst = synth.spreader_3d_scaled(n, seed=3, out=out)
    assert inst.points is out and np.isfinite(out).all()
    box = 1e5 * (n / 2e6) ** (1.0 / 3.0)
    # walkers start in the box and take a 50-unit step every 100 points; points
    # lie within the ball radius of a walker position
    per = (n - max(1, round(n * 1e-4))) // max(1, n // 20000)
    reach = 100.0 + 50.0 * (per // 100) + 1.0
    assert out.min() >= -reach and out.max() <= box + reach


def test_scaled_spreader_shuffle_is_a_permutation():
    """The rows form the same multiset for two thread counts, and the shuffle
    leaves no spatial order in memory."""
    n = 50_000
    x = synth.spreader_3d_scaled(n, seed=5, threads=2).points
    y = synth.spreader_3d_scaled(n, seed=5, threads=7).points
    order = np.lexsort(x.T[::-1])
    assert np.array_equal(x[order], y[np.lexsort(y.T[::-1])])
    # memory order carries no spatial coherence: consecutive rows are not from
    # one ball (radius 100) as an unshuffled walker segment would be
    gaps = np.linalg.norm(np.diff(x.astype(np.float64), axis=0), axis=1)
    assert np.median(gaps) > 500.0
