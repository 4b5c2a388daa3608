"""Seeded synthetic point sets shaped like the paper's workloads.

The paper evaluates on seed-spreader data (points emitted around a random walk,
with similar or variable cluster density), on UniformFill (uniform points in a
hypergrid) and on real datasets (Sec. 6, "Datasets").  None of those files is
available here, so these generators stand in for them.  Every generator draws
from ``numpy.random.Generator(PCG64(seed))`` and shuffles its output with the
same generator, so that memory order carries no spatial coherence.

This module holds input generation only: it computes nothing of the clustering
method, and both the CUDA path and the CPU oracle take their inputs from it.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _ball(rng: np.random.Generator, count: int, d: int, radius) -> np.ndarray:
    """Uniform samples in the d-ball: Gaussian direction scaled by R * U^(1/d)."""
    g = rng.standard_normal((count, d))
    norm = np.linalg.norm(g, axis=1, keepdims=True)
    norm[norm == 0.0] = 1.0
    r = np.asarray(radius, dtype=np.float64).reshape(-1, 1) * rng.random((count, 1)) ** (1.0 / d)
    return g / norm * r


def _unit(rng: np.random.Generator, count: int, d: int) -> np.ndarray:
    g = rng.standard_normal((count, d))
    norm = np.linalg.norm(g, axis=1, keepdims=True)
    norm[norm == 0.0] = 1.0
    return g / norm


def gaussian_blobs(rng, n: int, d: int, n_blobs: int, box: float, sigma: float,
                   noise_frac: float) -> np.ndarray:
    """Isotropic Gaussian blobs with centres uniform in [0, box]^d plus uniform noise."""
    n_noise = int(round(n * noise_frac))
    n_clustered = n - n_noise
    centres = rng.random((n_blobs, d)) * box
    per = np.full(n_blobs, n_clustered // n_blobs, dtype=np.int64)
    per[: n_clustered - per.sum()] += 1
    owner = np.repeat(np.arange(n_blobs), per)
    pts = centres[owner] + rng.standard_normal((n_clustered, d)) * sigma
    noise = rng.random((n_noise, d)) * box
    out = np.concatenate([pts, noise], axis=0)
    return out[rng.permutation(out.shape[0])]


def seed_spreader(rng, d: int, n_walkers: int, pts_per_walker: int, box: float,
                  radius, step, n_noise: int, seg: int = 100) -> np.ndarray:
    """Random-walk seed spreader.

    Each walker starts uniform in [0, box]^d and emits points uniformly in a ball
    of its radius around its current position; after every ``seg`` of its points
    it moves ``step`` units in a uniform random direction.  ``radius`` and
    ``step`` are scalars or per-walker arrays.  ``n_noise`` uniform points over
    [0, box]^d are added.
    """
    radius = np.broadcast_to(np.asarray(radius, dtype=np.float64), (n_walkers,))
    step = np.broadcast_to(np.asarray(step, dtype=np.float64), (n_walkers,))
    n_seg = -(-pts_per_walker // seg)
    parts = []
    for w in range(n_walkers):
        start = rng.random(d) * box
        moves = _unit(rng, n_seg, d) * step[w]
        moves[0] = 0.0
        pos = start + np.cumsum(moves, axis=0)
        centre = np.repeat(pos, seg, axis=0)[:pts_per_walker]
        parts.append(centre + _ball(rng, pts_per_walker, d, radius[w]))
    parts.append(rng.random((n_noise, d)) * box)
    out = np.concatenate(parts, axis=0)
    return out[rng.permutation(out.shape[0])]


@dataclass
class Instance:
    """One DBSCAN problem: points [n, d], eps, minPts and a descriptive name."""
    points: np.ndarray
    eps: float
    min_pts: int
    name: str
    meta: dict = field(default_factory=dict)


def blobs_2d_20k(seed: int = 1000, n: int = 20000) -> Instance:
    """2D: 10 Gaussian blobs (sigma 1, centres in [0,100]^2) + 10% noise, FP64, eps 0.5, minPts 10."""
    rng = _rng(seed)
    pts = gaussian_blobs(rng, n, 2, 10, 100.0, 1.0, 0.10).astype(np.float64)
    return Instance(pts, 0.5, 10, f"blobs2d-n{n}-eps0.5-minpts10-f64")


def spreader_3d_2m(seed: int = 1001, n: int = 2_000_000) -> Instance:
    """3D seed spreader: 100 walkers in [0,1e5]^3, ball radius 100, step 50 per 100
    points, 0.01% uniform noise; FP32; eps 100, minPts 100.  ``n`` scales the
    workload down for tests while keeping walker count and local density."""
    rng = _rng(seed)
    n_noise = max(1, int(round(n * 1e-4)))
    n_walkers = 100 if n >= 200_000 else max(2, n // 2000)
    per = (n - n_noise) // n_walkers
    n_noise = n - per * n_walkers
    pts = seed_spreader(rng, 3, n_walkers, per, 1e5 if n >= 200_000 else 1e5 * (n / 2e6) ** (1 / 3),
                        100.0, 50.0, n_noise)
    return Instance(pts.astype(np.float32), 100.0, 100, f"spreader3d-n{n}-eps100-minpts100-f32")


def spreader_5d_10m(seed: int = 1002, n: int = 10_000_000, eps: float = 200.0) -> Instance:
    """5D: half uniform in [0,1e5]^5, half from 100 walkers with radius U[50,500]
    and step radius/2 per 100 points; FP32; minPts 10."""
    rng = _rng(seed)
    n_uni = n // 2
    n_walkers = 100
    per = (n - n_uni) // n_walkers
    n_uni = n - per * n_walkers
    radius = rng.uniform(50.0, 500.0, n_walkers)
    pts = seed_spreader(rng, 5, n_walkers, per, 1e5, radius, radius / 2, n_uni)
    return Instance(pts.astype(np.float32), float(eps), 10, f"mixed5d-n{n}-eps{eps:g}-minpts10-f32")


def spreader_7d_10m(seed: int = 1004, n: int = 10_000_000, eps: float = 1000.0) -> Instance:
    """7D varying density: 100 walkers, radius log-uniform in [20,2000], step
    radius/2 per 100 points, 0.05% noise, box [0,1e5]^7; FP32; minPts 100."""
    rng = _rng(seed)
    n_noise = int(round(n * 5e-4))
    n_walkers = 100
    per = (n - n_noise) // n_walkers
    n_noise = n - per * n_walkers
    radius = np.exp(rng.uniform(math.log(20.0), math.log(2000.0), n_walkers))
    pts = seed_spreader(rng, 7, n_walkers, per, 1e5, radius, radius / 2, n_noise)
    return Instance(pts.astype(np.float32), float(eps), 100, f"varden7d-n{n}-eps{eps:g}-minpts100-f32")


def batch_256(seed: int = 1003, count: int = 256, lo: float = 1e3, hi: float = 1e6) -> list[Instance]:
    """Independent 2D/3D blob-plus-noise instances with log-uniform sizes.

    Instance i has d = 2 (even i) or 3 (odd i), n_i = round(exp(U[ln lo, ln hi])),
    max(1, round(n_i/2000)) blobs of sigma 1 in a box of side 100*(n_i/20000)^(1/d),
    10% noise, eps ~ U[0.2, 1.0], minPts ~ U{5..50}; FP32.
    """
    rng = _rng(seed)
    out = []
    for i in range(count):
        d = 2 if i % 2 == 0 else 3
        n_i = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        blobs = max(1, int(round(n_i / 2000)))
        box = 100.0 * (n_i / 20000.0) ** (1.0 / d)
        eps = float(rng.uniform(0.2, 1.0))
        mp = int(rng.integers(5, 51))
        pts = gaussian_blobs(rng, n_i, d, blobs, box, 1.0, 0.10).astype(np.float32)
        out.append(Instance(pts, eps, mp, f"batch{i}-d{d}-n{n_i}"))
    return out


def uniform_fill(seed: int, n: int, d: int, dtype=np.float32) -> np.ndarray:
    """UniformFill: n points uniform in a hypergrid of side sqrt(n) (Sec. 6)."""
    rng = _rng(seed)
    return (rng.random((n, d)) * math.sqrt(n)).astype(dtype)


def random_small(seed: int, n: int, d: int, dtype=np.float64, clustered: bool = True) -> np.ndarray:
    """Small mixed inputs for parity cases: a few blobs plus uniform noise in [0,10]^d."""
    rng = _rng(seed)
    if not clustered:
        return (rng.random((n, d)) * 10.0).astype(dtype)
    k = max(1, n // 60)
    return gaussian_blobs(rng, n, d, k, 10.0, 0.35, 0.15).astype(dtype)


def spreader_3d_scaled(n: int, seed: int = 1005, threads: int = 0, out: np.ndarray | None = None) -> Instance:
    """The 3D seed spreader at any size with the 2M-point workload's local
    density, as a stand-in for the paper's largest 3D inputs (Sec. 6 uses
    Cosmo50, 321M points, and billion-point sets): one walker per 20,000
    points (ball radius 100, a step of 50 every 100 points) in a box of side
    1e5 (n / 2e6)^(1/3), 0.01% uniform noise; FP32; eps 100, minPts 100.

    Built for hundreds of millions of points: the walkers are generated in
    blocks of 256, block k from its own PCG64 stream seeded by (seed, k), on
    ``threads`` threads (0: all cores); the points are then shuffled in
    parallel by sending each to a uniformly random one of 256 buckets and
    shuffling every bucket uniformly, which is a uniform random permutation.
    ``out`` may be a float32 [n, 3] array (e.g. pinned memory) to fill."""
    import os
    from concurrent.futures import ThreadPoolExecutor

    threads = threads or os.cpu_count() or 1
    n_walkers = max(1, n // 20000)
    n_noise = max(1, int(round(n * 1e-4)))
    per = (n - n_noise) // n_walkers
    n_noise = n - per * n_walkers
    box = 1e5 * (n / 2e6) ** (1.0 / 3.0)
    WB, NBK = 256, 256
    blocks = [(k, min(WB, n_walkers - k * WB)) for k in range(-(-n_walkers // WB))]
    noise_id = len(blocks)

    def gen(k):
        rng = np.random.Generator(np.random.PCG64([seed, k]))
        if k == noise_id:
            pts = (rng.random((n_noise, 3)) * box).astype(np.float32)
        else:
            w = blocks[k][1]
            n_seg = -(-per // 100)
            moves = _unit(rng, w * n_seg, 3).reshape(w, n_seg, 3) * 50.0
            moves[:, 0] = 0.0
            pos = rng.random((w, 1, 3)) * box + np.cumsum(moves, axis=1)
            centre = np.repeat(pos, 100, axis=1)[:, :per].reshape(-1, 3)
            pts = (centre + _ball(rng, w * per, 3, 100.0)).astype(np.float32)
        bucket = rng.integers(0, NBK, len(pts), dtype=np.int32)
        order = np.argsort(bucket, kind="stable")
        return pts[order], np.bincount(bucket, minlength=NBK)

    with ThreadPoolExecutor(threads) as ex:
        parts = list(ex.map(gen, range(noise_id + 1)))
    counts = np.stack([c for _, c in parts])            # [block, bucket]
    bucket_start = np.concatenate([[0], np.cumsum(counts.sum(0))])
    within = np.cumsum(counts, axis=0) - counts         # earlier blocks' share of each bucket
    res = np.empty((n, 3), np.float32) if out is None else out

    def place(k):
        pts, c = parts[k]
        src = np.concatenate([[0], np.cumsum(c)])
        for b in range(NBK):
            if c[b]:
                at = bucket_start[b] + within[k, b]
                res[at:at + c[b]] = pts[src[b]:src[b + 1]]

    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(place, range(len(parts))))
    parts.clear()

    def shuffle(b):
        rng = np.random.Generator(np.random.PCG64([seed, 1 << 20, b]))
        lo, hi = bucket_start[b], bucket_start[b + 1]
        res[lo:hi] = res[lo:hi][rng.permutation(hi - lo)]

    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(shuffle, range(NBK)))
    return Instance(res, 100.0, 100, f"spreader3d-scaled-n{n}-eps100-minpts100-f32")
