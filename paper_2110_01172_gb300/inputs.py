"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module only draws random numbers and shapes; it contains none of the
transform arithmetic, so the GPU library and the CPU oracle can both be fed
from it without sharing any of the method's code.

Workload recipes (arXiv 2110.01172 measures on random matrices of the shapes in
Table V and on ISPD 2005 placement density maps, Table VII; the density maps
are not available, so seeded Gaussian-blob maps stand in for them):

* ``uniform``: i.i.d. U[-1, 1] drawn in float64 by ``numpy.random.default_rng``
  and rounded to float32.
* ``gaussian_bumps``: a smooth field, the sum of ``n_bumps`` isotropic Gaussian
  bumps with centres uniform over the grid, widths sigma ~ U[0.01, 0.05] times
  the array width and amplitudes ~ U[-1, 1].
* ``density_blobs``: a nonnegative density map made of ``n_blobs`` Gaussian
  blobs (sigma ~ U[1%, 5%] of the shorter side, weights ~ U[0.1, 1]).
* ``batched_shapes``: 2D shapes whose sides are powers of two drawn with a
  uniform exponent between 64 and 1024, half squares and half 1:2 rectangles.
* ``poisson_arrivals``: arrival times of a Poisson process (exponential gaps).
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "uniform", "gaussian_bumps", "density_blobs", "batched_shapes",
    "poisson_arrivals", "serving_shapes",
]


def uniform(shape, seed: int = 0) -> np.ndarray:
    """i.i.d. U[-1, 1] values, drawn in float64 and rounded to float32."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=tuple(shape)).astype(np.float32)


def _separable_bump_sum(shape, centres, sigmas, weights) -> np.ndarray:
    n1, n2 = shape
    r1 = np.arange(n1, dtype=np.float64)
    r2 = np.arange(n2, dtype=np.float64)
    out = np.zeros((n1, n2), dtype=np.float64)
    for (c1, c2), s, w in zip(centres, sigmas, weights):
        g1 = np.exp(-0.5 * ((r1 - c1) / s) ** 2)
        g2 = np.exp(-0.5 * ((r2 - c2) / s) ** 2)
        out += w * np.outer(g1, g2)
    return out


def gaussian_bumps(shape, seed: int = 0, n_bumps: int = 32) -> np.ndarray:
    """Smooth field: sum of ``n_bumps`` Gaussian bumps, float32."""
    n1, n2 = shape
    rng = np.random.default_rng(seed)
    centres = np.stack([rng.uniform(0, n1, n_bumps), rng.uniform(0, n2, n_bumps)], 1)
    sigmas = rng.uniform(0.01, 0.05, n_bumps) * n2
    weights = rng.uniform(-1.0, 1.0, n_bumps)
    return _separable_bump_sum(shape, centres, sigmas, weights).astype(np.float32)


def density_blobs(shape, seed: int = 0, n_blobs: int | None = None) -> np.ndarray:
    """Nonnegative density map of Gaussian blobs (100-2000 of them), float32."""
    n1, n2 = shape
    rng = np.random.default_rng(seed)
    if n_blobs is None:
        n_blobs = int(rng.integers(100, 2001))
    centres = np.stack([rng.uniform(0, n1, n_blobs), rng.uniform(0, n2, n_blobs)], 1)
    sigmas = rng.uniform(0.01, 0.05, n_blobs) * min(n1, n2)
    weights = rng.uniform(0.1, 1.0, n_blobs)
    return _separable_bump_sum(shape, centres, sigmas, weights).astype(np.float32)


def batched_shapes(count: int, seed: int = 0, lo: int = 64, hi: int = 1024):
    """``count`` 2D shapes, power-of-two sides between ``lo`` and ``hi``.

    Each shape is a square (n, n) or a 1:2 rectangle (n, 2n) / (2n, n) with
    equal probability; the side exponent is uniform, so sides are log-uniform.
    """
    rng = np.random.default_rng(seed)
    elo, ehi = int(np.log2(lo)), int(np.log2(hi))
    shapes = []
    for _ in range(count):
        kind = int(rng.integers(0, 3))
        if kind == 0:
            e = int(rng.integers(elo, ehi + 1))
            shapes.append((1 << e, 1 << e))
        else:
            e = int(rng.integers(elo, ehi))  # the long side 2n stays <= hi
            n = 1 << e
            shapes.append((n, 2 * n) if kind == 1 else (2 * n, n))
    return shapes


def serving_shapes(count: int, seed: int = 0, lo: int = 64, hi: int = 2048):
    """Request shapes with N1, N2 drawn independently from {lo, 2 lo, ..., hi}."""
    rng = np.random.default_rng(seed)
    elo, ehi = int(np.log2(lo)), int(np.log2(hi))
    e = rng.integers(elo, ehi + 1, size=(count, 2))
    return [(1 << int(a), 1 << int(b)) for a, b in e]


def poisson_arrivals(count: int, rate_per_s: float, seed: int = 0) -> np.ndarray:
    """Arrival times (seconds, from 0) of a Poisson process of the given rate."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=count)
    return np.cumsum(gaps) - gaps[0]
