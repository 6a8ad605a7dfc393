"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the solver: only a counter-based random
number generator and the geometry/recipes of the synthetic workloads
(channel and duct grids stretched by a tanh law, i.i.d. uniform or Gaussian
fields).  Both the CPU oracle and the GPU path read the bytes produced here,
so they see identical inputs.

Random numbers: SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) evaluated at counter
``seed * 2**32 + i``; uniform doubles take the top 53 bits; Gaussians use the
Box-Muller transform on two consecutive counters.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22


def splitmix64(counter: np.ndarray) -> np.ndarray:
    """SplitMix64 output for each uint64 counter value (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = counter * _GOLDEN + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _counters(seed: int, start: int, count: int) -> np.ndarray:
    base = np.uint64((int(seed) & 0xFFFFFFFF) << 32)
    return base + np.arange(start, start + count, dtype=np.uint64)


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles in [0, 1) from counters offset..offset+n-1 of stream ``seed``."""
    out = np.empty(n, dtype=np.float64)
    for s in range(0, n, _CHUNK):
        c = min(_CHUNK, n - s)
        z = splitmix64(_counters(seed, offset + s, c))
        out[s:s + c] = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return out


def uniform(seed: int, shape, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    n = int(np.prod(shape))
    return (lo + (hi - lo) * uniform01(seed, n)).reshape(shape)


def gaussian(seed: int, shape, sigma: float = 1.0) -> np.ndarray:
    """Box-Muller: element i uses counters 2i (radius) and 2i+1 (angle)."""
    n = int(np.prod(shape))
    out = np.empty(n, dtype=np.float64)
    for s in range(0, n, _CHUNK):
        c = min(_CHUNK, n - s)
        u = uniform01(seed, 2 * c, offset=2 * s)
        u1 = 1.0 - u[0::2]               # (0, 1]
        u2 = u[1::2]
        out[s:s + c] = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)
    return (sigma * out).reshape(shape)


def remove_mean(f: np.ndarray, weights_z: np.ndarray | None = None) -> np.ndarray:
    """Subtract the (optionally z-weighted) mean; input preparation, not the solver."""
    if weights_z is None:
        return f - f.mean()
    w = weights_z.reshape(-1, 1, 1)
    return f - (f * w).sum() / (w.sum() * f.shape[1] * f.shape[2])


def tanh_faces(nz: int, beta: float, length: float = 2.0) -> np.ndarray:
    """Wall-normal faces z_k = L/2 * (1 + tanh(beta (2k/nz - 1)) / tanh(beta)), k=0..nz.

    beta <= 0 gives a uniform grid.
    """
    k = np.arange(nz + 1, dtype=np.float64)
    if beta <= 0.0:
        return length * k / nz
    return 0.5 * length * (1.0 + np.tanh(beta * (2.0 * k / nz - 1.0)) / math.tanh(beta))


def velocity_field(seed: int, nx: int, ny: int, nz: int, sigma: float = 1.0):
    """Gaussian staggered velocity (u at x-faces, v at y-faces, w at z-faces).

    u, v: [nz][ny][nx] (face i+1/2 / j+1/2 of cell (i,j,k)); w: [nz+1][ny][nx]
    with the wall values w[0] = w[nz] = 0 (impermeable walls).
    """
    u = gaussian(seed, (nz, ny, nx), sigma)
    v = gaussian(seed + 1, (nz, ny, nx), sigma)
    w = gaussian(seed + 2, (nz + 1, ny, nx), sigma)
    w[0] = 0.0
    w[nz] = 0.0
    return u, v, w


# Workload shapes (periodic x, y unless stated; lengths of the domain).
CHANNEL = dict(lx=2.0 * math.pi, ly=math.pi, lz=2.0)
DUCT = dict(lx=6.0, ly=2.0, lz=2.0)

BATCH_DOMAINS = [
    (64, 64, 64), (80, 64, 64), (96, 64, 80), (96, 96, 80),
    (128, 64, 96), (128, 96, 96), (160, 96, 96), (160, 128, 96),
    (192, 96, 128), (192, 128, 128), (240, 128, 128), (256, 128, 128),
    (256, 160, 128), (320, 160, 144), (320, 192, 160), (384, 192, 160),
]
