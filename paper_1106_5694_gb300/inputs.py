"""Seeded synthetic inputs for the LSAP solver and its tests.

This module holds only input generation -- none of the solver's arithmetic --
so that the CUDA path and the CPU oracle can be fed the very same host
buffer.  All generators are numpy PCG64 streams keyed by an integer seed.

Workloads (benefit matrices are n x n int32, row = agent, column = job):

* ``uniform(n, lo, hi, seed)`` -- i.i.d. integers in [lo, hi).
* ``peer_shaped(n, seed)`` -- the peer-assignment shape of the P2P streaming
  scenario that motivates the paper (Section 1): agents and jobs get random
  positions in the unit square and log-uniform capacities in [1, 100];
  b[i, j] = floor(1e4 * min(up_i, down_j) / 100 * exp(-4 * dist(i, j)))
  plus uniform integer noise in [0, 16).  Values lie in [0, 10015]; ties are
  frequent, which exercises every tie-break rule.
* ``geom(n, c, seed)`` -- the GEOM family of the paper's evaluation
  (Section 4): n random points in [0, c]^2, a_ij = Euclidean distance between
  points i and j, floored to an integer.
* ``batched_sizes`` / ``poisson_arrivals`` -- size and arrival mixes for the
  batched and served workloads.
"""
from __future__ import annotations

import numpy as np

MAX_ABS_BENEFIT = 1 << 29  # every |a| must be below this (gains fit int32)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def uniform(n: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """n x n int32 benefits i.i.d. uniform in [lo, hi)."""
    return _rng(seed).integers(lo, hi, size=(n, n), dtype=np.int32)


def peer_shaped(n: int, seed: int, chunk_rows: int = 2048) -> np.ndarray:
    """n x n int32 peer-assignment benefits (see module docstring)."""
    rng = _rng(seed)
    agent_xy = rng.random((n, 2))
    job_xy = rng.random((n, 2))
    up = np.exp(rng.uniform(0.0, np.log(100.0), size=n))
    down = np.exp(rng.uniform(0.0, np.log(100.0), size=n))
    noise_rng = _rng(seed ^ 0x5EED5EED)
    out = np.empty((n, n), dtype=np.int32)
    for r0 in range(0, n, chunk_rows):
        r1 = min(n, r0 + chunk_rows)
        d = np.sqrt(((agent_xy[r0:r1, None, :] - job_xy[None, :, :]) ** 2).sum(-1))
        cap = np.minimum(up[r0:r1, None], down[None, :])
        base = np.floor(1e4 * cap / 100.0 * np.exp(-4.0 * d)).astype(np.int32)
        out[r0:r1] = base + noise_rng.integers(0, 16, size=(r1 - r0, n), dtype=np.int32)
    return out


def geom(n: int, c: float, seed: int) -> np.ndarray:
    """GEOM instance: floored Euclidean distances between n random points in [0,c]^2."""
    p = _rng(seed).random((n, 2)) * c
    d = np.sqrt(((p[:, None, :] - p[None, :, :]) ** 2).sum(-1))
    return np.floor(d).astype(np.int32)


def identity_like(n: int, big: int, small_hi: int, seed: int):
    """Planted optimum: a[i, pi(i)] = big, all other entries in [0, small_hi).

    Returns (a, pi) with pi a seeded permutation (agent -> job)."""
    rng = _rng(seed)
    a = rng.integers(0, small_hi, size=(n, n), dtype=np.int32)
    pi = rng.permutation(n).astype(np.int32)
    a[np.arange(n), pi] = big
    return a, pi


def random_permutation(n: int, seed: int) -> np.ndarray:
    """A seeded permutation (used as a caller-supplied initial assignment)."""
    return _rng(seed).permutation(n).astype(np.int32)


def batched_sizes(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Instance sizes log-uniform in [lo, hi] (int32)."""
    u = _rng(seed).uniform(np.log(lo), np.log(hi + 1), size=count)
    return np.clip(np.floor(np.exp(u)), lo, hi).astype(np.int32)


def poisson_arrivals(count: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Arrival times (seconds, float64) of a Poisson stream."""
    gaps = _rng(seed).exponential(1.0 / rate_per_s, size=count)
    return np.cumsum(gaps)
