"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module only draws numbers; it holds none of the matrix-product arithmetic.
All generators run on the host with numpy's PCG64 so that the same seed gives
the same bytes on every machine.  The workload recipes mirror the shapes and
distributions the benchmarks use: uniform[-1, 1] square and rank-k matrices,
small integers in [-4, 4], Gaussian N(0, 1), and a badly scaled variant whose
rows of A and columns of B are multiplied by 10**u, u ~ U(-3, 3).
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform(shape, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """float32 uniform[lo, hi)."""
    g = rng(seed)
    x = g.random(shape, dtype=np.float32)
    x *= np.float32(hi - lo)
    x += np.float32(lo)
    return x


def small_int(shape, seed: int, lo: int = -4, hi: int = 4) -> np.ndarray:
    """float32 holding integers drawn uniformly from [lo, hi]."""
    g = rng(seed)
    return g.integers(lo, hi + 1, size=shape).astype(np.float32)


def gaussian(shape, seed: int) -> np.ndarray:
    """float32 N(0, 1)."""
    g = rng(seed)
    return g.standard_normal(shape, dtype=np.float32)


def badly_scaled(A: np.ndarray, B: np.ndarray, seed: int, span: float = 3.0):
    """Scale row i of A by 10**u_i and column j of B by 10**v_j, u, v ~ U(-span, span)."""
    g = rng(seed)
    u = g.uniform(-span, span, size=A.shape[0])
    v = g.uniform(-span, span, size=B.shape[1])
    As = (A.astype(np.float64) * (10.0 ** u)[:, None]).astype(np.float32)
    Bs = (B.astype(np.float64) * (10.0 ** v)[None, :]).astype(np.float32)
    return As, Bs


def problem(m: int, n: int, k: int, seed: int, dist: str = "uniform"):
    """(A, B) float32 of shapes (m, k) and (k, n) for a named distribution."""
    if dist == "uniform":
        return uniform((m, k), seed), uniform((k, n), seed + 1)
    if dist == "int":
        return small_int((m, k), seed), small_int((k, n), seed + 1)
    if dist == "gaussian":
        return gaussian((m, k), seed), gaussian((k, n), seed + 1)
    if dist == "badly_scaled":
        A, B = uniform((m, k), seed), uniform((k, n), seed + 1)
        return badly_scaled(A, B, seed + 2)
    raise ValueError(dist)


def uneven_batch(count: int, seed: int, lo: int = 1024, hi: int = 8192, step: int = 256):
    """``count`` (m, n, k) triples drawn uniformly from multiples of ``step`` in [lo, hi]."""
    g = rng(seed)
    vals = np.arange(lo, hi + 1, step)
    return [tuple(int(v) for v in g.choice(vals, size=3)) for _ in range(count)]
