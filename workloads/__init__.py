"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module only draws random numbers (numpy PCG64).  It holds none of the
method's arithmetic: no scaling, powering, transforms or products.  Seeds are
1511 + the workload's index unless a caller passes its own.

Workloads (shapes and distributions of the p-norm (x,max) product and APSP
problems the library targets):

* ``uniform_pair`` -- A (M x K), B (K x N) i.i.d. Uniform(0,1] (as 1 - U[0,1)).
* ``wide_range_pair`` -- entries exp(-Exponential(rate 4)) = U^(1/4): values
  near 1 that spread over many binades only once raised to large powers.
* ``apsp_weights`` -- dense directed graph: off-diagonal edges present with a
  given probability, weights Uniform[0,1] (or a given range), diagonal 0,
  missing edges +inf.
* ``grouped_sizes`` -- square sizes n = round(16 * 64^U), log-uniform in [16, 1024].
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 1511


def rng(seed: int | None = None, index: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + index if seed is None else seed))


def uniform_pair(M: int, N: int, K: int, seed: int | None = None, index: int = 0,
                 dtype=np.float32):
    g = rng(seed, index)
    A = (1.0 - g.random((M, K))).astype(dtype)
    B = (1.0 - g.random((K, N))).astype(dtype)
    return A, B


def wide_range_pair(M: int, N: int, K: int, rate: float = 4.0, seed: int | None = None,
                    index: int = 4, dtype=np.float32):
    """exp(-E), E ~ Exponential(rate): drawn as U^(1/rate) with U = 1 - U[0,1)."""
    g = rng(seed, index)
    A = np.power(1.0 - g.random((M, K)), 1.0 / rate).astype(dtype)
    B = np.power(1.0 - g.random((K, N)), 1.0 / rate).astype(dtype)
    return A, B


def wide_range_entries(n: int, count: int, seed: int | None = None, index: int = 4):
    """Sampled output coordinates for the large product (distinct from the data draw)."""
    g = rng(None if seed is None else seed + 7, index + 100)
    return g.integers(0, n, count), g.integers(0, n, count)


def apsp_weights(n: int, density: float = 0.1, lo: float = 0.0, hi: float = 1.0,
                 seed: int | None = None, index: int = 1, dtype=np.float32):
    g = rng(seed, index)
    W = (lo + (hi - lo) * g.random((n, n))).astype(dtype)
    mask = g.random((n, n)) < density
    W = np.where(mask, W, np.inf).astype(dtype)
    np.fill_diagonal(W, 0.0)
    return W


def sampled_rows(n: int, count: int, seed: int | None = None, index: int = 1):
    g = rng(None if seed is None else seed + 11, index + 100)
    return np.sort(g.choice(n, size=min(count, n), replace=False))


def grouped_sizes(count: int = 4096, lo: int = 16, hi: int = 1024, seed: int | None = None,
                  index: int = 3):
    g = rng(seed, index)
    u = g.random(count)
    return np.rint(lo * np.power(hi / lo, u)).astype(np.int64)


def grouped_problems(sizes, seed: int | None = None, index: int = 3):
    """One (A, B) Uniform(0,1] FP32 pair per square size."""
    g = rng(None if seed is None else seed + 1, index + 200)
    out = []
    for n in sizes:
        n = int(n)
        A = (1.0 - g.random((n, n))).astype(np.float32)
        B = (1.0 - g.random((n, n))).astype(np.float32)
        out.append((A, B))
    return out
