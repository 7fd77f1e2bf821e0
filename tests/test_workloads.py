"""The seeded input generators follow the recipes they state: ranges, the
distributions (Kolmogorov-Smirnov against the stated law), APSP edge density
and diagonal, the log-uniform grouped sizes, and determinism per seed."""
import numpy as np
import pytest

import workloads

stats = pytest.importorskip("scipy.stats")


def test_uniform_pair_is_uniform_on_open_closed_unit_interval():
    A, B = workloads.uniform_pair(300, 200, 100)
    assert A.shape == (300, 100) and B.shape == (100, 200) and A.dtype == np.float32
    for X in (A, B):
        assert X.min() > 0.0 and X.max() <= 1.0
        assert stats.kstest(X.ravel()[:20000].astype(np.float64), "uniform").pvalue > 1e-3
    A2, B2 = workloads.uniform_pair(300, 200, 100)
    assert np.array_equal(A, A2) and np.array_equal(B, B2)
    A3, _ = workloads.uniform_pair(300, 200, 100, seed=5)
    assert not np.array_equal(A, A3)


def test_wide_range_pair_is_exp_of_minus_exponential_rate_4():
    A, B = workloads.wide_range_pair(200, 150, 100)
    for X in (A, B):
        assert X.min() > 0.0 and X.max() <= 1.0
        e = -np.log(X.ravel()[:20000].astype(np.float64))
        assert stats.kstest(e, "expon", args=(0.0, 0.25)).pvalue > 1e-3
    ii, jj = workloads.wide_range_entries(16384, 4096)
    assert ii.min() >= 0 and ii.max() < 16384 and jj.min() >= 0 and jj.max() < 16384
    assert len(np.unique(ii * 16384 + jj)) > 4000


def test_apsp_weights_density_diagonal_and_range():
    n = 1000
    W = workloads.apsp_weights(n, density=0.1)
    assert np.all(np.diag(W) == 0.0)
    off = ~np.eye(n, dtype=bool)
    finite = np.isfinite(W) & off
    frac = finite.sum() / off.sum()
    assert abs(frac - 0.1) < 4 * np.sqrt(0.1 * 0.9 / off.sum())
    w = W[finite].astype(np.float64)
    assert w.min() >= 0.0 and w.max() < 1.0
    assert stats.kstest(w[:20000], "uniform").pvalue > 1e-3
    assert np.all(np.isinf(W[off & ~finite]) & (W[off & ~finite] > 0))
    rows = workloads.sampled_rows(n, 64)
    assert len(rows) == 64 and len(np.unique(rows)) == 64 and np.all(np.diff(rows) > 0)


def test_grouped_sizes_are_log_uniform_between_16_and_1024():
    s = workloads.grouped_sizes(4096)
    assert s.dtype == np.int64 and s.min() >= 16 and s.max() <= 1024
    u = np.log(s / 16.0) / np.log(64.0)
    # rounding to integers perturbs u by at most 1/(2 n ln 64) <= 0.0113
    assert stats.kstest(u, "uniform").statistic < 0.0113 + 1.63 / np.sqrt(len(u))
    assert np.array_equal(s, workloads.grouped_sizes(4096))
    probs = workloads.grouped_problems(s[:5])
    for n, (A, B) in zip(s[:5], probs):
        assert A.shape == (n, n) and B.shape == (n, n) and A.min() > 0 and B.max() <= 1
