"""The GPU parity tolerance, checked against the arithmetic it is derived from.

The p-norm parity tests bound the relative error of each p-sum by s_tol: the
FP32 squaring chain, the cast of the powered operand to the tensor-core format,
flushes that tau allows, and FP32 accumulation.  Here that arithmetic is
emulated on the CPU (numpy FP32 squarings, round-to-nearest-even casts done on
the bits, exact products, sequential FP32 accumulation -- a worse order than
the tensor cores' tree) and compared with the FP64 oracle: every stable sum
must fall inside s_tol, and every estimate inside pnorm_tol; with few terms
the emulated error comes within a factor of about 3 of the bound.
"""
import numpy as np
import pytest

import workloads

pytest.importorskip("torch")
from test_gpu_product import pnorm_tol, s_tol  # noqa: E402


def _round_mantissa(x, keep):
    """Round FP32 values to `keep` explicit mantissa bits, nearest-even."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    drop = 23 - keep
    half = np.uint64((1 << (drop - 1)) - 1)
    b = (b + half + ((b >> np.uint64(drop)) & np.uint64(1))) & ~np.uint64((1 << drop) - 1)
    return b.astype(np.uint32).view(np.float32)


_KEEP = {"bf16": 7, "tf32": 10}


def _emulated_sums(A, B, r, c, plogs, mode):
    a = (A / r[:, None]).astype(np.float32)  # power-of-two scales: exact
    b = (B / c[None, :]).astype(np.float32)
    out = []
    for lp in plogs:
        x, y = a.copy(), b.copy()
        for _ in range(lp):  # x^p by log2(p) FP32 squarings
            x = (x * x).astype(np.float32)
            y = (y * y).astype(np.float32)
        x, y = _round_mantissa(x, _KEEP[mode]), _round_mantissa(y, _KEEP[mode])
        terms = (x[:, :, None].astype(np.float64) * y[None, :, :])  # exact in FP32 too
        S = np.add.accumulate(terms.astype(np.float32), axis=1, dtype=np.float32)[:, -1, :]
        out.append(S.astype(np.float64))
    return np.array(out)


@pytest.mark.parametrize("mode", ["bf16", "tf32"])
@pytest.mark.parametrize("K", [1, 5, 40, 700])
def test_emulated_sums_inside_the_parity_tolerance(orc, mode, K):
    A, B = workloads.wide_range_pair(24, 20, K, seed=3100 + K)
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    pl = list(range(7))
    tau = orc.default_tau(K, {"bf16": orc.BF16, "tf32": orc.TF32}[mode])
    ref = orc.pnorm(A64, B64, pl, tau, want_S=True)
    S_emu = _emulated_sums(A64, B64, ref["r"], ref["c"], pl, mode)
    worst = 0.0
    for q, lp in enumerate(pl):
        S = ref["S"][q]
        ok = S >= tau
        err = np.abs(S_emu[q][ok] - S[ok]) / S[ok]
        bound = s_tol(mode, K, lp)
        assert np.all(err <= bound), (mode, K, lp, err.max(), bound)
        worst = max(worst, float(err.max() / bound))
    assert worst > 0.01  # the bound is not vacuous for this arithmetic
    # the estimate at the oracle's p*, through the root and the scales
    q = (ref["p_sel"] & 0x7F).astype(np.int64)
    S_at = np.take_along_axis(S_emu, q[None], 0)[0]
    C = ref["r"][:, None] * ref["c"][None, :] * np.power(S_at, 1.0 / 2.0 ** q)
    tol = np.vectorize(lambda lp: pnorm_tol(mode, K, int(lp)))(q)
    assert np.all(np.abs(C - ref["C"]) / ref["C"] <= tol)


@pytest.mark.parametrize("mode", ["bf16", "tf32"])
def test_the_bound_is_within_a_small_factor(orc, mode):
    """Few terms (K = 1, 2, 5), where one product's cast error is not averaged
    away: the emulated error reaches at least 30 % of s_tol at some p, so the
    bound is at most about 3x loose there.  At these sizes s_tol is almost all
    cast term 2u plus flush term 2^-m, which are equal for BF16 and TF32; the
    flush term holds even where nothing is flushed, so either term alone would
    still cover the emulated error (up to about 90 % of it)."""
    for K in (1, 2, 5):
        A, B = workloads.wide_range_pair(24, 20, K, seed=3100 + K)
        A64, B64 = A.astype(np.float64), B.astype(np.float64)
        pl = list(range(7))
        ref = orc.pnorm(A64, B64, pl, 1e-300, want_S=True)
        S_emu = _emulated_sums(A64, B64, ref["r"], ref["c"], pl, mode)
        ratio = max(float((np.abs(S_emu[q] - ref["S"][q]) / ref["S"][q]).max() / s_tol(mode, K, lp))
                    for q, lp in enumerate(pl))
        assert 0.3 <= ratio <= 1.0, (mode, K, ratio)
