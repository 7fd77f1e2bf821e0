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
_CODE = {"tf32": 1, "bf16": 2, "f16": 3, "e4m3": 4}


def _cast(x, mode):
    """The powered operand as the tensor cores read it: BF16 / TF32 by mantissa
    rounding; FP16 and E4M3 after the operand shift 2^15 / 2^8 that moves
    [0, 1] into their range (undone here), nearest-even, with subnormals
    (E4M3: quantum 2^-9 below 2^-6)."""
    if mode in _KEEP:
        return _round_mantissa(x, _KEEP[mode])
    if mode == "f16":
        return ((x.astype(np.float64) * 2.0 ** 15).astype(np.float16).astype(np.float64)
                / 2.0 ** 15).astype(np.float32)
    v = x.astype(np.float64) * 2.0 ** 8
    e = np.floor(np.log2(np.where(v > 0, v, 1.0)))
    q = 2.0 ** (np.maximum(e, -6) - 3)
    v = np.minimum(np.round(v / q) * q, 448.0)
    return (v / 2.0 ** 8).astype(np.float32)


def _emulated_sums(A, B, r, c, plogs, mode):
    a = (A / r[:, None]).astype(np.float32)  # power-of-two scales: exact
    b = (B / c[None, :]).astype(np.float32)
    out = []
    for lp in plogs:
        x, y = a.copy(), b.copy()
        for _ in range(lp):  # x^p by log2(p) FP32 squarings
            x = (x * x).astype(np.float32)
            y = (y * y).astype(np.float32)
        x, y = _cast(x, mode), _cast(y, mode)
        terms = (x[:, :, None].astype(np.float64) * y[None, :, :])  # exact in FP32 too
        S = np.add.accumulate(terms.astype(np.float32), axis=1, dtype=np.float32)[:, -1, :]
        out.append(S.astype(np.float64))
    return np.array(out)


@pytest.mark.parametrize("mode", ["bf16", "tf32", "f16", "e4m3"])
@pytest.mark.parametrize("K", [1, 5, 40, 700])
def test_emulated_sums_inside_the_parity_tolerance(orc, mode, K):
    A, B = workloads.wide_range_pair(24, 20, K, seed=3100 + K)
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    pl = list(range(7))
    tau = orc.default_tau(K, _CODE[mode])
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


def _emulated_power(x, lp, half):
    """x^(2^lp) by FP32 squarings, times its FP32 square root for the half
    levels 1.5 * 2^lp (as the operand images form them)."""
    for _ in range(lp):
        x = (x * x).astype(np.float32)
    if half:
        x = (x * np.sqrt(x, dtype=np.float32)).astype(np.float32)
    return x


def _emulated_sum(a, b, lp, half, mode):
    x = _cast(_emulated_power(a, lp, half), mode)
    y = _cast(_emulated_power(b, lp, half), mode)
    terms = (x[:, :, None].astype(np.float64) * y[None, :, :]).astype(np.float32)
    return np.add.accumulate(terms, axis=1, dtype=np.float32)[:, -1, :].astype(np.float64)


def _library_r2(orc, s, pp, eta):
    """The library's r = 2 evaluation of (rounded) sums s: the r = 1 value
    where t3 - 1 = s1 s3 / s2^2 - 1 does not clear its margin eta, else the
    projection."""
    s1, s2, s3, s4 = s
    t3 = s1 * s3 / s2 ** 2 - 1
    return np.where(t3 > eta, orc.project_r2(s1, s2, s3, s4, pp), (s2 / s1) ** (1 / pp))


@pytest.mark.parametrize("mode", ["bf16", "tf32", "f16", "e4m3"])
@pytest.mark.parametrize("K", [5, 40, 700])
def test_r2_bounds_hold_the_emulated_projection(orc, mode, K):
    """The r = 2 parity bounds: the projection of sums carrying the emulated
    GPU arithmetic stays inside r2_bounds built from the exact sums, both in
    the well-resolved band (strong) and in the r = 1 .. plain bracket."""
    from test_gpu_projection_r2 import _ETA, r2_bounds
    A, B = workloads.wide_range_pair(24, 20, K, seed=3200 + K)
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    pl = list(range(7))
    tau = orc.default_tau(K, _CODE[mode])
    ref = orc.pnorm(A64, B64, pl, tau, want_S=True, estimator=2)
    r, c = ref["r"], ref["c"]
    a = (A64 / r[:, None]).astype(np.float32)
    b = (B64 / c[None, :]).astype(np.float32)
    n_strong = 0
    for ls in range(2, 7):
        sel = ((ref["p_sel"] & 0x7F) == ls) & ((ref["p_sel"] & 0x80) == 0)
        if not sel.any():
            continue
        ps = 2.0 ** ls
        exact = [ref["S"][ls - 2], ref["S"][ls - 1],
                 orc.psums_real(A64, B64, [0.75 * ps], r, c)[0], ref["S"][ls]]
        emu = [_emulated_sum(a, b, ls - 2, 0, mode), _emulated_sum(a, b, ls - 1, 0, mode),
               _emulated_sum(a, b, ls - 1, 1, mode), _emulated_sum(a, b, ls, 0, mode)]
        s = np.stack([e[sel] for e in exact])
        lo, hi, strong = r2_bounds(orc, s, ps, mode, K, tau)
        v = _library_r2(orc, [e[sel] for e in emu], ps / 4, _ETA[mode])
        assert np.all((v >= lo) & (v <= hi)), (mode, K, ls)
        n_strong += int(strong.sum())
    # the corner band, not only the bracket, is exercised -- except in E4M3,
    # whose margin eta = 2 is never cleared (every entry keeps the r = 1 value)
    assert (n_strong > 0) == (mode != "e4m3")


@pytest.mark.parametrize("mode", ["bf16", "tf32", "f16", "e4m3"])
@pytest.mark.parametrize("K", [1, 5, 40, 700])
def test_r1_tolerance_holds_the_emulated_projection(orc, mode, K):
    """The r = 1 parity tolerance: (S^(p*) / S^(p*/2))^(2/p*) from sums carrying
    the emulated GPU arithmetic stays within proj_tol of the oracle's
    projection at every projected entry."""
    from test_gpu_projection import proj_tol
    A, B = workloads.wide_range_pair(24, 20, K, seed=3300 + K)
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    pl = list(range(7))
    tau = orc.default_tau(K, _CODE[mode])
    ref = orc.pnorm(A64, B64, pl, tau, want_S=True, estimator=1)
    S_emu = _emulated_sums(A64, B64, ref["r"], ref["c"], pl, mode)
    rc = ref["r"][:, None] * ref["c"][None, :]
    checked = 0
    for ls in range(1, 7):
        sel = ((ref["p_sel"] & 0x7F) == ls) & ((ref["p_sel"] & 0x80) == 0)
        if not sel.any():
            continue
        v = rc[sel] * (S_emu[ls][sel] / S_emu[ls - 1][sel]) ** (2.0 / 2 ** ls)
        err = np.abs(v - ref["C"][sel]) / ref["C"][sel]
        assert np.all(err <= proj_tol(mode, K, ls)), (mode, K, ls, err.max())
        checked += int(sel.sum())
    assert checked > 0


def test_fft_bound_holds_for_a_standard_fft(orc):
    """The max-convolution tests bound one FP64 FFT convolution output by
    E = 4 log2(N) 2^-53 (|a|_1 |b|_2 + |b|_1 |a|_2); numpy's FP64 FFT of the
    powered, max-scaled vectors stays inside it against the oracle's naive
    convolution (the bound is loose for an accurate FFT: numpy uses under 5 %)."""
    import math
    from test_gpu_maxconv import _fft_err
    g = workloads.rng(3400)
    for nx, ny in ((37, 20), (1000, 1500), (6000, 5000), (3, 40000)):
        x, y = 1.0 - g.random(nx), 1.0 - g.random(ny)
        nz = nx + ny - 1
        N = max(2, 1 << math.ceil(math.log2(nz)))
        for p in (1, 8, 64):
            a, b = (x / x.max()) ** p, (y / y.max()) ** p
            w = orc.conv(a, b)[0]
            f = np.fft.irfft(np.fft.rfft(a, N) * np.fft.rfft(b, N), N)[:nz]
            assert np.abs(f - w).max() <= _fft_err(a, b, N), (nx, ny, p)


def _split_3xtf32(x):
    hi = _round_mantissa(x, 10)
    lo = _round_mantissa((x - hi).astype(np.float32), 10)
    return hi, lo


def _gemm_3xtf32(X, Y):
    """X (m x l) @ Y (l x n) as three TF32 products (each exact in FP32),
    accumulated sequentially in FP32 over l."""
    xh, xl = _split_3xtf32(X)
    yh, yl = _split_3xtf32(Y)
    t = (xh[:, :, None].astype(np.float64) * yh[None] + xh[:, :, None].astype(np.float64) * yl[None]
         + xl[:, :, None].astype(np.float64) * yh[None])
    return np.add.accumulate(t.astype(np.float32), axis=1, dtype=np.float32)[:, -1, :]


def _grad_factor(acc, x, s, k):
    """The gradient epilogue's acc * x'^(p-1) / s, x' = x / s, p = 2^k, in FP32:
    x' split into mantissa and exponent (frexp), the chain x' x'^2 ... run on
    mantissas in [0.5, 1) with every product renormalised and the exponents
    summed exactly, the total exponent applied once (one rounding)."""
    ls = np.frexp(s)[1] - 1
    xm, ex = np.frexp(x)
    ex = ex - ls
    rm = np.ones_like(x)
    re = np.zeros(x.shape, dtype=np.int64)
    for _ in range(k):
        rm, d = np.frexp((rm * xm).astype(np.float32))
        re = re + ex + d
        xm, d = np.frexp((xm * xm).astype(np.float32))
        ex = 2 * ex + d
    return np.ldexp((acc * rm).astype(np.float32).astype(np.float64), re - ls).astype(np.float32)


@pytest.mark.parametrize("shape,plog",
                         [((64, 48, 80), 4), ((30, 20, 300), 2), ((40, 90, 33), 6)])
def test_adjoint_tolerance_holds_the_emulated_gradient(orc, shape, plog):
    """The adjoint's parity tolerance grad_tol: for L = sum log C at a fixed p,
    W = G C / S = 1 / S, dA = (W B'^pT) a'^(p-1) / r and dB = (A'^pT W) b'^(p-1) / c,
    emulated with FP32 sums, 3xTF32 products with FP32 accumulation and the
    gradient epilogue's factor (mantissa chain with separate exponents), stay
    within grad_tol of the FP64 oracle gradient, plus FP32's subnormal spacing
    2^-149 for exact entries below the FP32 range.  K = 33 at p = 64 is the case
    where a'^(p-1) itself leaves the FP32 range (a' < 0.25) while W = 1/S lifts
    many gradient entries back into it: every such entry is kept."""
    from test_gpu_backward import grad_ok, grad_tol
    M, N, K = shape
    A, B = workloads.uniform_pair(M, N, K, seed=3500 + M)
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    r, c = orc.row_scales(A64), orc.col_scales(B64)
    a = (A64 / r[:, None]).astype(np.float32)
    b = (B64 / c[None, :]).astype(np.float32)
    ap, bp = a.copy(), b.copy()
    for _ in range(plog):  # x^p by squaring
        ap, bp = (ap * ap).astype(np.float32), (bp * bp).astype(np.float32)
    S = _gemm_3xtf32(ap, bp)
    W = (np.float32(1.0) / S).astype(np.float32)
    r32, c32 = r.astype(np.float32), c.astype(np.float32)
    dA = _grad_factor(_gemm_3xtf32(W, bp.T), A, np.broadcast_to(r32[:, None], A.shape), plog)
    dB = _grad_factor(_gemm_3xtf32(ap.T, W), B, np.broadcast_to(c32[None, :], B.shape), plog)
    plogs = np.full((M, N), plog, dtype=np.uint8)
    Cref = orc.pnorm(A64, B64, [plog], 1e-300)["C"]
    gA, gB = orc.pnorm_grad(A64, B64, plogs, 1.0 / Cref)
    rescued = 0
    for d, g, x, L in ((dA, gA, a, N), (dB, gB, b, M)):
        assert grad_ok(d, g, grad_tol(plog, L)), (d, g)
        # entries whose factor x'^(p-1) lies below FP32's normal range but whose
        # gradient does not: lost by a plain FP32 product of the squarings
        rescued += int(np.sum((x.astype(np.float64) ** (2 ** plog - 1) < 2.0 ** -126)
                              & (g >= 2.0 ** -126)))
    if plog == 6:
        assert rescued > 0


def _grad_factor_fast(acc, x, s, k):
    """The gradient epilogue's fast path: the plain FP32 chain with x' = x 2^-E
    (s = 2^E), used where s has a normal reciprocal and x'^(2^k - 1), acc times
    it and the result are normal; NaN marks entries that take the exponent-
    carrying path."""
    f32 = np.float32
    inv = (1.0 / s.astype(np.float64)).astype(np.float32)
    y = (x * inv).astype(f32)
    r = np.ones_like(y)
    for _ in range(k):
        r = (r * y).astype(f32)
        y = (y * y).astype(f32)
    ar = (acc * r).astype(f32)
    g = (ar * inv).astype(f32)
    fmin = f32(2.0 ** -126)
    ok = (r >= fmin) & (np.abs(ar) >= fmin) & (np.abs(g) >= fmin) & np.isfinite(g)
    return np.where(ok, g, np.nan).astype(f32)


@pytest.mark.parametrize("k", [0, 1, 3, 6])
def test_grad_factor_fast_path_matches_exponent_path(k):
    """Where the fast path applies it gives the same bits as the mantissa chain
    with separate exponents: over x' spread across enough binades that
    x'^(2^k - 1) leaves the FP32 range for part of them (so that both paths
    occur), random accumulators and power-of-two scales."""
    g = workloads.rng(None, 77 + k)
    n = 200000
    s = np.ldexp(np.ones(n, dtype=np.float32), g.integers(-60, 60, n)).astype(np.float32)
    xp = np.ldexp(g.random(n), -g.integers(0, max(2, 300 // 2 ** k), n))
    x = (xp * s).astype(np.float32)
    acc = (g.random(n) * np.ldexp(1.0, g.integers(-20, 20, n))).astype(np.float32)
    fast = _grad_factor_fast(acc, x, s, k)
    slow = _grad_factor(acc, x, s, k)
    used = ~np.isnan(fast)
    assert used.mean() > 0.2
    assert used.all() if k == 0 else (~used).sum() > 100
    assert np.array_equal(fast[used].view(np.uint32), slow[used].view(np.uint32))


def test_grad_factor_renormalisation_equals_frexp():
    """The gradient epilogue's exponent-carrying chain renormalises each
    product of two mantissas in [0.5, 1] by at most one doubling instead of
    calling frexp: the same mantissas and exponents, step by step."""
    g = workloads.rng(None, 91)
    f32 = np.float32
    xm = (0.5 + 0.5 * g.random(100000)).astype(f32)
    xm[:3] = [0.5, np.nextafter(f32(1), f32(0)), 0.75]
    rm_a = np.ones_like(xm)
    rm_b = np.ones_like(xm)
    ea = np.zeros(xm.shape, dtype=np.int64)
    eb = np.zeros(xm.shape, dtype=np.int64)
    xa, xb = xm.copy(), xm.copy()
    for _ in range(6):
        rm_a, d = np.frexp((rm_a * xa).astype(f32))
        ea += d
        xa = np.frexp((xa * xa).astype(f32))[0]
        p = (rm_b * xb).astype(f32)
        low = p < 0.5
        rm_b = np.where(low, p * 2, p).astype(f32)
        eb -= low
        xb = (xb * xb).astype(f32)
        xb = np.where(xb < 0.5, xb * 2, xb).astype(f32)
        assert np.array_equal(rm_a.view(np.uint32), rm_b.view(np.uint32))
        assert np.array_equal(xa.view(np.uint32), xb.view(np.uint32))
        assert np.array_equal(ea, eb)
