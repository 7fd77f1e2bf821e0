"""GPU parity of the r = 2 multiset-projection estimator (Sec. 2.1,
pn_opts.estimator = 2) against the FP64 oracle, through the C ABI.

The estimate at p* is a function of the four sums at p*/4, p*/2, 3p*/4 and
p*: the larger root of a small Prony system, clamped between the r = 1 value
and the plain norm (the interval of the larger Gauss node).  The oracle
projects its exact FP64 sums (Sec. 2.1 as written; its margin 1e-6 only
guards FP64 rounding).  The library's sums carry the operand format's
rounding, so it keeps the r = 1 value where t3 - 1 = s1 s3 / s2^2 - 1 is
below eta = 32 u of the format; that fallback lives only in the acceptance
band below, never in the oracle.  Bounds: every sum may carry its relative
error d_m (operand rounding, squaring chains, FP32 accumulation, the flush
allowance 2^-m tau / S, as in the plain-estimator tests).  Where the oracle's
t3 - 1 clears both eta and 8 times the sums' error of t3 (the system is well
resolved), the library's value must lie within the smallest and largest
oracle projection over the 16 corners of the error box (widened by 10 % of
its width, plus 1e-4 for the library's FP32 evaluation of the projection).
Elsewhere it must lie between the r = 1 value and the plain norm over that
box, which holds the library's r = 1 fallback.
"""
import itertools

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

_U = {"f32": 2.0 ** -21, "tf32": 2.0 ** -11, "bf16": 2.0 ** -8, "f16": 2.0 ** -11, "e4m3": 2.0 ** -4}
_M = {"f32": 21, "tf32": 10, "bf16": 7, "f16": 10, "e4m3": 3}
_CODE = {"f32": 0, "tf32": 1, "bf16": 2, "f16": 3, "e4m3": 4}


@pytest.fixture(scope="module")
def pn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1511_05690_gb300 as pn
    pn.lib()
    return pn


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


# the library's resolution margin, 32 u of the operand format (not the oracle's)
_ETA = {"f32": 2.0 ** -16, "tf32": 2.0 ** -6, "bf16": 2.0 ** -3, "f16": 2.0 ** -6, "e4m3": 2.0}


def s_tol(mode, K, p):
    """Relative error bound of a GPU p-sum at (real) p."""
    return 2 * (p - 1) * 2.0 ** -24 + 2 * _U[mode] + 2.0 ** -_M[mode] + K * 2.0 ** -23


def sum_tol(mode, K, p, S, tau):
    """The same for a sum S well above tau: the flush allowance is 2^-m tau / S."""
    return 2 * (p - 1) * 2.0 ** -24 + 2 * _U[mode] + 2.0 ** -_M[mode] * tau / S + K * 2.0 ** -23


def plain_tol(mode, K, plog):
    return 1.5 * ((1 + s_tol(mode, K, 2.0 ** plog)) ** (1.0 / 2 ** plog) - 1) + 2e-7


EPS = 1e-4 + 2.0 ** -21  # the library's FP32 projection, root and scale


def r2_bounds(orc, s, p_star, mode, K, tau):
    """s: (4, n) sums at p*/4, p*/2, 3p*/4, p*.  Returns (lo, hi, strong):
    the corner band where the system is well resolved (strong), else the
    r = 1 .. plain bracket over the error box."""
    d = np.stack([sum_tol(mode, K, p_star * f, s[m], tau)
                  for m, f in enumerate((0.25, 0.5, 0.75, 1.0))])
    eta = _ETA[mode]
    t3 = s[2] * s[0] / s[1] ** 2 - 1
    strong = t3 >= np.maximum(eta, 8 * (d[0] + d[2] + 2 * d[1]))
    vals = []
    for signs in itertools.product((-1.0, 1.0), repeat=4):
        sm = [s[m] * (1 + signs[m] * d[m]) for m in range(4)]
        vals.append(orc.project_r2(*sm, p_star / 4))
    vals = np.array(vals)
    lo, hi = vals.min(axis=0), vals.max(axis=0)
    w = hi - lo
    lo, hi = lo - 0.1 * w, hi + 0.1 * w
    pp = p_star / 4
    r1lo = (s[1] * (1 - d[1]) / (s[0] * (1 + d[0]))) ** (1 / pp)
    r1hi = (s[1] * (1 + d[1]) / (s[0] * (1 - d[0]))) ** (1 / pp)
    plhi = (s[3] * (1 + d[3])) ** (1 / p_star)
    lo = np.where(strong, lo, r1lo)
    hi = np.where(strong, hi, np.maximum(plhi, r1hi))
    return lo, hi, strong


def _chain(pl):
    """p_log2 values whose p/2 and p/4 are the two p below them in P."""
    return {pl[q] for q in range(2, len(pl)) if pl[q - 1] == pl[q] - 1 and pl[q - 2] == pl[q] - 2}


def _check(pn, orc, A, B, mode, pl, tau=None, tile_n=0):
    M, K = A.shape
    tau = orc.default_tau(K, _CODE[mode]) if tau is None else tau
    dA, dB = _dev(A), _dev(B)
    C, psel, ssel = pn.maxprod_pnorm(dA, dB, p_log2=pl, compute=mode, tau=tau, tile_n=tile_n,
                                     estimator=2)
    C0, psel0, ssel0 = pn.maxprod_pnorm(dA, dB, p_log2=pl, compute=mode, tau=tau, tile_n=tile_n,
                                        estimator=0)
    # p_sel and S_sel keep their meaning (p* and S^(p*)): identical to the plain run
    assert torch.equal(psel, psel0)
    assert torch.equal(ssel, ssel0)
    C, psel = C.cpu().numpy(), psel.cpu().numpy()
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    ref = orc.pnorm(A64, B64, pl, tau, want_S=True, estimator=2)
    r, c = ref["r"], ref["c"]
    S34 = orc.psums_real(A64, B64, [0.75 * 2.0 ** lp for lp in pl], r, c)
    near = np.zeros(C.shape, dtype=bool)
    for q, lp in enumerate(pl):
        near |= np.abs(ref["S"][q] / tau - 1) < 4 * s_tol(mode, K, 2.0 ** lp)
    agree = psel == ref["p_sel"]
    assert np.all(agree | near)
    lp_sel = (psel & 0x7F).astype(int)
    chain = _chain(pl)
    projected = np.isin(lp_sel, list(chain)) & ((psel & 0x80) == 0)
    ok = agree & (ref["C"] > 0)
    rc = r[:, None] * c[None, :]
    idx = {lp: q for q, lp in enumerate(pl)}
    checked = strong_n = 0
    for lp in chain:
        m = ok & projected & (lp_sel == lp)
        if not m.any():
            continue
        q = idx[lp]
        s = np.stack([ref["S"][q - 2][m], ref["S"][q - 1][m], S34[q][m], ref["S"][q][m]])
        lo, hi, strong = r2_bounds(orc, s, 2.0 ** lp, mode, K, tau)
        g = C[m] / rc[m]
        assert np.all(g >= lo * (1 - EPS)) and np.all(g <= hi * (1 + EPS)), (
            mode, lp, float(np.max(lo / g - 1)), float(np.max(g / hi - 1)))
        checked += int(m.sum())
        strong_n += int(strong.sum())
    plain = ok & ~projected
    tol = np.vectorize(lambda lp: plain_tol(mode, K, lp))(lp_sel)
    err = np.abs(C - ref["C"]) / np.maximum(ref["C"], 1e-300)
    assert np.all(err[plain] <= tol[plain]), float(err[plain].max())
    return C, psel, projected, checked, strong_n


@pytest.mark.parametrize("shape", [(1, 1, 1), (5, 7, 3), (130, 300, 257), (129, 77, 33),
                                   (200, 64, 500)])
def test_r2_f32_matches_oracle(pn, orc, shape):
    M, N, K = shape
    A, B = workloads.uniform_pair(M, N, K, seed=1900 + M)
    _check(pn, orc, A, B, "f32", list(range(7)))


def _multilevel_inputs(M, N, K, seed):
    g = workloads.rng(seed)
    A = (0.05 * (0.5 + 0.5 * g.random((M, K)))).astype(np.float32)
    B = (0.05 * (0.5 + 0.5 * g.random((K, N)))).astype(np.float32)
    A[np.arange(M), np.arange(M) % K] = 1.0
    B[(np.arange(N) + 1) % K, np.arange(N)] = 1.0
    return A, B


@pytest.mark.parametrize("mode", ["f32", "bf16"])
def test_r2_multilevel(pn, orc, mode):
    """p* spread over several levels: chains of different lengths share the
    half levels and the parked sums."""
    A, B = _multilevel_inputs(150, 170, 128, seed=1910)
    C, psel, projected, checked, strong_n = _check(pn, orc, A, B, mode, list(range(7)))
    assert len(np.unique(psel[projected] & 0x7F)) >= 2
    assert checked > 1000
    if mode == "f32":  # resolved by FP32-accurate sums; not by BF16 ones (t3 - 1 <= 0.13)
        assert strong_n > 1000


@pytest.mark.parametrize("mode", ["tf32", "bf16", "f16", "e4m3"])
def test_r2_low_precision_formats(pn, orc, mode):
    A, B = workloads.wide_range_pair(140, 260, 300, seed=1920)
    _, _, _, checked, strong_n = _check(pn, orc, A, B, mode, list(range(7)),
                                        tile_n=256 if mode != "tf32" else 128)
    if mode != "e4m3":  # E4M3's 2^-4 rounding resolves no second value (eta = 2)
        assert strong_n > 0.9 * checked


def test_r2_recovers_two_valued_products(pn, orc):
    """Every entry's terms take two values (1 and 1/2): the r = 2 estimate is the
    exact max, where the plain estimate is K^(1/p*) high and r = 1 low."""
    M, N, K = 64, 96, 200
    A = np.full((M, K), 0.5, np.float32)
    A[np.arange(M), np.arange(M) % 7] = 1.0
    B = np.ones((K, N), np.float32)
    dA, dB = _dev(A), _dev(B)
    pl = list(range(5))
    tau = orc.default_tau(K, 0)
    C2 = pn.maxprod_pnorm(dA, dB, p_log2=pl, compute="f32", tau=tau, estimator=2)[0].cpu().numpy()
    C1 = pn.maxprod_pnorm(dA, dB, p_log2=pl, compute="f32", tau=tau, estimator=1)[0].cpu().numpy()
    C0 = pn.maxprod_pnorm(dA, dB, p_log2=pl, compute="f32", tau=tau)[0].cpu().numpy()
    np.testing.assert_allclose(C2, 1.0, rtol=2e-5)
    assert np.all(C1 < 1 - 1e-3) and np.all(C0 > 1 + 1e-5)


def test_r2_gap_in_P_is_plain(pn):
    """No chain p*/4, p*/2 below any p* in P: bit-identical to the plain estimator."""
    A, B = workloads.uniform_pair(100, 90, 80, seed=1930)
    dA, dB = _dev(A), _dev(B)
    for pl in ([0, 2, 5], [4], [0, 1]):
        C2 = pn.maxprod_pnorm(dA, dB, p_log2=pl, compute="bf16", estimator=2)[0]
        C0 = pn.maxprod_pnorm(dA, dB, p_log2=pl, compute="bf16", estimator=0)[0]
        assert torch.equal(C0, C2)


def test_r2_n2048_sampled(pn, orc):
    """n = 2048 wide-range entries, BF16: 512 sampled entries against the
    oracle's projection from its own sums at those entries; the r = 2 estimate
    is closer to the exact max than r = 1 and the plain norm."""
    n = 2048
    A, B = workloads.wide_range_pair(n, n, n, seed=1940)
    pl = list(range(7))
    tau = orc.default_tau(n, _CODE["bf16"])
    dA, dB = _dev(A), _dev(B)
    C, psel, _ = pn.maxprod_pnorm(dA, dB, p_log2=pl, compute="bf16", tau=tau, estimator=2)
    C, psel = C.cpu().numpy(), psel.cpu().numpy()
    g = workloads.rng(None, 1941)
    ii, jj = g.integers(0, n, 512), g.integers(0, n, 512)
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    r, c = orc.row_scales(A64), orc.col_scales(B64)
    exact, S = orc.entries(A64, B64, ii, jj, pl, r, c)
    S34 = orc.entries_real(A64, B64, ii, jj, [0.75 * 2.0 ** lp for lp in pl], r, c)
    Chat, ps, _ = orc.estimate(S.T[:, None, :], pl, np.ones(1), r[ii] * c[jj], tau, estimator=2,
                               S34=S34.T[:, None, :])
    Chat, ps = Chat[0], ps[0]
    assert np.array_equal(psel[ii, jj], ps)
    assert np.all(ps == 6)  # every sampled entry stable at p = 64: one chain
    q = 6
    s = np.stack([S[:, q - 2], S[:, q - 1], S34[:, q], S[:, q]])
    lo, hi, strong = r2_bounds(orc, s, 64.0, "bf16", n, tau)
    assert strong.mean() > 0.9
    gv = C[ii, jj] / (r[ii] * c[jj])
    assert np.all(gv >= lo * (1 - EPS)) and np.all(gv <= hi * (1 + EPS))
    C1 = pn.maxprod_pnorm(dA, dB, p_log2=pl, compute="bf16", tau=tau, estimator=1)[0].cpu().numpy()
    C0 = pn.maxprod_pnorm(dA, dB, p_log2=pl, compute="bf16", tau=tau)[0].cpu().numpy()
    e2 = np.median(np.abs(C[ii, jj] - exact) / exact)
    e1 = np.median(np.abs(C1[ii, jj] - exact) / exact)
    e0 = np.median(np.abs(C0[ii, jj] - exact) / exact)
    assert e2 < e1 < e0


def test_r2_n16384_sampled(pn, orc):
    """The bench's r = 2 configuration at full size: n = 16384, entries
    exp(-Exp(4)), BF16, the default tau, CTA pairs; 512 sampled entries within
    the bounds the oracle's own sums at those entries give."""
    n = 16384
    A, B = workloads.wide_range_pair(n, n, n)
    pl = list(range(7))
    C, psel, _ = pn.maxprod_pnorm(_dev(A), _dev(B), p_log2=pl, compute="bf16", estimator=2)
    g = workloads.rng(None, 1942)
    ii, jj = g.integers(0, n, 512), g.integers(0, n, 512)
    ti, tj = torch.from_numpy(ii).cuda(), torch.from_numpy(jj).cuda()
    Cs, ps_gpu = C[ti, tj].cpu().numpy(), psel[ti, tj].cpu().numpy()
    del C, psel
    tau = orc.default_tau(n, _CODE["bf16"])
    rows = np.unique(ii)
    rr = np.zeros(n)
    rr[rows] = orc.row_scales(A[rows].astype(np.float64))
    c = orc.col_scales(B.astype(np.float64))
    exact, S = orc.entries(A, B, ii, jj, pl, rr, c)
    S34 = orc.entries_real(A, B, ii, jj, [0.75 * 2.0 ** lp for lp in pl], rr, c)
    _, ps, _ = orc.estimate(S.T[:, None, :], pl, np.ones(1), rr[ii] * c[jj], tau, estimator=2,
                            S34=S34.T[:, None, :])
    ps = ps[0]
    assert np.array_equal(ps_gpu, ps)
    assert np.all(ps == 6)  # every sampled entry stable at p = 64: one chain
    q = 6
    s = np.stack([S[:, q - 2], S[:, q - 1], S34[:, q], S[:, q]])
    lo, hi, strong = r2_bounds(orc, s, 64.0, "bf16", n, tau)
    assert strong.mean() > 0.9
    gv = Cs / (rr[ii] * c[jj])
    assert np.all(gv >= lo * (1 - EPS)) and np.all(gv <= hi * (1 + EPS))
    assert np.all(Cs <= exact * (1 + EPS))


def test_r2_rejected_where_unsupported(pn):
    """APSP, the adjoint and the grouped call take no r = 2; it excludes the
    affine correction."""
    W = torch.rand(16, 16, device="cuda")
    with pytest.raises(pn.PnError) as ei:
        pn.apsp_pnorm(W, estimator=2)
    assert ei.value.status == 7
    probs = workloads.grouped_problems(np.array([20, 30]), seed=1960)
    with pytest.raises(pn.PnError) as ei:
        pn.GroupedProduct([_dev(a) for a, _ in probs], [_dev(b) for _, b in probs],
                          compute="bf16", estimator=2).run()
    assert ei.value.status == 7
    A = torch.rand(8, 8, device="cuda")
    fi = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises((pn.PnError, ValueError)):
        pn.maxprod_pnorm(A, A, estimator=2, correction=2, fit_i=fi, fit_j=fi)
