"""GPU parity of the r = 1 multiset-projection estimator (Sec. 2.1,
pn_opts.estimator = 1) against the FP64 oracle, through the C ABI.

At p* with p' = p*/2 in P the estimate is (S^(p*) / S^(p'))^(1/p'): a relative
error d1 of S^(p*) and d2 of S^(p') (each bounded as in the plain-estimator
tests) become ((1 + d1) / (1 - d2))^(1/p') - 1, plus a few FP32 roundings of
the division, the root and the scale.
"""
import math

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


def s_tol(mode, K, plog):
    p = 2.0 ** plog
    return 2 * (p - 1) * 2.0 ** -24 + 2 * _U[mode] + 2.0 ** -_M[mode] + K * 2.0 ** -23


def proj_tol(mode, K, plog):
    """Tolerance at p* = 2^plog (plog >= 1, p* / 2 in P)."""
    d1, d2 = s_tol(mode, K, plog), s_tol(mode, K, plog - 1)
    return 1.5 * (((1 + d1) / (1 - d2)) ** (1.0 / 2 ** (plog - 1)) - 1) + 4e-7


def plain_tol(mode, K, plog):
    return 1.5 * ((1 + s_tol(mode, K, plog)) ** (1.0 / 2 ** plog) - 1) + 2e-7


def _multilevel_inputs(M, N, K, seed):
    """Rows with one dominant term resolve at large p, rows of small flat terms
    at small p (S^(p) drops below tau), so p* varies across the output."""
    g = workloads.rng(seed)
    A = (0.05 * (0.5 + 0.5 * g.random((M, K)))).astype(np.float32)
    B = (0.05 * (0.5 + 0.5 * g.random((K, N)))).astype(np.float32)
    A[np.arange(M), np.arange(M) % K] = 1.0
    B[(np.arange(N) + 1) % K, np.arange(N)] = 1.0
    return A, B


def _check(pn, orc, A, B, mode, pl, tau=None, tile_n=0):
    M, K = A.shape
    tau = orc.default_tau(K, _CODE[mode]) if tau is None else tau
    dA, dB = _dev(A), _dev(B)
    C, psel, ssel = pn.maxprod_pnorm(dA, dB, p_log2=pl, compute=mode, tau=tau, tile_n=tile_n,
                                     estimator=1)
    C0, psel0, ssel0 = pn.maxprod_pnorm(dA, dB, p_log2=pl, compute=mode, tau=tau, tile_n=tile_n,
                                        estimator=0)
    # p_sel and S_sel keep their meaning (p* and S^(p*)): identical to the plain run
    assert torch.equal(psel, psel0)
    assert torch.equal(ssel, ssel0)
    C, psel = C.cpu().numpy(), psel.cpu().numpy()
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    ref = orc.pnorm(A64, B64, pl, tau, want_S=True, estimator=1)
    near = np.zeros(C.shape, dtype=bool)
    for q, lp in enumerate(pl):
        near |= np.abs(ref["S"][q] / tau - 1) < 4 * s_tol(mode, K, lp)
    agree = psel == ref["p_sel"]
    assert np.all(agree | near)
    lp_sel = (psel & 0x7F).astype(int)
    prev = {pl[q]: (q > 0 and pl[q - 1] == pl[q] - 1) for q in range(len(pl))}
    projected = np.vectorize(lambda b: bool(prev[int(b) & 0x7F]) and not (int(b) & 0x80))(psel)
    tol = np.where(projected, np.vectorize(lambda lp: proj_tol(mode, K, max(lp, 1)))(lp_sel),
                   np.vectorize(lambda lp: plain_tol(mode, K, lp))(lp_sel))
    err = np.abs(C - ref["C"]) / np.maximum(ref["C"], 1e-300)
    ok = agree & (ref["C"] > 0)
    assert np.all(err[ok] <= tol[ok]), (mode, float(err[ok].max()), np.argwhere(ok & (err > tol))[:5])
    # Sec. 2.1 envelope of the projection: exact * (2/(sqrt(K)+1))^(2/p*) <= Chat <= exact
    exact = orc.maxprod(A64, B64)
    pstar = 2.0 ** lp_sel
    low = np.where(projected, exact * (2 / (math.sqrt(K) + 1)) ** (2 / pstar), exact)
    high = np.where(projected, exact, exact * K ** (1 / pstar))
    assert np.all(C <= high * (1 + tol) + 1e-30)
    assert np.all(C >= low * (1 - tol) - 1e-30)
    return C, psel, err, projected


@pytest.mark.parametrize("shape", [(1, 1, 1), (5, 7, 3), (130, 300, 257), (129, 77, 33),
                                   (200, 64, 500)])
def test_projection_f32_matches_oracle(pn, orc, shape):
    M, N, K = shape
    A, B = workloads.uniform_pair(M, N, K, seed=1700 + M)
    _check(pn, orc, A, B, "f32", list(range(7)))


@pytest.mark.parametrize("mode", ["f32", "bf16"])
def test_projection_multilevel(pn, orc, mode):
    """p* spread over several levels: each projected entry's S^(p*/2) comes from
    the level below the one that resolved it."""
    A, B = _multilevel_inputs(150, 170, 128, seed=1710)
    C, psel, _, projected = _check(pn, orc, A, B, mode, list(range(7)))
    assert len(np.unique(psel[projected] & 0x7F)) >= 2


@pytest.mark.parametrize("mode", ["tf32", "bf16", "f16", "e4m3"])
def test_projection_low_precision_formats(pn, orc, mode):
    A, B = workloads.wide_range_pair(140, 260, 300, seed=1720)
    _check(pn, orc, A, B, mode, list(range(7)), tile_n=256 if mode != "tf32" else 128)


def test_projection_gap_in_P_is_plain(pn):
    """No p* / 2 in P anywhere: bit-identical to the plain estimator."""
    A, B = workloads.uniform_pair(100, 90, 80, seed=1730)
    dA, dB = _dev(A), _dev(B)
    for pl in ([0, 2, 5], [4]):
        C1 = pn.maxprod_pnorm(dA, dB, p_log2=pl, compute="bf16", estimator=1)[0]
        C0 = pn.maxprod_pnorm(dA, dB, p_log2=pl, compute="bf16", estimator=0)[0]
        assert torch.equal(C0, C1)


def test_projection_n2048_sampled(pn, orc):
    """n = 2048 wide-range entries, BF16: 512 sampled entries against the
    oracle's projection from its own p-sums at those entries."""
    n = 2048
    A, B = workloads.wide_range_pair(n, n, n, seed=1740)
    pl = list(range(7))
    tau = orc.default_tau(n, _CODE["bf16"])
    C, psel, _ = pn.maxprod_pnorm(_dev(A), _dev(B), p_log2=pl, compute="bf16", tau=tau,
                                  estimator=1)
    C, psel = C.cpu().numpy(), psel.cpu().numpy()
    g = workloads.rng(None, 1741)
    ii, jj = g.integers(0, n, 512), g.integers(0, n, 512)
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    r, c = orc.row_scales(A64), orc.col_scales(B64)
    exact, S = orc.entries(A64, B64, ii, jj, pl, r, c)
    Chat, ps, _ = orc.estimate(S.T[:, None, :], pl, np.ones(1), r[ii] * c[jj], tau, estimator=1)
    Chat, ps = Chat[0], ps[0]
    assert np.array_equal(psel[ii, jj], ps)
    tol = np.vectorize(lambda lp: proj_tol("bf16", n, lp))(ps & 0x7F)
    err = np.abs(C[ii, jj] - Chat) / Chat
    assert np.all(err <= tol), float(err.max())
    pstar = 2.0 ** (ps & 0x7F)
    assert np.all(C[ii, jj] <= exact * (1 + tol))
    assert np.all(C[ii, jj] >= exact * (2 / (math.sqrt(n) + 1)) ** (2 / pstar) * (1 - tol))
    # the projection is closer to the exact max than the plain norm on this data
    C0 = pn.maxprod_pnorm(_dev(A), _dev(B), p_log2=pl, compute="bf16", tau=tau)[0].cpu().numpy()
    e1 = np.median(np.abs(C[ii, jj] - exact) / exact)
    e0 = np.median(np.abs(C0[ii, jj] - exact) / exact)
    assert e1 < e0


def test_projection_n16384_sampled(pn, orc):
    """The bench's r = 1 configuration at full size: n = 16384, entries
    exp(-Exp(4)), BF16, the default tau, CTA pairs; 512 sampled entries against
    the oracle's projection from its own p-sums at those entries."""
    n = 16384
    A, B = workloads.wide_range_pair(n, n, n)
    pl = list(range(7))
    C, psel, _ = pn.maxprod_pnorm(_dev(A), _dev(B), p_log2=pl, compute="bf16", estimator=1)
    g = workloads.rng(None, 1742)
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
    Chat, ps, _ = orc.estimate(S.T[:, None, :], pl, np.ones(1), rr[ii] * c[jj], tau, estimator=1)
    Chat, ps = Chat[0], ps[0]
    assert np.array_equal(ps_gpu, ps)
    tol = np.vectorize(lambda lp: proj_tol("bf16", n, lp))(ps & 0x7F)
    err = np.abs(Cs - Chat) / Chat
    assert np.all(err <= tol), float(err.max())
    pstar = 2.0 ** (ps & 0x7F)
    assert np.all(Cs <= exact * (1 + tol))
    assert np.all(Cs >= exact * (2 / (math.sqrt(n) + 1)) ** (2 / pstar) * (1 - tol))


def test_projection_grouped(pn, orc):
    sizes = np.minimum(workloads.grouped_sizes(12, seed=1750), 300)
    probs = workloads.grouped_problems(sizes, seed=1750)
    g = workloads.rng(1751)
    probs.append(((1 - g.random((37, 129))).astype(np.float32),
                  (1 - g.random((129, 5))).astype(np.float32)))
    pl = list(range(7))
    for tile_n in (128, 256):
        plan = pn.GroupedProduct([_dev(a) for a, _ in probs], [_dev(b) for _, b in probs],
                                 compute="bf16", tile_n=tile_n, estimator=1)
        Cs = [c.cpu().numpy() for c in plan.run(check=True)]
        for (A, B), C in zip(probs, Cs):
            K = A.shape[1]
            tau = orc.default_tau(K, _CODE["bf16"])
            ref = orc.pnorm(A.astype(np.float64), B.astype(np.float64), pl, tau, want_S=True,
                            estimator=1)
            near = np.zeros(C.shape, bool)
            for q in range(7):
                near |= np.abs(ref["S"][q] / tau - 1) < 4 * s_tol("bf16", K, 6)
            q = ref["p_sel"] & 0x7F
            tol = np.vectorize(lambda lp: proj_tol("bf16", K, max(lp, 1)))(q)
            err = np.abs(C - ref["C"]) / ref["C"]
            assert np.all((err <= tol) | near), (A.shape, B.shape, float(err.max()))


def test_projection_rejected_where_unsupported(pn):
    """APSP and the adjoint take the plain estimator only; a grouped table built
    for one estimator refuses the other."""
    W = torch.rand(16, 16, device="cuda")
    with pytest.raises(pn.PnError) as ei:
        pn.apsp_pnorm(W, estimator=1)
    assert ei.value.status == 7
    probs = workloads.grouped_problems(np.array([20, 30]), seed=1760)
    plan = pn.GroupedProduct([_dev(a) for a, _ in probs], [_dev(b) for _, b in probs],
                             compute="bf16")
    plan.opts.estimator = 1
    with pytest.raises(pn.PnError) as ei:
        plan.run(check=True)
    assert ei.value.status == 1
