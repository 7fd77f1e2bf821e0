"""GPU parity of the bias corrections (pn_opts.correction) against the FP64
oracle, through the C ABI.

correction 1 divides the scaled estimate by K^(1/p*) (Sec. 2.1); its
tolerance is the plain estimator's.  correction 2 fits exact = a_q est + b_q
per p* class on caller-given sample entries (Discussion).  The library forms
the sample estimates directly in FP32 (relative error about K 2^-24), the
oracle in FP64, so the two fitted lines are compared by their predictions at
the samples (within 1e-4), and every corrected entry against the oracle's with
the estimate's own tolerance scaled by the slope, plus that 1e-4.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

_U = {"f32": 2.0 ** -21, "bf16": 2.0 ** -8, "e4m3": 2.0 ** -4}
_M = {"f32": 21, "bf16": 7, "e4m3": 3}
_CODE = {"f32": 0, "bf16": 2, "e4m3": 4}
FIT_TOL = 1e-4


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


def plain_tol(mode, K, plog):
    return 1.5 * ((1 + s_tol(mode, K, plog)) ** (1.0 / 2 ** plog) - 1) + 2e-7


def _multilevel(M, N, K, seed):
    g = workloads.rng(seed)
    A = (0.05 * (0.5 + 0.5 * g.random((M, K)))).astype(np.float32)
    B = (0.05 * (0.5 + 0.5 * g.random((K, N)))).astype(np.float32)
    A[np.arange(M), np.arange(M) % K] = 1.0
    B[(np.arange(N) + 1) % K, np.arange(N)] = 1.0
    return A, B


def _agree_mask(orc, ref, psel, pl, tau, mode, K):
    near = np.zeros(psel.shape, dtype=bool)
    for q, lp in enumerate(pl):
        near |= np.abs(ref["S"][q] / tau - 1) < 4 * s_tol(mode, K, lp)
    return (psel == ref["p_sel"]) & ~near


@pytest.mark.parametrize("data", ["uniform", "multilevel"])
def test_divide_by_K_matches_oracle(pn, orc, data):
    M, N, K = 130, 300, 257
    A, B = (workloads.uniform_pair(M, N, K, seed=1900) if data == "uniform"
            else _multilevel(M, N, K, seed=1901))
    pl = list(range(7))
    tau = orc.default_tau(K, _CODE["f32"])
    C, psel, _ = pn.maxprod_pnorm(_dev(A), _dev(B), p_log2=pl, compute="f32", tau=tau,
                                  correction=1)
    C, psel = C.cpu().numpy(), psel.cpu().numpy()
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    ref = orc.pnorm(A64, B64, pl, tau, want_S=True, correction=1)
    ok = _agree_mask(orc, ref, psel, pl, tau, "f32", K) & (ref["C"] > 0)
    tol = np.vectorize(lambda lp: plain_tol("f32", K, lp))(psel & 0x7F)
    err = np.abs(C - ref["C"]) / np.maximum(ref["C"], 1e-300)
    assert np.all(err[ok] <= tol[ok]), float(err[ok].max())
    exact = orc.maxprod(A64, B64)
    pstar = 2.0 ** (psel & 0x7F)
    assert np.all(C <= exact * (1 + tol))
    assert np.all(C >= exact * K ** (-1 / pstar) * (1 - tol))


def _affine_case(pn, orc, A, B, mode, pl, n_fit, seed, estimator=0):
    M, K = A.shape
    N = B.shape[1]
    g = workloads.rng(seed)
    ii, jj = g.integers(0, M, n_fit), g.integers(0, N, n_fit)
    tau = orc.default_tau(K, _CODE[mode])
    dA, dB = _dev(A), _dev(B)
    coef = torch.zeros(2 * len(pl), dtype=torch.float32, device="cuda")
    fi = torch.from_numpy(ii.astype(np.int32)).cuda()
    fj = torch.from_numpy(jj.astype(np.int32)).cuda()
    C2, psel, _ = pn.maxprod_pnorm(dA, dB, p_log2=pl, compute=mode, tau=tau, correction=2,
                                   fit_i=fi, fit_j=fj, fit_coef=coef, estimator=estimator)
    C0, psel0, _ = pn.maxprod_pnorm(dA, dB, p_log2=pl, compute=mode, tau=tau,
                                    estimator=estimator)
    assert torch.equal(psel, psel0)
    C2, C0, psel = C2.cpu().numpy(), C0.cpu().numpy(), psel.cpu().numpy()
    coef = coef.cpu().numpy().reshape(-1, 2).astype(np.float64)
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    ref = orc.pnorm(A64, B64, pl, tau, want_S=True, estimator=estimator, correction=2,
                    fit_ij=(ii, jj))
    # 1. the fitted lines agree at the samples' own (oracle) estimates
    r, c = ref["r"], ref["c"]
    _, S = orc.entries(A64, B64, ii, jj, pl, r, c)
    est, ps, _ = orc.estimate(S.T[:, None, :], pl, np.ones(1), np.ones(len(ii)), tau, estimator)
    idx = {lp: q for q, lp in enumerate(pl)}
    cls = np.array([idx[int(b) & 0x7F] for b in ps[0]])
    x = est[0]
    pg = coef[cls, 0] * x + coef[cls, 1]
    po = ref["coef"][cls, 0] * x + ref["coef"][cls, 1]
    assert np.all(np.abs(pg - po) <= FIT_TOL * np.abs(po)), float(np.max(np.abs(pg - po) / po))
    # 2. the GPU applied its own line to its own estimate (FP32 rounding)
    rc = r[:, None] * c[None, :]
    q_of = np.vectorize(lambda b: idx[int(b) & 0x7F])(psel)
    want = rc * (coef[q_of, 0] * (C0 / rc) + coef[q_of, 1])
    scale = rc * (np.abs(coef[q_of, 0] * (C0 / rc)) + np.abs(coef[q_of, 1]))
    assert np.all(np.abs(C2 - want) <= 8 * 2.0 ** -24 * scale + 1e-30)
    # 3. every corrected entry against the oracle's corrected entry
    ok = _agree_mask(orc, ref, psel, pl, tau, mode, K) & (ref["C"] > 0)
    t = np.vectorize(lambda lp: plain_tol(mode, K, lp))(psel & 0x7F)
    if estimator == 1:
        t = 3 * t  # the projection's ratio of two sums
    a = np.abs(coef[q_of, 0])
    tol = t * a * (C0 / rc) / np.maximum(np.abs(ref["C"] / rc), 1e-300) + 2 * FIT_TOL
    err = np.abs(C2 - ref["C"]) / np.maximum(np.abs(ref["C"]), 1e-300)
    assert np.all(err[ok] <= tol[ok]), float(err[ok].max())
    return C0, C2, ref


@pytest.mark.parametrize("mode", ["f32", "bf16"])
def test_affine_matches_oracle(pn, orc, mode):
    A, B = workloads.wide_range_pair(150, 260, 700, seed=1910)
    _affine_case(pn, orc, A, B, mode, list(range(7)), 300, 1911)


def test_affine_several_classes(pn, orc):
    """p* spread over several levels: one line per class."""
    A, B = _multilevel(150, 170, 128, seed=1920)
    C0, C2, ref = _affine_case(pn, orc, A, B, "f32", list(range(7)), 400, 1921)
    assert len(np.unique(ref["p_sel"] & 0x7F)) >= 2


def test_affine_with_projection(pn, orc):
    A, B = workloads.wide_range_pair(140, 200, 500, seed=1930)
    _affine_case(pn, orc, A, B, "bf16", list(range(7)), 256, 1931, estimator=1)


def test_affine_reduces_error_n2048(pn, orc):
    """n = 2048 wide-range entries, BF16: 512 samples fit the line; on 1024
    other entries the median relative error against the exact max drops by
    more than 5x."""
    n = 2048
    A, B = workloads.wide_range_pair(n, n, n, seed=1940)
    g = workloads.rng(1941)
    fi = torch.from_numpy(g.integers(0, n, 512).astype(np.int32)).cuda()
    fj = torch.from_numpy(g.integers(0, n, 512).astype(np.int32)).cuda()
    dA, dB = _dev(A), _dev(B)
    C0 = pn.maxprod_pnorm(dA, dB, compute="bf16")[0].cpu().numpy()
    C2 = pn.maxprod_pnorm(dA, dB, compute="bf16", correction=2, fit_i=fi, fit_j=fj)[0]
    C2 = C2.cpu().numpy()
    ii, jj = g.integers(0, n, 1024), g.integers(0, n, 1024)
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    exact, _ = orc.entries(A64, B64, ii, jj, [0], orc.row_scales(A64), orc.col_scales(B64))
    e0 = np.median(np.abs(C0[ii, jj] - exact) / exact)
    e2 = np.median(np.abs(C2[ii, jj] - exact) / exact)
    assert e2 < e0 / 5, (e0, e2)


def test_affine_n16384_sampled(pn, orc):
    """The bench's affine-correction configuration at full size: n = 16384,
    entries exp(-Exp(4)), BF16, the default tau, CTA pairs, 1024 fit samples
    drawn as the bench draws them.  The library's fitted lines against the
    oracle's fit of its own estimates and exact maxima at those samples (by
    their predictions there), and 512 other corrected entries against the
    oracle's line applied to the oracle's estimate."""
    n = 16384
    A, B = workloads.wide_range_pair(n, n, n)
    pl = list(range(7))
    gfit = workloads.rng(None, 150)
    fi, fj = gfit.integers(0, n, 1024), gfit.integers(0, n, 1024)
    coef = torch.zeros(2 * len(pl), dtype=torch.float32, device="cuda")
    dA, dB = _dev(A), _dev(B)
    C2, psel, _ = pn.maxprod_pnorm(dA, dB, p_log2=pl, compute="bf16", correction=2,
                                   fit_i=torch.from_numpy(fi.astype(np.int32)).cuda(),
                                   fit_j=torch.from_numpy(fj.astype(np.int32)).cuda(),
                                   fit_coef=coef)
    g = workloads.rng(None, 151)
    ii, jj = g.integers(0, n, 512), g.integers(0, n, 512)
    ti, tj = torch.from_numpy(ii).cuda(), torch.from_numpy(jj).cuda()
    C2s, ps_gpu = C2[ti, tj].cpu().numpy().astype(np.float64), psel[ti, tj].cpu().numpy()
    del C2, psel, dA, dB
    coef = coef.cpu().numpy().reshape(-1, 2).astype(np.float64)
    tau = orc.default_tau(n, _CODE["bf16"])
    rows = np.unique(np.concatenate([fi, ii]))
    r = np.zeros(n)
    r[rows] = orc.row_scales(A[rows].astype(np.float64))
    c = orc.col_scales(B.astype(np.float64))
    idx = {lp: q for q, lp in enumerate(pl)}

    def scaled(ei, ej):
        exact, S = orc.entries(A, B, ei, ej, pl, r, c)
        est, ps, _ = orc.estimate(S.T[:, None, :], pl, np.ones(1), np.ones(len(ei)), tau, 0)
        cls = np.array([idx[int(b) & 0x7F] for b in ps[0]])
        return est[0], exact / (r[ei] * c[ej]), cls, ps[0]
    x, y, cls, _ = scaled(fi, fj)
    co = orc.affine_fit(x, y, cls, len(pl))
    pg = coef[cls, 0] * x + coef[cls, 1]
    po = co[cls, 0] * x + co[cls, 1]
    assert np.all(np.abs(pg - po) <= FIT_TOL * np.abs(po)), float(np.max(np.abs(pg - po) / po))
    x2, _, cls2, ps2 = scaled(ii, jj)
    assert np.array_equal(ps_gpu, ps2)
    rc = r[ii] * c[jj]
    want = rc * (co[cls2, 0] * x2 + co[cls2, 1])
    t = np.array([plain_tol("bf16", n, int(b) & 0x7F) for b in ps2])
    tol = t * np.abs(co[cls2, 0]) * x2 * rc / np.abs(want) + 2 * FIT_TOL
    err = np.abs(C2s - want) / np.abs(want)
    assert np.all(err <= tol), float(err.max())


def test_correction_grouped_divide(pn, orc):
    sizes = np.minimum(workloads.grouped_sizes(10, seed=1950), 260)
    probs = workloads.grouped_problems(sizes, seed=1950)
    plan = pn.GroupedProduct([_dev(a) for a, _ in probs], [_dev(b) for _, b in probs],
                             compute="f32", tile_n=128)
    plan.opts.correction = 1
    Cs = [c.cpu().numpy() for c in plan.run(check=True)]
    pl = list(range(7))
    for (A, B), C in zip(probs, Cs):
        K = A.shape[1]
        tau = orc.default_tau(K, _CODE["f32"])
        ref = orc.pnorm(A.astype(np.float64), B.astype(np.float64), pl, tau, want_S=True,
                        correction=1)
        ok = _agree_mask(orc, ref, ref["p_sel"], pl, tau, "f32", K)
        tol = np.vectorize(lambda lp: plain_tol("f32", K, lp))(ref["p_sel"] & 0x7F)
        err = np.abs(C - ref["C"]) / ref["C"]
        assert np.all(err[ok] <= tol[ok]), float(err[ok].max())


def test_correction_errors(pn):
    A = torch.rand(40, 30, device="cuda")
    B = torch.rand(30, 20, device="cuda")
    fi = torch.tensor([0, 39, 40], dtype=torch.int32, device="cuda")  # 40 is out of range
    fj = torch.tensor([0, 19, 3], dtype=torch.int32, device="cuda")
    with pytest.raises(pn.PnError) as ei:
        pn.maxprod_pnorm(A, B, correction=2, fit_i=fi, fit_j=fj)
    assert ei.value.status == 1
    W = torch.rand(16, 16, device="cuda")
    with pytest.raises(pn.PnError) as ei:
        pn.apsp_pnorm(W, correction=1)
    assert ei.value.status == 7
    probs = workloads.grouped_problems(np.array([20, 30]), seed=1960)
    plan = pn.GroupedProduct([_dev(a) for a, _ in probs], [_dev(b) for _, b in probs],
                             compute="bf16")
    plan.opts.correction = 2
    plan.opts.n_fit = 1
    plan.opts.fit_i = fi.data_ptr()
    plan.opts.fit_j = fj.data_ptr()
    with pytest.raises(pn.PnError) as ei:
        plan.run(check=True)
    assert ei.value.status == 7
