"""GPU parity of the p-norm APSP driver (Sec. 2.2) against the FP64 oracle.

x = exp(-w), ceil(log2 n) p-norm squarings with the diagonal reset, d = -log x.
Tolerances follow from the product's (see test_gpu_product.pnorm_tol): one
squaring is homogeneous of degree 2 in X, so a relative error e in X_t becomes
at most 2e in X_(t+1); over T squarings the x-space error is at most
(2^T - 1) times the per-squaring tolerance, and x-space relative error equals
distance-space absolute error.
"""
import math

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1511_05690_gb300 as pn
    pn.lib()
    return pn


def _step_tol(n, plog=6):
    p = 2.0 ** plog
    s = 2 * (p - 1) * 2.0 ** -24 + 3 * 2.0 ** -21 + n * 2.0 ** -23
    return 1.5 * ((1 + s) ** (1.0 / p) - 1) + 2e-7


PL = list(range(7))


@pytest.mark.parametrize("n,density", [(37, 0.3), (300, 0.1), (512, 0.05)])
def test_apsp_full_pipeline_matches_oracle(pn, orc, n, density):
    """Weights in [0, 0.3]: every shortest path is short enough that each
    squaring is stable at p = 64 for every entry, so GPU and oracle take the
    same p* everywhere and the error bound above applies."""
    W = workloads.apsp_weights(n, density=density, hi=0.3, seed=600 + n)
    tau = orc.default_tau(n, orc.F32_EXACT)
    D = pn.apsp_pnorm(torch.from_numpy(W).cuda(), p_log2=PL, compute="f32", tau=tau).cpu().numpy()
    Dref, psel = orc.apsp_pnorm(W.astype(np.float64), PL, tau)
    T = math.ceil(math.log2(n))
    assert np.all(psel == 6)  # premise of the bound (a property of the data)
    fin = np.isfinite(Dref)
    assert np.array_equal(np.isfinite(D), fin)
    tol = (2 ** T - 1) * _step_tol(n) + 1e-6
    err = np.abs(D[fin] - Dref[fin])
    assert err.max() <= tol, (err.max(), tol)
    assert np.all(np.diag(D) == 0.0)
    # exact APSP: the p-norm distance never exceeds it (Chat >= C at every step)
    Dfw = orc.floyd_warshall(W.astype(np.float64))
    assert np.all(D[fin] <= Dfw[fin] + tol)


def test_apsp_n4096_per_squaring_on_sampled_entries(pn, orc):
    """Config: n = 4096, density 0.1, weights U[0,1], 12 squarings.  For
    t = 1, 6, 11 the GPU's X_t (from D_t) is fed to the oracle, which computes
    4096 sampled entries of one more squaring; the GPU's D_(t+1) must agree."""
    n = 4096
    W = workloads.apsp_weights(n, density=0.1, index=1)
    dW = torch.from_numpy(W).cuda()
    tau = orc.default_tau(n, orc.F32_EXACT)
    g = workloads.rng(None, 101)
    ii, jj = g.integers(0, n, 4096), g.integers(0, n, 4096)
    for t in (1, 6, 11):
        Dt = pn.apsp_pnorm(dW, n_squarings=t, p_log2=PL, compute="f32", tau=tau).cpu().numpy()
        Dn = pn.apsp_pnorm(dW, n_squarings=t + 1, p_log2=PL, compute="f32", tau=tau)
        Dn = Dn.cpu().numpy()
        X = np.exp(-Dt.astype(np.float64))
        r, c = orc.row_scales(X), orc.col_scales(X)
        _, S = orc.entries(X, X, ii, jj, PL, r, c)
        # the oracle's own p* per entry; entries whose S sits within the
        # error band of tau at some p could legitimately pick another p*
        stable = S >= tau
        q = np.where(stable.any(axis=1), 6 - np.argmax(stable[:, ::-1], axis=1), 0)
        band = np.any(np.abs(S / tau - 1) < 1e-3, axis=1)
        S_at = S[np.arange(len(ii)), q]
        xhat = r[ii] * c[jj] * np.power(S_at, 1.0 / 2.0 ** q)
        xhat[ii == jj] = 1.0
        dref = -np.log(xhat)
        keep = ~band & np.isfinite(dref)
        assert keep.mean() > 0.99
        err = np.abs(Dn[ii, jj][keep] - dref[keep])
        # one squaring at the entry's p*, plus the FP32 rounding of D_t (2^-24 relative in d)
        tol = np.array([_step_tol(n, int(x)) for x in q[keep]])
        tol += 4 * 2.0 ** -24 * (1 + np.abs(Dt[np.isfinite(Dt)]).max())
        assert np.all(err <= tol), (t, float(err.max()))


def test_apsp_n4096_against_floyd_warshall(pn, orc):
    """Final 12-squaring estimate against exact Floyd-Warshall distances on 64
    sampled rows: never above the exact distance; error statistics reported."""
    n = 4096
    W = workloads.apsp_weights(n, density=0.1, index=1)
    D = pn.apsp_pnorm(torch.from_numpy(W).cuda(), p_log2=PL, compute="f32").cpu().numpy()
    Dfw = orc.floyd_warshall(W.astype(np.float64))
    rows = workloads.sampled_rows(n, 64)
    d, dfw = D[rows], Dfw[rows]
    assert np.all(np.isfinite(d) == np.isfinite(dfw))
    fin = np.isfinite(dfw)
    tol = (2 ** 12 - 1) * _step_tol(n)
    assert np.all(d[fin] <= dfw[fin] + tol)
    mse = float(np.mean((d[fin] - dfw[fin]) ** 2))
    print(f"APSP n=4096: MSE vs Floyd-Warshall {mse:.4g}, max abs {np.max(dfw[fin] - d[fin]):.4g}")


def test_apsp_domain_error(pn):
    W = workloads.apsp_weights(50, density=0.2, seed=5)
    W[3, 4] = -0.5
    with pytest.raises(pn.PnError) as ei:
        pn.apsp_pnorm(torch.from_numpy(W).cuda())
    assert ei.value.status == 4


def test_apsp_trivial_sizes(pn, orc):
    D = pn.apsp_pnorm(torch.zeros((1, 1), device="cuda")).cpu().numpy()
    assert D[0, 0] == 0.0
    W = np.array([[0.0, 2.0], [np.inf, 0.0]], dtype=np.float32)
    tau = orc.default_tau(2, orc.F32_EXACT)
    D = pn.apsp_pnorm(torch.from_numpy(W).cuda(), tau=tau).cpu().numpy()
    Dref, _ = orc.apsp_pnorm(W.astype(np.float64), PL, tau)
    assert D[0, 0] == 0 and D[1, 1] == 0 and np.isinf(D[1, 0])
    # two equal 2-hop terms: the estimate is 2 - ln(2)/p* (p* = 16 here: e^-128
    # underflows FP32 at p = 64 and 32), i.e. the method's own error
    assert abs(D[0, 1] - Dref[0, 1]) < 1e-5 and D[0, 1] <= 2.0
