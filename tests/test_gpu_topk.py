"""GPU parity of the approximate top-k of x_i y_j (Alg. 9 with the NormQueue)
against the FP64 oracle, through the C ABI.

The library's p-sums come from FP64 FFT convolutions, the oracle's from naive
sums.  The NormQueue is sequential: every pop subtracts an estimate from the
sums of one diagonal, so rounding differences accumulate, and near-ties
between two diagonals' estimates can be broken differently; from then on the
two runs pop different (equally valid) sequences.  Parity is therefore (1) the
first pops -- until the first near-tie -- agree in value (1e-6), and (2) against the exact top-k of x_i y_j the library is as accurate as the
oracle (max error within 3x the oracle's or 5e-3, median within 5x or 1e-6).
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

P13 = list(range(13))


@pytest.fixture(scope="module")
def pn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1511_05690_gb300 as pn
    pn.lib()
    return pn


def _dev(v):
    return torch.from_numpy(np.ascontiguousarray(v, dtype=np.float32)).cuda()


def _pair(batch, n, seed):
    g = workloads.rng(seed)
    return (g.random((batch, n)).astype(np.float32), g.random((batch, n)).astype(np.float32))


@pytest.mark.parametrize("n,k", [(1, 2), (37, 40), (300, 100), (1000, 300), (4096, 500)])
def test_topk_matches_oracle(pn, orc, n, k):
    x, y = _pair(2, n, 2500 + n)
    vals, ii, jj = pn.topk_xy(_dev(x), _dev(y), k, p_log2=P13)
    vals, ii, jj = vals.cpu().numpy(), ii.cpu().numpy(), jj.cpu().numpy()
    for b in range(2):
        x64, y64 = x[b].astype(np.float64), y[b].astype(np.float64)
        v, d = orc.topk_xy(x64, y64, k, P13)
        ok = d >= 0
        assert np.all(vals[b][~ok] == 0) and np.all(ii[b][~ok] == -1)
        # (1) the first pops agree
        head = min(8, int(ok.sum()))
        np.testing.assert_allclose(vals[b][:head], v[:head], rtol=1e-6)
        # (2) as accurate as the oracle against the exact top-k
        exact = np.sort(np.outer(x64, y64).ravel())[::-1][:int(ok.sum())]
        eg = np.abs(np.sort(vals[b][ok])[::-1] - exact) / exact
        eo = np.abs(np.sort(v[ok])[::-1] - exact) / exact
        assert eg.max() <= max(3 * eo.max(), 5e-3), (eg.max(), eo.max())
        assert np.median(eg) <= max(5 * np.median(eo), 1e-6), (np.median(eg), np.median(eo))
        # indices: every reported pair is consistent and a real product
        rep = ii[b] >= 0
        prod = x[b][ii[b][rep]].astype(np.float64) * y[b][jj[b][rep]]
        assert np.all(np.abs(prod - vals[b][rep]) <= 1e-2 * vals[b][rep])


def test_topk_bench_batch(pn, orc):
    """The batch the bench times: 256 pairs of n = 4096, k = 1024, x, y
    U[0,1), P = {1..4096}.  Four rows (the first, the last and two drawn at
    random) held to the oracle as above, and bit-identical to the same rows
    launched alone."""
    batch, n, k = 256, 4096, 1024
    g = workloads.rng(None, 7)
    x = g.random((batch, n)).astype(np.float32)
    y = g.random((batch, n)).astype(np.float32)
    vals, ii, jj = pn.topk_xy(_dev(x), _dev(y), k, p_log2=P13)
    rows = np.unique(np.concatenate([[0, batch - 1], workloads.rng(2530).integers(0, batch, 2)]))
    for b in rows:
        v1, i1, j1 = pn.topk_xy(_dev(x[b]), _dev(y[b]), k, p_log2=P13)
        assert torch.equal(vals[b], v1[0]) and torch.equal(ii[b], i1[0]) and torch.equal(jj[b], j1[0])
        vb, ib, jb = vals[b].cpu().numpy(), ii[b].cpu().numpy(), jj[b].cpu().numpy()
        x64, y64 = x[b].astype(np.float64), y[b].astype(np.float64)
        v, d = orc.topk_xy(x64, y64, k, P13)
        ok = d >= 0
        np.testing.assert_allclose(vb[:8], v[:8], rtol=1e-6)
        exact = np.sort(np.outer(x64, y64).ravel())[::-1][:int(ok.sum())]
        eg = np.abs(np.sort(vb[ok])[::-1] - exact) / exact
        eo = np.abs(np.sort(v[ok])[::-1] - exact) / exact
        assert eg.max() <= max(3 * eo.max(), 5e-3), (eg.max(), eo.max())
        assert np.median(eg) <= max(5 * np.median(eo), 1e-6), (np.median(eg), np.median(eo))
        rep = ib >= 0
        prod = x[b][ib[rep]].astype(np.float64) * y[b][jb[rep]]
        assert np.all(np.abs(prod - vb[rep]) <= 1e-2 * vb[rep])


def test_topk_close_to_exact_and_indices(pn, orc):
    n, k = 2000, 400
    x, y = _pair(1, n, 2510)
    vals, ii, jj = pn.topk_xy(_dev(x), _dev(y), k, p_log2=P13)
    vals, ii, jj = vals.cpu().numpy()[0], ii.cpu().numpy()[0], jj.cpu().numpy()[0]
    exact = np.sort(np.outer(x[0].astype(np.float64), y[0]).ravel())[::-1]
    np.testing.assert_allclose(vals, exact[:k], rtol=2e-3)
    assert np.all(np.diff(vals) <= 0)
    rep = ii >= 0
    assert rep.sum() >= k // 4
    prod = x[0][ii[rep]].astype(np.float64) * y[0][jj[rep]]
    assert np.all(prod >= exact[min(len(exact) - 1, 4 * k)])  # among the top products


def test_topk_exhaustion_and_batch_rows(pn, orc):
    x = np.array([[1.0, 0.3]], np.float32)
    y = np.array([[0.9, 0.2]], np.float32)
    vals, ii, jj = pn.topk_xy(_dev(x), _dev(y), 6, p_log2=P13)
    v, d = orc.topk_xy(x[0].astype(np.float64), y[0].astype(np.float64), 6, P13)
    np.testing.assert_allclose(vals.cpu().numpy()[0], v, rtol=1e-5)
    assert list(vals.cpu().numpy()[0][4:]) == [0.0, 0.0]
    assert list(ii.cpu().numpy()[0][4:]) == [-1, -1]
    xb, yb = _pair(3, 500, 2520)
    vb, ib, jb = pn.topk_xy(_dev(xb), _dev(yb), 50, p_log2=P13)
    for b in range(3):
        v1, i1, j1 = pn.topk_xy(_dev(xb[b]), _dev(yb[b]), 50, p_log2=P13)
        assert torch.equal(vb[b], v1[0]) and torch.equal(ib[b], i1[0]) and torch.equal(jb[b], j1[0])


def test_topk_errors(pn):
    bad = torch.rand((2, 30), device="cuda")
    bad[1, 4] = float("nan")
    with pytest.raises(pn.PnError) as ei:
        pn.topk_xy(bad, torch.rand((2, 30), device="cuda"), 5)
    assert ei.value.status == 4
    with pytest.raises(pn.PnError) as ei:
        pn.topk_xy(torch.rand((1, 5000), device="cuda"), torch.rand((1, 5000), device="cuda"), 5)
    assert ei.value.status == 7
