"""GPU parity of the max-convolution entry points against the FP64 oracle.

maxconv_exact: bit-identical to the oracle's FP64 max-convolution rounded to
FP32 (each FP32 product is correctly rounded and max is exact).

maxconv_pnorm (H = FP64 FFT): an FFT convolution of a, b (the powered, scaled
vectors) has an absolute error of about log2(N) 2^-53 (|a|_1 |b|_2 + |b|_1 |a|_2)
per output; the tolerance takes 4 times that bound E for S, adds the relative
error 2 (p - 1) 2^-24 of the FP32 powers, maps both through the root,
(1 + E/S + 2 (p - 1) 2^-24)^(1/p) - 1, and adds the FP32 root and output
roundings.  p_sel may differ from the oracle's only where an oracle S lies
within that band of tau.
"""
import math

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

U64 = 2.0 ** -53


@pytest.fixture(scope="module")
def pn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1511_05690_gb300 as pn
    pn.lib()
    return pn


def _dev(v):
    return torch.from_numpy(np.ascontiguousarray(v, dtype=np.float32)).cuda()


def _pair(batch, nx, ny, seed, kind="wide"):
    g = workloads.rng(seed)
    if kind == "wide":  # exp(-Exponential(4)) as U^(1/4)
        x = (1.0 - g.random((batch, nx))) ** 0.25
        y = (1.0 - g.random((batch, ny))) ** 0.25
    else:
        x = 1.0 - g.random((batch, nx))
        y = 1.0 - g.random((batch, ny))
    return x.astype(np.float32), y.astype(np.float32)


EXACT_SHAPES = [(3, 1, 1), (2, 5, 3), (4, 300, 200), (2, 2500, 3000), (1, 1, 4000),
                (3, 4096, 4096), (2, 9000, 9000), (1, 20000, 300), (1, 300, 20000)]


@pytest.mark.parametrize("shape", EXACT_SHAPES)
def test_maxconv_exact_bit_exact(pn, orc, shape):
    batch, nx, ny = shape
    x, y = _pair(batch, nx, ny, 2100 + nx)
    z = pn.maxconv_exact(_dev(x), _dev(y)).cpu().numpy()
    want = orc.maxconv(x.astype(np.float64), y.astype(np.float64)).astype(np.float32)
    np.testing.assert_array_equal(z, want)


def test_maxconv_exact_strided_and_large_batch(pn, orc):
    x, y = _pair(70000, 3, 2, 2110, kind="uniform")  # batch beyond one grid dimension
    z = pn.maxconv_exact(_dev(x), _dev(y)).cpu().numpy()
    want = orc.maxconv(x.astype(np.float64), y.astype(np.float64)).astype(np.float32)
    np.testing.assert_array_equal(z, want)
    xb = np.zeros((4, 50), np.float32)
    xs, ys = _pair(4, 37, 20, 2111)
    xb[:, :37] = xs
    z = pn.maxconv_exact(_dev(xb)[:, :37], _dev(ys)).cpu().numpy()
    np.testing.assert_array_equal(
        z, orc.maxconv(xs.astype(np.float64), ys.astype(np.float64)).astype(np.float32))


def _fft_err(a, b, N):
    """The absolute error bound E of one FFT convolution output."""
    l1a, l2a = np.abs(a).sum(), np.sqrt((a * a).sum())
    l1b, l2b = np.abs(b).sum(), np.sqrt((b * b).sum())
    return 4 * math.log2(N) * U64 * (l1a * l2b + l1b * l2a)


def _check_pnorm(pn, orc, x, y, pl, tau=1e-12):
    batch, nx = x.shape
    ny = y.shape[1]
    nz = nx + ny - 1
    N = max(2, 1 << math.ceil(math.log2(nz)))
    z, psel = pn.maxconv_pnorm(_dev(x), _dev(y), p_log2=pl, tau=tau)
    z, psel = z.cpu().numpy(), psel.cpu().numpy()
    x64, y64 = x.astype(np.float64), y.astype(np.float64)
    ref = orc.maxconv_pnorm(x64, y64, pl, tau, want_S=True)
    exact = orc.maxconv(x64, y64)
    for b in range(batch):
        sx = x64[b].max() if x64[b].max() > 0 else 1.0
        sy = y64[b].max() if y64[b].max() > 0 else 1.0
        E = np.array([_fft_err((x64[b] / sx) ** 2.0 ** lp, (y64[b] / sy) ** 2.0 ** lp, N)
                      for lp in pl])
        S = ref["S"][b]                                  # (n_p, nz)
        rel = np.array([2 * (2.0 ** lp - 1) * 2.0 ** -24 for lp in pl])
        near = np.any(np.abs(S - tau) <= E[:, None] + rel[:, None] * S, axis=0)
        agree = psel[b] == ref["p_sel"][b]
        assert np.all(agree | near), np.argwhere(~(agree | near))[:5]
        idx = {lp: q for q, lp in enumerate(pl)}
        q = np.array([idx[int(v) & 0x7F] for v in psel[b]])
        S_at = S[q, np.arange(nz)]
        p = 2.0 ** (psel[b] & 0x7F)
        stable = (psel[b] & 0x80) == 0
        want = sx * sy * np.power(np.maximum(S_at, 0.0), 1.0 / p)
        Eq = E[q]
        tol = (1.5 * ((1 + Eq / np.maximum(S_at, 1e-300) + rel[q]) ** (1.0 / p) - 1)
               + 8 * 2.0 ** -24)
        err = np.abs(z[b] - want) / np.maximum(want, 1e-300)
        ok = stable & (want > 0)
        assert np.all(err[ok] <= tol[ok]), (b, float(err[ok].max()))
        # envelope against the exact max-convolution (stable entries)
        L = np.array([min(m, nx - 1) - max(0, m - ny + 1) + 1 for m in range(nz)])
        e = exact[b]
        assert np.all(z[b][ok] >= e[ok] * (1 - tol[ok]) - 1e-30)
        assert np.all(z[b][ok] <= e[ok] * L[ok] ** (1.0 / p[ok]) * (1 + tol[ok]) + 1e-30)
    return z, psel, ref


@pytest.mark.parametrize("shape", [(2, 1, 1), (3, 7, 5), (2, 300, 200), (2, 1000, 1500),
                                   (1, 4096, 4096)])
def test_maxconv_pnorm_matches_oracle(pn, orc, shape):
    batch, nx, ny = shape
    x, y = _pair(batch, nx, ny, 2120 + nx)
    _check_pnorm(pn, orc, x, y, list(range(7)))


def test_maxconv_pnorm_bench_batch(pn, orc):
    """The batch the bench times: 1024 problems of n = 4096 (8191 outputs,
    one CTA each), entries U^(1/4) as in the bench.  Six rows (the first, the
    last and four drawn at random) against the oracle, and the same rows of
    the full batch's launch bit-identical to them."""
    batch, n = 1024, 4096
    g = workloads.rng(None, 5)
    x = ((1.0 - g.random((batch, n))) ** 0.25).astype(np.float32)
    y = ((1.0 - g.random((batch, n))) ** 0.25).astype(np.float32)
    zf, pf = pn.maxconv_pnorm(_dev(x), _dev(y))
    rows = np.unique(np.concatenate([[0, batch - 1], workloads.rng(2140).integers(0, batch, 4)]))
    z, psel, _ = _check_pnorm(pn, orc, x[rows], y[rows], list(range(7)))
    assert np.array_equal(zf.cpu().numpy()[rows], z)
    assert np.array_equal(pf.cpu().numpy()[rows], psel)


def test_maxconv_pnorm_several_levels(pn, orc):
    """Vectors with a few large entries and a small floor: indices far from the
    large ones resolve at small p (S^(p) falls below tau), so p* varies."""
    g = workloads.rng(2130)
    x = (1e-3 * (0.5 + 0.5 * g.random((2, 400)))).astype(np.float32)
    y = (1e-3 * (0.5 + 0.5 * g.random((2, 300)))).astype(np.float32)
    x[:, 17] = 1.0
    y[:, 250] = 1.0
    z, psel, ref = _check_pnorm(pn, orc, x, y, list(range(7)))
    assert len(np.unique(psel & 0x7F)) >= 3


def test_maxconv_pnorm_families_and_tau(pn, orc):
    x, y = _pair(2, 200, 150, 2140, kind="uniform")
    _check_pnorm(pn, orc, x, y, [0, 2, 5])
    _check_pnorm(pn, orc, x, y, [3])
    _check_pnorm(pn, orc, x, y, list(range(7)), tau=1e-6)


def test_maxconv_pnorm_edge_cases(pn, orc):
    z, psel = pn.maxconv_pnorm(torch.zeros((2, 10), device="cuda"),
                               torch.rand((2, 7), device="cuda"))
    assert torch.all(z == 0) and torch.all(psel == 0x80)
    with pytest.raises(pn.PnError) as ei:  # longer than the long path's 2^22 outputs
        pn.maxconv_pnorm(torch.ones((1, 1 << 22), device="cuda"), torch.ones((1, 2), device="cuda"))
    assert ei.value.status == 7
    bad = torch.rand((2, 30), device="cuda")
    bad[1, 3] = -1.0
    with pytest.raises(pn.PnError) as ei:
        pn.maxconv_pnorm(bad, torch.rand((2, 30), device="cuda"))
    assert ei.value.status == 4
    # the context stays usable after a device-detected domain error
    x, y = _pair(1, 20, 20, 2150)
    _check_pnorm(pn, orc, x, y, list(range(7)))


# ---------------------------------------------------------- long problems ---
def _check_long(pn, orc, x, y, pl, m, tau=1e-12):
    """GPU long path against the oracle at the outputs m (plus the FFT bound)."""
    nx, ny = len(x), len(y)
    nz = nx + ny - 1
    N = 1 << max(14, math.ceil(math.log2(nz)))
    z, psel = pn.maxconv_pnorm(_dev(x), _dev(y), p_log2=pl, tau=tau)
    z, psel = z.cpu().numpy()[0], psel.cpu().numpy()[0]
    x64, y64 = x.astype(np.float64), y.astype(np.float64)
    sx, sy = x64.max(), y64.max()
    ex, S = orc.maxconv_entries(x64, y64, m, pl)
    E = np.array([_fft_err((x64 / sx) ** 2.0 ** lp, (y64 / sy) ** 2.0 ** lp, N) for lp in pl])
    rel = np.array([2 * (2.0 ** lp - 1) * 2.0 ** -24 for lp in pl])
    est, ps, _ = orc.estimate(S.T[:, None, :], pl, np.ones(1), np.full(len(m), sx * sy), tau)
    near = np.any(np.abs(S.T - tau) <= E[:, None] + rel[:, None] * S.T, axis=0)
    agree = psel[m] == ps[0]
    assert np.all(agree | near), m[~(agree | near)][:5]
    idx = {lp: q for q, lp in enumerate(pl)}
    q = np.array([idx[int(v) & 0x7F] for v in psel[m]])
    S_at = S[np.arange(len(m)), q]
    p = 2.0 ** (psel[m] & 0x7F)
    want = sx * sy * np.power(np.maximum(S_at, 0.0), 1.0 / p)
    tol = 1.5 * ((1 + E[q] / np.maximum(S_at, 1e-300) + rel[q]) ** (1.0 / p) - 1) + 8 * 2.0 ** -24
    err = np.abs(z[m] - want) / np.maximum(want, 1e-300)
    ok = ((psel[m] & 0x80) == 0) & (want > 0)
    assert np.all(err[ok] <= tol[ok]), float(err[ok].max())
    assert np.all(z[m][ok] >= ex[ok] * (1 - tol[ok]))
    return z, psel


def _sample_outputs(nz, count, seed):
    g = workloads.rng(seed)
    edge = np.concatenate([np.arange(40), np.arange(nz - 40, nz)])
    return np.unique(np.concatenate([edge, g.integers(0, nz, count)]))


@pytest.mark.parametrize("nx,ny", [(6000, 5000), (40000, 30000), (9000, 1)])
def test_maxconv_long_matches_oracle(pn, orc, nx, ny):
    x, y = _pair(1, nx, ny, 2300 + nx)
    m = _sample_outputs(nx + ny - 1, 300, 2301)
    _check_long(pn, orc, x[0], y[0], list(range(7)), m)


def test_maxconv_long_bench_size(pn, orc):
    """The long path at the size the bench times: n = 2^21 per vector (2^22 - 1
    outputs through the four-step transform of length 2^22), entries U^(1/4)
    as in the bench; the 40 outputs at each end and 160 interior ones (about
    2^21 terms each) against the oracle."""
    n = 1 << 21
    g = workloads.rng(None, 6)
    x = ((1.0 - g.random(n)) ** 0.25).astype(np.float32)
    y = ((1.0 - g.random(n)) ** 0.25).astype(np.float32)
    m = _sample_outputs(2 * n - 1, 160, 2330)
    _check_long(pn, orc, x, y, list(range(7)), m)


def test_maxconv_long_several_levels(pn, orc):
    """Small floor and a few spikes: most indices resolve at small p, so the
    open terms stay many and the FFT levels run down the family."""
    g = workloads.rng(2310)
    x = (1e-3 * (0.5 + 0.5 * g.random(12000))).astype(np.float32)
    y = (1e-3 * (0.5 + 0.5 * g.random(9000))).astype(np.float32)
    x[[100, 7000]] = 1.0
    y[4000] = 1.0
    m = _sample_outputs(20999, 400, 2311)
    z, psel = _check_long(pn, orc, x, y, list(range(7)), m)
    assert len(np.unique(psel & 0x7F)) >= 4


def test_maxconv_long_batch_rows_and_exact(pn, orc):
    """Two rows through the long path equal two single calls; the exact
    kernel at this length is bit-identical to the oracle."""
    x, y = _pair(2, 7000, 6000, 2320)
    z, psel = pn.maxconv_pnorm(_dev(x), _dev(y))
    for b in range(2):
        zb, pb = pn.maxconv_pnorm(_dev(x[b]), _dev(y[b]))
        assert torch.equal(z[b], zb[0]) and torch.equal(psel[b], pb[0])
    ze = pn.maxconv_exact(_dev(x), _dev(y)).cpu().numpy()
    want = orc.maxconv(x.astype(np.float64), y.astype(np.float64)).astype(np.float32)
    np.testing.assert_array_equal(ze, want)
