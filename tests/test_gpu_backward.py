"""GPU parity of the adjoint (maxprod_pnorm_backward) against the FP64 oracle.

Loss L = sum_ij log C_ij, so dL/dC = 1/C.  The GPU gradient comes from the
GPU forward's own outputs (C, S_sel, p_sel); the oracle gradient from the
oracle's own forward.  Tolerance (relative, every gradient entry is a sum of
nonnegative terms here): the two powered operands carry up to (p-1) 2^-24 each
from their squaring chains, the 3xTF32 products about 3 * 2^-21, FP32
accumulation over the contraction length L at most L * 2^-23, and the
elementwise factor a few 2^-24.
"""
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


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def grad_tol(plog, L):
    p = 2.0 ** plog
    return 1.5 * (2 * (p - 1) * 2.0 ** -24 + 3 * 2.0 ** -21 + L * 2.0 ** -23 + 8 * 2.0 ** -24)


def rel_err(g, r):
    """Relative error, 0 where both are 0."""
    return np.abs(g - r) / np.maximum(np.abs(r), 1e-300)


def grad_ok(g, r, tol):
    """Every entry within tol relative, plus FP32's subnormal spacing 2^-149:
    an exact entry below the FP32 range can only be stored to that spacing."""
    return bool(np.all(np.abs(g.astype(np.float64) - r) <= tol * np.abs(r) + 2.0 ** -149))


def _gpu_fwd_bwd(pn, A, B, pl, tau):
    dA_, dB_ = _dev(A), _dev(B)
    C, psel, ssel = pn.maxprod_pnorm(dA_, dB_, p_log2=pl, compute="f32", tau=tau)
    G = 1.0 / C
    gA, gB = pn.maxprod_pnorm_backward(dA_, dB_, C, ssel, psel, G, p_log2=pl, compute="f32",
                                       tau=tau)
    return psel.cpu().numpy(), gA.cpu().numpy(), gB.cpu().numpy()


def _multilevel_inputs(M, N, K, seed):
    g = workloads.rng(seed)
    A = (0.05 * (0.5 + 0.5 * g.random((M, K)))).astype(np.float32)
    B = (0.05 * (0.5 + 0.5 * g.random((K, N)))).astype(np.float32)
    A[np.arange(M), np.arange(M) % K] = 1.0
    B[(np.arange(N) + 1) % K, np.arange(N)] = 1.0
    return A, B


# (40, 90, 33) at p = 64: short contractions make W = 1/S large, so gradient
# entries stay in the FP32 range while the factor a'^(p-1) (a' < 0.25) does not
CASES = [((64, 48, 80), [4], "uniform"), ((130, 200, 257), list(range(7)), "uniform"),
         ((129, 77, 33), [0, 2, 5], "uniform"), ((150, 170, 128), list(range(7)), "multilevel"),
         ((40, 90, 33), [6], "uniform")]


@pytest.mark.parametrize("shape,pl,data", CASES)
def test_backward_matches_oracle_gradient(pn, orc, shape, pl, data):
    M, N, K = shape
    if data == "uniform":
        A, B = workloads.uniform_pair(M, N, K, seed=700 + M)
    else:
        A, B = _multilevel_inputs(M, N, K, seed=701)
    tau = orc.default_tau(K, orc.F32_EXACT)
    psel, gA, gB = _gpu_fwd_bwd(pn, A, B, pl, tau)
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    ref = orc.pnorm(A64, B64, pl, tau)
    assert np.array_equal(psel, ref["p_sel"])  # same p* everywhere (data away from tau)
    if data == "multilevel":
        assert len(np.unique(psel & 0x7F)) >= 2
    rA, rB = orc.pnorm_grad(A64, B64, ref["p_sel"], 1.0 / ref["C"])
    pmax = int(np.max(psel & 0x7F))
    assert grad_ok(gA, rA, grad_tol(pmax, N)), rel_err(gA, rA)[rA >= 2.0 ** -126].max()
    assert grad_ok(gB, rB, grad_tol(pmax, M)), rel_err(gB, rB)[rB >= 2.0 ** -126].max()


@pytest.mark.parametrize("pl", [[4], list(range(7))])
def test_backward_n2048_sampled(pn, orc, pl):
    """n = 2048, Uniform(0,1]: p fixed at 16, and stable p over {1..64}.  64
    sampled entries of dA and of dB against the oracle's analytic gradient and
    against central differences (relative step 1e-3) of the oracle's forward."""
    n = 2048
    A, B = workloads.uniform_pair(n, n, n, index=2)
    tau = orc.default_tau(n, orc.F32_EXACT)
    psel, gA, gB = _gpu_fwd_bwd(pn, A, B, pl, tau)
    g = workloads.rng(None, 102)
    ia, ka = g.integers(0, n, 64), g.integers(0, n, 64)
    kb, jb = g.integers(0, n, 64), g.integers(0, n, 64)
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    r, c = orc.row_scales(A64), orc.col_scales(B64)
    # the oracle's own p* and C on the rows ia and columns jb it needs
    plog = np.full((n, n), pl[-1], dtype=np.uint8)
    G = np.ones((n, n))
    rows_i = np.repeat(np.unique(ia), n)
    cols_j = np.tile(np.arange(n), len(np.unique(ia)))
    rows_c = np.tile(np.arange(n), len(np.unique(jb)))
    cols_c = np.repeat(np.unique(jb), n)
    ei = np.concatenate([rows_i, rows_c])
    ej = np.concatenate([cols_j, cols_c])
    _, S = orc.entries(A64, B64, ei, ej, pl, r, c)
    stable = S >= tau
    q = np.where(stable.any(axis=1), len(pl) - 1 - np.argmax(stable[:, ::-1], axis=1), 0)
    lp = np.array(pl)[q]
    S_at = S[np.arange(len(ei)), q]
    Cq = r[ei] * c[ej] * np.power(S_at, 1.0 / 2.0 ** lp)
    plog[ei, ej] = lp
    G[ei, ej] = 1.0 / Cq
    assert np.array_equal(psel[ei, ej] & 0x7F, lp)  # GPU forward chose the same p*
    rA, rB = orc.pnorm_grad_entries(A64, B64, plog, G, ia, ka, kb, jb)
    pmax = int(lp.max())
    assert grad_ok(gA[ia, ka], rA, grad_tol(pmax, n)), rel_err(gA[ia, ka], rA).max()
    assert grad_ok(gB[kb, jb], rB, grad_tol(pmax, n)), rel_err(gB[kb, jb], rB).max()
    # central differences of the oracle's FP64 forward (p* held fixed)
    fdA, fdB = [], []
    for i, k in zip(ia[:64], ka[:64]):
        h = 1e-3 * A64[i, k]
        ap, am = A64[i].copy(), A64[i].copy()
        ap[k] += h
        am[k] -= h
        fdA.append((orc.row_logloss(ap, B64, plog[i]) - orc.row_logloss(am, B64, plog[i])) / (2 * h))
    for k, j in zip(kb[:64], jb[:64]):
        h = 1e-3 * B64[k, j]
        bp, bm = B64[:, j].copy(), B64[:, j].copy()
        bp[k] += h
        bm[k] -= h
        fdB.append((orc.col_logloss(A64, bp, plog[:, j]) - orc.col_logloss(A64, bm, plog[:, j]))
                   / (2 * h))
    fdA, fdB = np.array(fdA), np.array(fdB)
    # central differences of x^p at relative step e are off by about
    # (p-1)(p-2) e^2 / 6 (6.5e-4 at p = 64, e = 1e-3); a loss difference below
    # FP64 resolution (|L| 2^-52 / 2h) makes the difference quotient 0
    p = 2.0 ** pmax
    fd_rel = 1e-4 + 1.5 * (p - 1) * (p - 2) * 1e-6 / 6
    LA = np.array([abs(orc.row_logloss(A64[i], B64, plog[i])) for i in ia])
    LB = np.array([abs(orc.col_logloss(A64, B64[:, j], plog[:, j])) for j in jb])
    resA = 8 * 2.0 ** -52 * (LA + 1) / (2e-3 * A64[ia, ka])
    resB = 8 * 2.0 ** -52 * (LB + 1) / (2e-3 * B64[kb, jb])
    assert np.all(np.abs(gA[ia, ka] - fdA) <= fd_rel * np.abs(fdA) + resA)
    assert np.all(np.abs(gB[kb, jb] - fdB) <= fd_rel * np.abs(fdB) + resB)


@pytest.mark.parametrize("mode", ["f32", "tf32", "bf16"])
@pytest.mark.parametrize("shape", [(300, 520, 384), (256, 300, 700)])
def test_backward_pairs_equal_single(pn, orc, mode, shape):
    """The gradient GEMMs on CTA pairs (256 x 256 tiles; automatic for larger
    products) give dA and dB bit-identical to one CTA per tile -- with odd
    counts of 128-row blocks on either GEMM's output rows (300 rows of dA,
    384 and 700 rows of dB, padded with a zero block), and entries selected
    at several p.  The 3xTF32 case is also held to the oracle's gradient."""
    M, N, K = shape
    A, B = _multilevel_inputs(M, N, K, seed=720 + K)
    pl = list(range(7))
    tau = orc.default_tau(K, {"f32": orc.F32_EXACT, "tf32": orc.TF32, "bf16": orc.BF16}[mode])
    dA_, dB_ = _dev(A), _dev(B)
    C, psel, ssel = pn.maxprod_pnorm(dA_, dB_, p_log2=pl, compute=mode, tau=tau)
    assert len(torch.unique(psel & 0x7F)) >= 2
    G = 1.0 / C
    got = pn.maxprod_pnorm_backward(dA_, dB_, C, ssel, psel, G, p_log2=pl, compute=mode, tau=tau)
    one = pn.maxprod_pnorm_backward(dA_, dB_, C, ssel, psel, G, p_log2=pl, compute=mode, tau=tau,
                                    tile_m=128)
    pair = pn.maxprod_pnorm_backward(dA_, dB_, C, ssel, psel, G, p_log2=pl, compute=mode,
                                     tau=tau, tile_m=256)
    for x, y, z in zip(got, one, pair):
        assert torch.equal(x, z) and torch.equal(y, z)
    if mode == "f32":
        A64, B64 = A.astype(np.float64), B.astype(np.float64)
        ref = orc.pnorm(A64, B64, pl, tau)
        assert np.array_equal(psel.cpu().numpy(), ref["p_sel"])
        rA, rB = orc.pnorm_grad(A64, B64, ref["p_sel"], 1.0 / ref["C"])
        pmax = int(np.max(ref["p_sel"] & 0x7F))
        assert grad_ok(pair[0].cpu().numpy(), rA, grad_tol(pmax, N))
        assert grad_ok(pair[1].cpu().numpy(), rB, grad_tol(pmax, M))


def test_backward_bf16_mode(pn, orc):
    """BF16 operands: error stated against the oracle (BF16 u = 2^-8 per operand)."""
    M, N, K = 200, 190, 300
    A, B = workloads.uniform_pair(M, N, K, seed=710)
    tau = orc.default_tau(K, orc.BF16)
    dA_, dB_ = _dev(A), _dev(B)
    C, psel, ssel = pn.maxprod_pnorm(dA_, dB_, compute="bf16", tau=tau)
    gA, gB = pn.maxprod_pnorm_backward(dA_, dB_, C, ssel, psel, 1.0 / C, compute="bf16", tau=tau)
    ref = orc.pnorm(A.astype(np.float64), B.astype(np.float64), list(range(7)), tau)
    assert np.array_equal(psel.cpu().numpy(), ref["p_sel"])
    rA, rB = orc.pnorm_grad(A, B, ref["p_sel"], 1.0 / ref["C"])
    bound = 1.5 * (2 * 63 * 2.0 ** -24 + 3 * 2.0 ** -8 + 2.0 ** -7 + 300 * 2.0 ** -23)
    assert grad_ok(gA.cpu().numpy(), rA, bound) and grad_ok(gB.cpu().numpy(), rB, bound)


def test_backward_edge_cases(pn):
    z = torch.zeros
    A = torch.rand(5, 4, device="cuda")
    B = torch.rand(4, 0, device="cuda")
    C = z((5, 0), device="cuda")
    gA, gB = pn.maxprod_pnorm_backward(A, B, C, C, torch.zeros((5, 0), dtype=torch.uint8,
                                                               device="cuda"), C)
    assert torch.all(gA == 0) and gB.shape == (4, 0)
    with pytest.raises(pn.PnError) as ei:
        A = torch.rand(8, 8, device="cuda")
        C, psel, ssel = pn.maxprod_pnorm(A, A, compute="f32")
        pn.maxprod_pnorm_backward(A, A, C, ssel, psel, C, compute="e4m3")
    assert ei.value.status == 7


def test_autograd_function(pn):
    A, B = workloads.uniform_pair(96, 80, 112, seed=720)
    tA = _dev(A).requires_grad_(True)
    tB = _dev(B).requires_grad_(True)
    C, psel, ssel = pn.PNormMaxProd.apply(tA, tB)
    C.log().sum().backward()
    dA, dB = pn.maxprod_pnorm_backward(tA.detach(), tB.detach(), C.detach(), ssel, psel,
                                       1.0 / C.detach())
    assert torch.equal(tA.grad, dA) and torch.equal(tB.grad, dB)
