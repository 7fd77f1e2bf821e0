"""GPU parity of the exact and p-norm (x,max) products against the FP64 oracle.

Calls go through the C ABI (ctypes binding).  Tolerances are derived from the
arithmetic of each operand format (see ``pnorm_tol``).
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


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


# Unit roundoff of the powered operands and mantissa bits m of the tau reading.
_U = {"f32": 2.0 ** -21, "tf32": 2.0 ** -11, "bf16": 2.0 ** -8, "f16": 2.0 ** -11, "e4m3": 2.0 ** -4}
_M = {"f32": 21, "tf32": 10, "bf16": 7, "f16": 10, "e4m3": 3}
_CODE = {"f32": 0, "tf32": 1, "bf16": 2, "f16": 3, "e4m3": 4}


def s_tol(mode, K, plog):
    """Relative error bound of the GPU's p-sum S^(p) against the FP64 oracle:
    x^p by log2(p) FP32 squarings carries up to (p-1) 2^-24 per operand (each
    squaring doubles the error and adds one rounding), the cast to the operand
    format adds u per operand, flushed operands can drop up to 2^-m of S (tau
    reading), and FP32 accumulation of K nonnegative terms adds at most K 2^-23."""
    p = 2.0 ** plog
    return 2 * (p - 1) * 2.0 ** -24 + 2 * _U[mode] + 2.0 ** -_M[mode] + K * 2.0 ** -23


def pnorm_tol(mode, K, plog):
    """Relative tolerance of Chat at p* = 2^plog: the 1/p root maps a relative
    error e of S to (1 + e)^(1/p) - 1, plus a few FP32 roundings of root and scale."""
    return 1.5 * ((1 + s_tol(mode, K, plog)) ** (1.0 / 2 ** plog) - 1) + 2e-7


# ------------------------------------------------------------------ exact ---
EXACT_SHAPES = [(1, 1, 1), (7, 13, 5), (129, 257, 65), (300, 200, 1000), (128, 128, 8),
                (64, 3, 130)]


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("shape", EXACT_SHAPES)
def test_exact_maxprod_bit_exact(pn, orc, shape, variant):
    M, N, K = shape
    A, B = workloads.uniform_pair(M, N, K, seed=100 + M)
    C = pn.maxprod_exact(_dev(A), _dev(B), variant=variant).cpu().numpy()
    np.testing.assert_array_equal(C, orc.maxprod_f32(A, B))


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("shape", [(7, 13, 5), (129, 257, 65), (33, 70, 300)])
def test_exact_minplus_bit_exact(pn, orc, shape, variant):
    M, N, K = shape
    g = workloads.rng(200 + M)
    X = (g.random((M, K)) * 10).astype(np.float32)
    Y = (g.random((K, N)) * 10).astype(np.float32)
    X[g.random((M, K)) < 0.3] = np.inf
    C = pn.maxprod_exact(_dev(X), _dev(Y), semiring=1, variant=variant).cpu().numpy()
    np.testing.assert_array_equal(C, orc.minplus_f32(X, Y))


def test_exact_strided_operands(pn, orc):
    A, B = workloads.uniform_pair(50, 40, 30, seed=5)
    Abig = np.zeros((50, 37), np.float32)
    Abig[:, :30] = A
    dA = _dev(Abig)[:, :30]
    C = pn.maxprod_exact(dA, _dev(B)).cpu().numpy()
    np.testing.assert_array_equal(C, orc.maxprod_f32(A, B))


def test_exact_empty_k(pn):
    A = torch.zeros((5, 0), device="cuda")
    B = torch.zeros((0, 6), device="cuda")
    C = pn.maxprod_exact(A, B).cpu().numpy()
    assert np.all(C == 0.0)
    C = pn.maxprod_exact(A, B, semiring=1).cpu().numpy()
    assert np.all(np.isinf(C))


# ----------------------------------------------------------------- p-norm ---
def _compare(pn, orc, A, B, mode, plog_list, tau=None, tile_n=0, scaling=2, tile_m=0):
    M, K = A.shape
    tau = orc.default_tau(K, _CODE[mode]) if tau is None else tau
    C, psel, ssel = pn.maxprod_pnorm(_dev(A), _dev(B), p_log2=plog_list, compute=mode, tau=tau,
                                     tile_n=tile_n, scaling=scaling, tile_m=tile_m)
    C, psel, ssel = C.cpu().numpy(), psel.cpu().numpy(), ssel.cpu().numpy()
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    ref = orc.pnorm(A64, B64, plog_list, tau, scaling=scaling, want_S=True)
    S = ref["S"]
    # p_sel equals the oracle's except where the oracle's S sits at tau within
    # the operand-format error band
    near = np.zeros(C.shape, dtype=bool)
    for q, lp in enumerate(plog_list):
        near |= np.abs(S[q] / tau - 1) < 4 * s_tol(mode, K, lp)
    agree = psel == ref["p_sel"]
    assert np.all(agree | near), f"p_sel mismatch at {np.argwhere(~(agree | near))[:5]}"
    # value at the GPU's own p*: oracle (S^(p*))^(1/p*) r c
    idx = {lp: q for q, lp in enumerate(plog_list)}
    q_gpu = np.vectorize(lambda b: idx[int(b) & 0x7F])(psel)
    S_at = np.take_along_axis(S, q_gpu[None], axis=0)[0]
    pstar = 2.0 ** (psel & 0x7F)
    expect = ref["r"][:, None] * ref["c"][None, :] * np.power(S_at, 1.0 / pstar)
    tol = np.vectorize(lambda lp: pnorm_tol(mode, K, lp))(psel & 0x7F)
    err = np.abs(C - expect) / np.maximum(expect, 1e-300)
    bad = (err > tol) & (expect > 0)
    assert not np.any(bad), (f"{mode}: max rel err {err[expect > 0].max():.3e}, "
                             f"worst at {np.argwhere(bad)[:5]}")
    if mode == "f32":
        # the FP32 (3xTF32) bar: 1e-5 relative against the FP64 oracle everywhere
        assert err[expect > 0].max(initial=0.0) <= 1e-5, float(err[expect > 0].max())
    assert np.all(C[expect == 0] == 0)
    # S_sel is the scaled p-sum at p*
    serr = np.abs(ssel - S_at) / np.maximum(S_at, 1e-300)
    stol = 1.5 * np.vectorize(lambda lp: s_tol(mode, K, lp))(psel & 0x7F) + 1e-7
    assert np.all((serr <= stol) | (S_at == 0)), f"S_sel max rel err {serr.max():.3e}"
    # envelope of Sec. 1: exact <= Chat <= K^(1/p*) exact (up to the same tolerance)
    exact = orc.maxprod(A64, B64)
    assert np.all(C >= exact * (1 - tol) - 1e-30)
    assert np.all(C <= exact * K ** (1.0 / pstar) * (1 + tol) + 1e-30)
    return C, psel, ssel, err


PN_SHAPES = [(1, 1, 1), (5, 7, 3), (130, 300, 257), (129, 129, 33), (200, 64, 500)]


@pytest.mark.parametrize("shape", PN_SHAPES)
def test_pnorm_f32_small_shapes(pn, orc, shape):
    M, N, K = shape
    A, B = workloads.uniform_pair(M, N, K, seed=300 + M + N)
    _compare(pn, orc, A, B, "f32", list(range(7)))


def test_pnorm_f32_config_n256(pn, orc):
    """n = 256, P = {1, ..., 128}, Uniform(0,1] (FP64 draws rounded to FP32)."""
    A, B = workloads.uniform_pair(256, 256, 256, index=0, dtype=np.float64)
    _, _, _, err = _compare(pn, orc, A.astype(np.float32), B.astype(np.float32), "f32",
                            list(range(8)))
    assert err.max() <= 1e-5


@pytest.mark.parametrize("mode", ["bf16", "f16", "e4m3", "tf32"])
@pytest.mark.parametrize("tile_n", [128, 256])
def test_pnorm_modes(pn, orc, mode, tile_n):
    A, B = workloads.wide_range_pair(260, 300, 384, seed=400)
    tau = None
    if mode == "f16":
        tau = orc.default_tau(384, 3)
    _compare(pn, orc, A, B, mode, list(range(7)), tau=tau, tile_n=tile_n)


def _multilevel_inputs(M, N, K, seed):
    """Rows of A peak at column i mod K, columns of B at row (j+1) mod K, with
    small cross terms: most entries have max product ~0.05 (unstable at large
    p), entries with i = j + 1 (mod K) have max 1 (stable at p_max)."""
    g = workloads.rng(seed)
    A = (0.05 * (0.5 + 0.5 * g.random((M, K)))).astype(np.float32)
    B = (0.05 * (0.5 + 0.5 * g.random((K, N)))).astype(np.float32)
    A[np.arange(M), np.arange(M) % K] = 1.0
    B[(np.arange(N) + 1) % K, np.arange(N)] = 1.0
    return A, B


@pytest.mark.parametrize("mode", ["f32", "bf16"])
def test_pnorm_lower_levels(pn, orc, mode):
    """Tiles that are not stable at p_max go down the family (work lists, state bits)."""
    A, B = _multilevel_inputs(300, 400, 256, seed=500)
    C, psel, _, _ = _compare(pn, orc, A, B, mode, list(range(7)))
    levels = set(np.unique(psel & 0x7F).tolist())
    assert len(levels) >= 2, levels


def test_pnorm_unstable_flag(pn, orc):
    """No p stable: smallest p with the 0x80 flag (tau above every S)."""
    A, B = workloads.uniform_pair(40, 50, 60, seed=7)
    C, psel, _, _ = _compare(pn, orc, A, B, "f32", [2, 4], tau=1e6)
    assert np.all(psel == (0x80 | 2))


def test_pnorm_single_p(pn, orc):
    A, B = workloads.uniform_pair(150, 170, 90, seed=8)
    _compare(pn, orc, A, B, "f32", [4])


@pytest.mark.parametrize("scaling", [0, 1])
def test_pnorm_scaling_modes(pn, orc, scaling):
    A, B = workloads.uniform_pair(70, 90, 110, seed=9)
    _compare(pn, orc, A, B, "f32", list(range(7)), scaling=scaling)


def test_pnorm_zero_rows_and_cols(pn, orc):
    A, B = workloads.uniform_pair(70, 90, 110, seed=10)
    A[3] = 0
    B[:, 5] = 0
    C, psel, _, _ = _compare(pn, orc, A, B, "f32", list(range(7)))
    assert np.all(C[3] == 0) and np.all(C[:, 5] == 0)
    assert np.all(psel[3] == 0x80) and np.all(psel[:, 5] == 0x80)


def test_pnorm_empty_dims(pn):
    z = torch.zeros
    C, psel, ssel = pn.maxprod_pnorm(z((4, 0), device="cuda"), z((0, 3), device="cuda"))
    assert torch.all(C == 0) and torch.all(psel == 0x80) and torch.all(ssel == 0)
    C, _, _ = pn.maxprod_pnorm(z((0, 5), device="cuda"), z((5, 3), device="cuda"))
    assert C.shape == (0, 3)


def test_pnorm_domain_error(pn):
    A, B = workloads.uniform_pair(20, 30, 40, seed=11)
    A[2, 3] = -1.0
    with pytest.raises(pn.PnError) as ei:
        pn.maxprod_pnorm(_dev(A), _dev(B))
    assert ei.value.status == 4
    A[2, 3] = np.nan
    with pytest.raises(pn.PnError):
        pn.maxprod_pnorm(_dev(A), _dev(B))
    # the context is still usable
    A[2, 3] = 0.5
    pn.maxprod_pnorm(_dev(A), _dev(B))


@pytest.mark.parametrize("shape", [(20, 30, 40), (130, 260, 1024)])
@pytest.mark.parametrize("where", ["A", "B"])
def test_pnorm_domain_values(pn, shape, where):
    """Inputs must lie in [0, 2^127]: a negative value, +-inf, NaN or a value
    above 2^127 anywhere in either operand gives PN_EDOMAIN, in the maxima
    pass's 16-byte path (full aligned segments: K = 1024 rows of A, 128 columns
    x 256 rows of B) and in its scalar path (K = 40, N = 30); -0 acts as 0 and
    2^127 itself is accepted."""
    M, N, K = shape
    A, B = workloads.uniform_pair(M, N, K, seed=12)
    X = A if where == "A" else B
    pos = (M // 2, K - 1) if where == "A" else (K - 1, N // 2)
    for bad in (-1.0, np.nan, np.inf, -np.inf, 3.0e38):
        X[pos] = bad
        with pytest.raises(pn.PnError) as ei:
            pn.maxprod_pnorm(_dev(A), _dev(B))
        assert ei.value.status == 4, bad
    X[pos] = 0.0
    C0, p0, _ = pn.maxprod_pnorm(_dev(A), _dev(B))
    X[pos] = -0.0
    C1, p1, _ = pn.maxprod_pnorm(_dev(A), _dev(B))
    assert torch.equal(C0, C1) and torch.equal(p0, p1)
    X[pos] = 2.0 ** 127
    C2, _, _ = pn.maxprod_pnorm(_dev(A), _dev(B))
    assert torch.isfinite(C2).all()


def test_pnorm_host_errors(pn):
    import ctypes
    L = pn.lib()
    o = pn.make_opts(tile_n=256, tile_m=128)  # a fixed tile shape: the size query is then exact
    A = torch.rand(64, 64, device="cuda")
    C = torch.empty(64, 64, device="cuda")
    need = L.pn_workspace_size(64, 64, 64, ctypes.byref(o))
    ws = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    args = (64, 64, 64, A.data_ptr(), 64, A.data_ptr(), 64, C.data_ptr(), 64, None, None)
    assert L.maxprod_pnorm(*args, ctypes.byref(o), ws.data_ptr(), need - 1, s) == 3
    assert L.maxprod_pnorm(*args, ctypes.byref(o), ws.data_ptr() + 16, need, s) == 2
    bad = pn.make_opts()
    bad.n_p = 0
    assert L.maxprod_pnorm(*args, ctypes.byref(bad), ws.data_ptr(), need, s) == 1
    assert L.maxprod_pnorm(64, 64, 64, A.data_ptr(), 10, A.data_ptr(), 64, C.data_ptr(), 64,
                           None, None, ctypes.byref(o), ws.data_ptr(), need, s) == 1
    assert L.maxprod_pnorm(*args, ctypes.byref(o), ws.data_ptr(), need, s) == 0
    torch.cuda.synchronize()


def test_pnorm_large_sampled_entries(pn, orc):
    """n = 16384, entries exp(-Exp(4)), BF16 and E4M3 operands, 4096 sampled entries
    checked against the FP64 oracle at the GPU's p*."""
    n = 16384
    A, B = workloads.wide_range_pair(n, n, n)
    ii, jj = workloads.wide_range_entries(n, 4096)
    dA, dB = _dev(A), _dev(B)
    r = orc.row_scales(A[np.unique(ii)].astype(np.float64))  # only sampled rows needed
    rr = np.zeros(n)
    rr[np.unique(ii)] = r
    c = orc.col_scales(B.astype(np.float64))
    pl = list(range(7))
    exact, S = orc.entries(A, B, ii, jj, pl, rr, c)
    for mode in ["bf16", "e4m3"]:
        C, psel, _ = pn.maxprod_pnorm(dA, dB, p_log2=pl, compute=mode)
        Cs = C[torch.from_numpy(ii).cuda(), torch.from_numpy(jj).cuda()].cpu().numpy()
        ps = psel[torch.from_numpy(ii).cuda(), torch.from_numpy(jj).cuda()].cpu().numpy()
        q = (ps & 0x7F).astype(np.int64)
        S_at = S[np.arange(len(ii)), q]
        expect = rr[ii] * c[jj] * np.power(S_at, 1.0 / 2.0 ** q)
        tol = np.array([pnorm_tol(mode, n, int(x)) for x in q])
        err = np.abs(Cs - expect) / expect
        assert np.all(err <= tol), (mode, err.max())
        assert np.all(Cs >= exact * (1 - tol))
        assert np.all(Cs <= exact * n ** (1.0 / 2.0 ** q) * (1 + tol))
        del C, psel


# ------------------------------------------------- top-level image paths ---
@pytest.mark.parametrize("mode", ["f32", "tf32", "bf16", "e4m3"])
@pytest.mark.parametrize("shape", [(203, 261, 517), (128, 256, 64), (5, 1000, 33)])
def test_tensor_copy_images_match_per_tile_images(pn, mode, shape):
    """Operands whose rows are 16-byte aligned get their top-level images from
    one 2-D tensor copy per tile (zeros past M, N, K); unaligned rows from the
    per-tile kernels.  Both build the same bytes, so the same values stored with
    a padded row pitch (aligned) and contiguously (odd pitch) give bit-identical
    C, p_sel and S_sel -- across ragged M, N, K tails and several p levels."""
    M, N, K = shape
    g = workloads.rng(2700 + M)
    # entries 0.025..0.05 with one 1 per row of A and per column of B: the
    # products through a matching pair are 1, all others at most 0.05, so
    # p* spreads over several levels
    A = (0.05 * (0.5 + 0.5 * g.random((M, K)))).astype(np.float32)
    B = (0.05 * (0.5 + 0.5 * g.random((K, N)))).astype(np.float32)
    A[np.arange(M), np.arange(M) % K] = 1.0
    B[(np.arange(N) + 1) % K, np.arange(N)] = 1.0
    Ap = torch.zeros((M, K + (4 - K % 4) % 4 + 4), dtype=torch.float32, device="cuda")
    Bp = torch.zeros((K, N + (4 - N % 4) % 4 + 4), dtype=torch.float32, device="cuda")
    Ap[:, :K] = _dev(A)
    Bp[:, :N] = _dev(B)
    Av, Bv = Ap[:, :K], Bp[:, :N]
    assert Av.stride(0) % 4 == 0 and Bv.stride(0) % 4 == 0
    # odd pitch: every row but the first misaligned
    Ao = torch.zeros((M, K + 1 + K % 2), dtype=torch.float32, device="cuda")[:, :K]
    Bo = torch.zeros((K, N + 1 + N % 2), dtype=torch.float32, device="cuda")[:, :N]
    Ao.copy_(Av)
    Bo.copy_(Bv)
    if M > 1:
        assert Ao.stride(0) % 2 == 1
    C1, p1, s1 = pn.maxprod_pnorm(Av, Bv, compute=mode)
    C2, p2, s2 = pn.maxprod_pnorm(Ao, Bo, compute=mode)
    assert torch.equal(p1, p2)
    assert torch.equal(C1, C2)
    assert torch.equal(s1, s2)
    assert len(torch.unique(p1 & 0x7F)) >= 2  # several levels took part
