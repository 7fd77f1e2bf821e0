"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a hand-worked
example, a closed form, a library routine (numpy, scipy), an invariant the
paper states, or a second independent algorithm.  Shapes are non-square so a
transposed operand or swapped index fails.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            rows.setdefault(key, []).append([Fraction(v) for v in vals])
    return rows


# ---------------------------------------------------------------- golden ---
def test_hand_worked_3x3(orc):
    """Hand-derived exact values (tests/golden/tiny_3x3.txt)."""
    g = _read_golden("tiny_3x3.txt")
    A = np.array(g["A"], dtype=np.float64)
    B = np.array(g["B"], dtype=np.float64)
    np.testing.assert_array_equal(orc.maxprod(A, B), np.array(g["C"], dtype=np.float64))
    np.testing.assert_array_equal(orc.row_scales(A), np.array(g["r"][0], dtype=np.float64))
    np.testing.assert_array_equal(orc.col_scales(B), np.array(g["c"][0], dtype=np.float64))
    S = orc.psums(A, B, [0, 1])
    np.testing.assert_array_equal(S[0], np.array(g["S1"], dtype=np.float64))
    np.testing.assert_array_equal(S[1], np.array(g["S2"], dtype=np.float64))
    out = orc.pnorm(A, B, [0, 1], tau=0.2)
    np.testing.assert_array_equal(out["p_sel"], np.array(g["psel"], dtype=np.uint8))
    r = np.array(g["r"][0], dtype=np.float64)
    c = np.array(g["c"][0], dtype=np.float64)
    S1 = np.array(g["S1"], dtype=np.float64)
    S2 = np.array(g["S2"], dtype=np.float64)
    psel = np.array(g["psel"])
    expect = np.where(psel == 1, np.sqrt(S2), S1) * r[:, None] * c[None, :]
    np.testing.assert_allclose(out["C"], expect, rtol=1e-15)


def _golden_value(tok):
    """A value of tests/golden/apsp_3node.txt: a rational, inf, ln<k>, or
    sqrt(<rational>) optionally divided by an integer."""
    import re
    if tok == "inf":
        return math.inf
    if tok.startswith("ln"):
        return math.log(int(tok[2:]))
    m = re.fullmatch(r"sqrt\(([0-9/]+)\)(?:/([0-9]+))?", tok)
    if m:
        return math.sqrt(Fraction(m.group(1))) / (int(m.group(2)) if m.group(2) else 1)
    return float(Fraction(tok))


def _read_apsp_golden():
    rows = {}
    with open(os.path.join(GOLDEN, "apsp_3node.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            rows.setdefault(key, []).append(vals)
    return rows


@pytest.mark.parametrize("policy", [1, 2])
def test_hand_worked_apsp_diag_policies(orc, policy):
    """Hand-derived p-norm APSP (tests/golden/apsp_3node.txt): a zero-weight
    edge makes one estimate exceed 1 after the first squaring.  Policy 1
    (diagonal reset) and policy 2 (reset and clamp to x <= 1) give different
    results, both fixed by hand; policy 2 never exceeds x = 1 and stays at or
    above the exact x = exp(-d) (Floyd-Warshall, also in the file).  Dropping
    the clamp gives policy 1's values; clamping only before a squaring leaves
    entries above 1 after the last one; both fail here."""
    g = _read_apsp_golden()
    W = np.array([[_golden_value(t) for t in row] for row in g["W"]])
    pl = [int(t) for t in g["p_log2"][0]]
    tau = float(g["tau"][0][0])
    T = int(g["squarings"][0][0])
    exact = np.array([[_golden_value(t) for t in row] for row in g["exact"]])
    np.testing.assert_allclose(orc.floyd_warshall(W), exact, rtol=1e-15, atol=0)
    want = np.array([[_golden_value(t) for t in row] for row in g[f"X{policy}"]])
    D, _ = orc.apsp_pnorm(W, pl, tau=tau, n_squarings=T, diag_policy=policy)
    X = np.exp(-D)
    np.testing.assert_allclose(X, want, rtol=1e-14)
    assert np.all(np.diag(D) == 0.0)
    x_exact = np.exp(-exact)
    assert np.all(X >= x_exact * (1 - 1e-14))
    if policy == 2:
        assert np.all(X <= 1.0) and np.all(D >= 0.0)
    else:
        assert np.any(X > 1.0 + 1e-3)
    # ceil(log2 n) squarings by default
    D0, _ = orc.apsp_pnorm(W, pl, tau=tau, diag_policy=policy)
    np.testing.assert_array_equal(D0, D)


# ------------------------------------------------------ exact products ---
def test_maxprod_rank_one_closed_form(orc):
    """A = u v^T, B = x y^T  =>  C_ij = u_i y_j max_k v_k x_k."""
    g = workloads.rng(7)
    u, v = g.random(9) + 0.1, g.random(13)
    x, y = g.random(13), g.random(6) + 0.1
    C = orc.maxprod(np.outer(u, v), np.outer(x, y))
    np.testing.assert_allclose(C, np.outer(u, y) * np.max(v * x), rtol=1e-15)


def test_maxprod_permutation(orc):
    """A permutation matrix P gives C = P B (rows of B reordered)."""
    g = workloads.rng(8)
    perm = g.permutation(11)
    P = np.eye(11)[perm]
    B = g.random((11, 5))
    np.testing.assert_array_equal(orc.maxprod(P, B), B[perm])


def test_maxprod_limit_of_ring_products(orc):
    """max_k u_k = lim_p (sum_k u_k^p)^(1/p) (Sec. 1), evaluated by scipy's
    logsumexp at p = 2^20; the gap is at most log(K)/p."""
    from scipy.special import logsumexp
    A, B = workloads.uniform_pair(7, 5, 19, seed=3, dtype=np.float64)
    p = 2.0 ** 20
    L = (np.log(A)[:, :, None] + np.log(B)[None, :, :]) * p
    approx = np.exp(logsumexp(L, axis=1) / p)
    C = orc.maxprod(A, B)
    assert np.all(C <= approx * (1 + 1e-12))
    assert np.all(approx <= C * np.exp(math.log(19) / p) * (1 + 1e-12))


def test_maxprod_f32_is_rounded_f64(orc):
    """Rounding is monotone, so max_k fl32(a b) = fl32(max_k a b) exactly."""
    A, B = workloads.uniform_pair(17, 23, 31, seed=4)
    C32 = orc.maxprod_f32(A, B)
    C64 = orc.maxprod(A.astype(np.float64), B.astype(np.float64))
    np.testing.assert_array_equal(C32, C64.astype(np.float32))


def test_exp_isomorphism_between_minplus_and_maxprod(orc):
    """x = exp(-w) maps (+,min) to (x,max) (Sec. 2.2)."""
    g = workloads.rng(9)
    X, Y = g.random((6, 10)) * 3, g.random((10, 8)) * 3
    np.testing.assert_allclose(orc.maxprod(np.exp(-X), np.exp(-Y)),
                               np.exp(-orc.minplus(X, Y)), rtol=1e-14)


def test_minplus_f32_exact_against_f64(orc):
    g = workloads.rng(10)
    X = g.random((9, 12)).astype(np.float32)
    Y = g.random((12, 7)).astype(np.float32)
    ref = (X.astype(np.float64)[:, :, None] + Y.astype(np.float64)[None]).astype(np.float32)
    np.testing.assert_array_equal(orc.minplus_f32(X, Y), ref.min(axis=1))


def test_ringprod_matches_numpy(orc):
    """Alg. 3 is the ordinary product; compare with numpy's GEMM."""
    A, B = workloads.uniform_pair(13, 7, 29, seed=5, dtype=np.float64)
    np.testing.assert_allclose(orc.ringprod(A, B), A @ B, rtol=1e-13)


def test_empty_reductions(orc):
    A = np.zeros((3, 0))
    B = np.zeros((0, 4))
    assert np.all(orc.maxprod(A, B) == 0.0)
    assert np.all(np.isinf(orc.minplus(A, B)))


# --------------------------------------------------------------- scales ---
def test_scales_are_powers_of_two_bracketing_the_max(orc):
    A, B = workloads.uniform_pair(40, 30, 50, seed=6, dtype=np.float64)
    A *= np.exp(workloads.rng(1).normal(0, 20, size=(40, 1)))
    A[3] = 0.0
    A[5, :] = 0.25  # exact power of two: scale must be 0.25, not 0.5
    r = orc.row_scales(A)
    assert r[3] == 1.0 and r[5] == 0.25
    m, e = np.frexp(r)
    assert np.all(m == 0.5)
    mx = A.max(axis=1)
    nz = mx > 0
    assert np.all(mx[nz] / r[nz] <= 1.0) and np.all(mx[nz] / r[nz] > 0.5)
    c = orc.col_scales(B)
    assert np.all(B.max(axis=0) / c <= 1.0) and np.all(B.max(axis=0) / c > 0.5)
    g = orc.row_scales(A, mode=1)
    assert np.all(g == g[0]) and A.max() / g[0] <= 1.0 and A.max() / g[0] > 0.5
    assert np.all(orc.row_scales(A, mode=0) == 1.0)


# ---------------------------------------------------------------- p-sums ---
def test_p1_equals_ordinary_product(orc):
    """p = 1 gives the ring product (Alg. 3): r_i c_j S^(1)_ij = (A B)_ij."""
    A, B = workloads.wide_range_pair(21, 9, 33, seed=11, dtype=np.float64)
    A *= 3.0
    B *= 0.01
    r, c = orc.row_scales(A), orc.col_scales(B)
    S = orc.psums(A, B, [0])
    np.testing.assert_allclose(S[0] * r[:, None] * c[None, :], A @ B, rtol=1e-13)


def test_psums_monotone_in_p(orc):
    """Scaled terms are <= 1, so S^(p) is non-increasing in p (Sec. 1)."""
    A, B = workloads.uniform_pair(12, 14, 40, seed=12, dtype=np.float64)
    S = orc.psums(A, B, list(range(8)))
    assert np.all(np.diff(S, axis=0) <= 1e-15)


def test_psums_expectation_uniform(orc):
    """For i.i.d. U(0,1] entries with unit scales, E[S^(p)] = K/(p+1)^2."""
    M = N = 64
    K = 512
    A, B = workloads.uniform_pair(M, N, K, seed=13, dtype=np.float64)
    assert np.all(orc.row_scales(A) == 1.0) and np.all(orc.col_scales(B) == 1.0)
    pl = [0, 1, 2, 3, 4]
    S = orc.psums(A, B, pl)
    for q, lp in enumerate(pl):
        p = 2 ** lp
        expect = K / (p + 1) ** 2
        tol = {1: 0.02, 2: 0.03, 4: 0.05, 8: 0.08, 16: 0.12}[p]
        assert abs(S[q].mean() / expect - 1) < tol, (p, S[q].mean(), expect)


# ------------------------------------------------------------- estimator ---
def test_estimator_selection_rule(orc):
    """p* = largest p in P with S^(p) >= tau (Alg. 5); none -> smallest p, flagged."""
    pl = [0, 1, 2, 3]
    S = np.array([[[5.0, 2.0, 1e-3, 0.0]],
                  [[4.0, 1.0, 1e-8, 0.0]],
                  [[3.0, 1e-9, 1e-20, 0.0]],
                  [[2.0, 1e-30, 1e-40, 0.0]]])  # shape (n_p=4, M=1, N=4)
    r = np.array([2.0])
    c = np.array([1.0, 0.5, 4.0, 1.0])
    Chat, psel, Ssel = orc.estimate(S, pl, r, c, tau=1e-6)
    assert list(psel[0]) == [3, 1, 0, 0x80 | 0]
    np.testing.assert_allclose(Chat[0, 0], 2 * 1 * 2.0 ** (1 / 8), rtol=1e-15)
    np.testing.assert_allclose(Chat[0, 1], 2 * 0.5 * 1.0 ** 0.5, rtol=1e-15)
    np.testing.assert_allclose(Chat[0, 2], 2 * 4.0 * 1e-3, rtol=1e-15)
    assert Chat[0, 3] == 0.0
    assert list(Ssel[0]) == [2.0, 1.0, 1e-3, 0.0]


def test_all_ones_upper_envelope_is_tight(orc):
    """A = B = ones(K): S^(p) = K, Chat = K^(1/p*), C = 1 (Sec. 1 bound n^(1/p))."""
    K = 37
    A = np.ones((5, K))
    B = np.ones((K, 6))
    out = orc.pnorm(A, B, [0, 1, 2, 3, 4], tau=1e-30, want_S=True)
    assert np.all(out["S"] == K)
    assert np.all(out["p_sel"] == 4)
    np.testing.assert_allclose(out["C"], K ** (1 / 16), rtol=1e-15)


def test_single_term_is_exact(orc):
    """A with one nonzero per row: every p-norm equals the max (u has one term)."""
    g = workloads.rng(14)
    K = 20
    A = np.zeros((8, K))
    A[np.arange(8), g.integers(0, K, 8)] = g.random(8) + 0.01
    B = g.random((K, 9)) + 0.01
    out = orc.pnorm(A, B, [0, 2, 5], tau=1e-300)
    np.testing.assert_allclose(out["C"], orc.maxprod(A, B), rtol=1e-14)


def test_envelope_and_convergence(orc):
    """C <= Chat <= K^(1/p*) C (Sec. 1), and the gap shrinks as p grows."""
    A, B = workloads.uniform_pair(16, 12, 64, seed=15, dtype=np.float64)
    C = orc.maxprod(A, B)
    prev = None
    for lp in range(0, 8):
        out = orc.pnorm(A, B, [lp], tau=1e-300)
        Chat = out["C"]
        assert np.all(Chat >= C * (1 - 1e-13))
        assert np.all(Chat <= C * 64 ** (1 / 2 ** lp) * (1 + 1e-13))
        if prev is not None:
            assert np.all(Chat <= prev * (1 + 1e-13))
        prev = Chat


def test_convergence_to_max_at_huge_p(orc):
    """With a unit maximal term per entry, p = 2^20 reproduces the max to ~log(K)/p."""
    K = 30
    g = workloads.rng(16)
    A = g.random((6, K)) * 0.9
    B = g.random((K, 7)) * 0.9
    A[:, 0] = 1.0
    B[0, :] = 1.0
    out = orc.pnorm(A, B, [20], tau=1e-300)
    np.testing.assert_allclose(out["C"], orc.maxprod(A, B), rtol=4e-6)


def test_default_tau_reading(orc):
    """tau = K * mu * 2^(m - s) per powered-operand format (reading of Sec. 2.1)."""
    assert orc.default_tau(16384, orc.BF16) == 16384 * 2.0 ** -119
    assert orc.default_tau(16384, orc.F32_EXACT) == 16384 * 2.0 ** -105
    assert orc.default_tau(100, orc.TF32) == 100 * 2.0 ** -116
    assert orc.default_tau(16384, orc.F16) == 16384 * 2.0 ** -19
    assert orc.default_tau(16384, orc.E4M3) == 8.0


# ------------------------------------------------------------------ APSP ---
def test_complete_graph_one_squaring_closed_form(orc):
    """Equal weights w on every edge, x = e^-w, X_ii = 1: for i != j,
    S^(p)_ij = 2 e^(-p w) + (n-2) e^(-2 p w) (k = i or j, or any other k)."""
    n, w = 9, 0.3
    X = np.full((n, n), math.exp(-w))
    np.fill_diagonal(X, 1.0)
    S = orc.psums(X, X, [0, 3, 6])
    for q, p in enumerate([1, 8, 64]):
        expect = 2 * math.exp(-p * w) + (n - 2) * math.exp(-2 * p * w)
        off = S[q][~np.eye(n, dtype=bool)]
        np.testing.assert_allclose(off, expect, rtol=1e-14)


def test_floyd_warshall_matches_scipy(orc):
    from scipy.sparse.csgraph import shortest_path
    W = workloads.apsp_weights(60, density=0.15, seed=17).astype(np.float64)
    D = orc.floyd_warshall(W)
    G = np.where(np.isinf(W), 0.0, W)
    np.fill_diagonal(G, 0.0)
    # scipy treats 0 as "no edge" in dense input; weights here are > 0 a.s.
    ref = shortest_path(G, method="D", directed=True)
    np.testing.assert_allclose(D, ref, rtol=1e-12)


def test_floyd_warshall_matches_repeated_minplus(orc):
    """APSP by repeated (+,min) squaring, ceil(log2 n) times (Sec. 1)."""
    n = 33
    W = workloads.apsp_weights(n, density=0.2, seed=18).astype(np.float64)
    D = W.copy()
    for _ in range(math.ceil(math.log2(n))):
        D = orc.minplus(D, D)
    np.testing.assert_allclose(orc.floyd_warshall(W), D, rtol=1e-14)


def test_apsp_pnorm_underestimates_distance(orc):
    """Chat >= C at every squaring, so the p-norm distance is <= the exact one."""
    n = 64
    W = workloads.apsp_weights(n, density=0.1, seed=19).astype(np.float64)
    D = orc.floyd_warshall(W)
    pl = list(range(7))
    Dh, psel = orc.apsp_pnorm(W, pl, tau=orc.default_tau(n, orc.F32_EXACT))
    finite = np.isfinite(D)
    assert np.all(np.isfinite(Dh) == finite)
    assert np.all(Dh[finite] <= D[finite] + 1e-12)
    assert np.all(np.diag(Dh) == 0.0)


def test_apsp_pnorm_one_squaring_envelope(orc):
    """One squaring: exact 2-hop distance d1 = minplus(W, W) (diagonal 0) and
    d1 - ln(n)/p* <= dhat <= d1, from C <= Chat <= n^(1/p*) C in x = exp(-w)."""
    n = 48
    W = workloads.apsp_weights(n, density=0.2, seed=22).astype(np.float64)
    d1 = orc.minplus(W, W)
    pl = list(range(7))
    Dh, psel = orc.apsp_pnorm(W, pl, tau=orc.default_tau(n, orc.F32_EXACT), n_squarings=1)
    finite = np.isfinite(d1)
    assert np.all(np.isfinite(Dh) == finite)
    p = 2.0 ** (psel & 0x7F)
    off = finite & ~np.eye(n, dtype=bool)
    assert np.all(Dh[off] <= d1[off] + 1e-12)
    assert np.all(Dh[off] >= d1[off] - np.log(n) / p[off] - 1e-12)


# -------------------------------------------------------------- gradient ---
def test_gradient_central_differences(orc):
    """Oracle gradient of L = sum log C against central differences (step 1e-3 rel)."""
    M, N, K = 6, 5, 9
    A, B = workloads.uniform_pair(M, N, K, seed=20, dtype=np.float64)
    pl = [4]  # p fixed at 16
    out = orc.pnorm(A, B, pl, tau=1e-300)
    plog = out["p_sel"] & 0x7F
    G = 1.0 / out["C"]
    dA, dB = orc.pnorm_grad(A, B, plog, G)
    for (i, k) in [(0, 0), (2, 5), (5, 8), (3, 1)]:
        h = 1e-3 * A[i, k]
        ap, am = A[i].copy(), A[i].copy()
        ap[k] += h
        am[k] -= h
        fd = (orc.row_logloss(ap, B, plog[i]) - orc.row_logloss(am, B, plog[i])) / (2 * h)
        assert abs(fd - dA[i, k]) <= 1e-4 * abs(dA[i, k]) + 1e-9, (i, k, fd, dA[i, k])
    for (k, j) in [(0, 0), (4, 2), (8, 4)]:
        h = 1e-3 * B[k, j]
        bp, bm = B[:, j].copy(), B[:, j].copy()
        bp[k] += h
        bm[k] -= h
        fd = (orc.col_logloss(A, bp, plog[:, j]) - orc.col_logloss(A, bm, plog[:, j])) / (2 * h)
        assert abs(fd - dB[k, j]) <= 1e-4 * abs(dB[k, j]) + 1e-9, (k, j, fd, dB[k, j])


def test_gradient_euler_homogeneity(orc):
    """C_ij is homogeneous of degree 1 in row i of A and in column j of B, so
    sum_k a_ik dC_ij/da_ik = C_ij = sum_k b_kj dC_ij/db_kj (one-hot G)."""
    M, N, K = 4, 3, 11
    A, B = workloads.wide_range_pair(M, N, K, seed=21, dtype=np.float64)
    out = orc.pnorm(A, B, [0, 2, 4], tau=1e-300)
    plog = out["p_sel"] & 0x7F
    for (i, j) in [(0, 0), (3, 2), (1, 1)]:
        G = np.zeros((M, N))
        G[i, j] = 1.0
        dA, dB = orc.pnorm_grad(A, B, plog, G)
        np.testing.assert_allclose(np.dot(A[i], dA[i]), out["C"][i, j], rtol=1e-12)
        np.testing.assert_allclose(np.dot(B[:, j], dB[:, j]), out["C"][i, j], rtol=1e-12)
        assert np.all(dA[np.arange(M) != i] == 0.0)


def test_gradient_entries_match_full_gradient(orc):
    """The sampled-entry gradient loops agree with the full-matrix ones."""
    M, N, K = 7, 9, 5
    A, B = workloads.uniform_pair(M, N, K, seed=23, dtype=np.float64)
    out = orc.pnorm(A, B, [0, 3, 5], tau=1e-300)
    plog = out["p_sel"] & 0x7F
    G = workloads.rng(24).random((M, N)) + 0.5
    dA, dB = orc.pnorm_grad(A, B, plog, G)
    ia, ka = np.array([0, 3, 6, 6]), np.array([0, 4, 1, 2])
    kb, jb = np.array([0, 4, 2]), np.array([8, 0, 5])
    eA, eB = orc.pnorm_grad_entries(A, B, plog, G, ia, ka, kb, jb)
    np.testing.assert_allclose(eA, dA[ia, ka], rtol=1e-13)
    np.testing.assert_allclose(eB, dB[kb, jb], rtol=1e-13)


def test_entries_match_full_psums(orc):
    """The selected-entry loops agree with the full p-sum and max-product loops."""
    A, B = workloads.wide_range_pair(23, 17, 41, seed=25, dtype=np.float64)
    pl = [0, 2, 4, 6]
    r, c = orc.row_scales(A), orc.col_scales(B)
    S = orc.psums(A, B, pl)
    g = workloads.rng(26)
    ii, jj = g.integers(0, 23, 50), g.integers(0, 17, 50)
    ex, Se = orc.entries(A, B, ii, jj, pl, r, c)
    np.testing.assert_array_equal(ex, orc.maxprod(A, B)[ii, jj])
    np.testing.assert_allclose(Se, S[:, ii, jj].T, rtol=1e-14)



def test_real_exponent_entries_match_full_sums(orc):
    """The selected-entry loop at real exponents (the 3p/4 family) agrees with
    the full real-exponent sums, and at integer powers of two with the
    selected-entry loop of Alg. 5's sums."""
    A, B = workloads.wide_range_pair(23, 17, 41, seed=27, dtype=np.float64)
    r, c = orc.row_scales(A), orc.col_scales(B)
    g = workloads.rng(28)
    ii, jj = g.integers(0, 23, 50), g.integers(0, 17, 50)
    pw = [0.75, 1.5, 3.0, 6.0, 12.0, 24.0, 48.0]
    Sf = orc.psums_real(A, B, pw, r, c)
    np.testing.assert_allclose(orc.entries_real(A, B, ii, jj, pw, r, c), Sf[:, ii, jj].T,
                               rtol=1e-14)
    _, Se = orc.entries(A, B, ii, jj, [0, 2, 4], r, c)
    np.testing.assert_allclose(orc.entries_real(A, B, ii, jj, [1.0, 4.0, 16.0], r, c), Se,
                               rtol=1e-14)

# ------------------------------------------------------ r = 1 projection ---
# Sec. 2.1 (multiset projection).  With v = (u / max u)^(p*/2) the r = 1
# estimate is max u * (||v||_2^2 / ||v||_1)^(2/p*), which never exceeds max u
# and is smallest, over v in [0,1]^n with v_1 = 1, at the two-valued
# v = (1, lam, ..., lam) with lam = 1/(sqrt(n)+1), where the ratio is
# 2/(sqrt(n)+1).
def _row_product(orc, u, pl, estimator, tau=1e-300):
    """The oracle on the 1 x n by n x 1 product whose only output entry has
    u_k = u[k] (B = ones, so the column scale is 1)."""
    u = np.asarray(u, dtype=np.float64)
    out = orc.pnorm(u[None, :], np.ones((len(u), 1)), pl, tau=tau, estimator=estimator)
    return out["C"][0, 0], out["p_sel"][0, 0]


def test_projection_r1_exact_on_single_valued_rows(orc):
    """All u_k equal: the multiset has one value, which r = 1 recovers exactly
    while the plain norm is K^(1/p*) too large."""
    for beta, K in ((0.3, 7), (0.71, 40), (1.0, 3)):
        c1, ps = _row_product(orc, [beta] * K, [0, 1, 2, 3, 4], 1)
        c0, _ = _row_product(orc, [beta] * K, [0, 1, 2, 3, 4], 0)
        assert ps == 4
        np.testing.assert_allclose(c1, beta, rtol=1e-14)
        np.testing.assert_allclose(c0, beta * K ** (1 / 16), rtol=1e-14)


@pytest.mark.parametrize("n,lp", [(2, 3), (5, 4), (33, 6), (1000, 2)])
def test_projection_r1_two_valued_closed_form(orc, n, lp):
    """u = (1, lam^(2/p*), ...): estimate = ((1+(n-1)lam^2)/(1+(n-1)lam))^(2/p*)."""
    p = 2.0 ** lp
    for lam in (0.0, 0.05, 1 / (math.sqrt(n) + 1), 0.5, 0.999):
        u = [1.0] + [lam ** (2 / p)] * (n - 1)
        est, ps = _row_product(orc, u, list(range(lp + 1)), 1)
        assert ps == lp
        want = ((1 + (n - 1) * lam * lam) / (1 + (n - 1) * lam)) ** (2 / p)
        np.testing.assert_allclose(est, want, rtol=1e-12)


@pytest.mark.parametrize("n", [2, 3, 4, 9])
def test_projection_r1_worst_case_brute_force(orc, n):
    """Brute force over v in [0,1]^n with v_1 = 1: (estimate / max)^(p*/2) =
    ||v||_2^2/||v||_1 >= 2/(sqrt(n)+1), attained at lam = 1/(sqrt(n)+1)."""
    lp = 3
    p = 2.0 ** lp
    bound = 2 / (math.sqrt(n) + 1)
    g = workloads.rng(1601 + n)
    worst = np.inf
    for _ in range(400):
        v = np.concatenate([[1.0], g.random(n - 1) ** g.choice([0.3, 1.0, 3.0])])
        est, _ = _row_product(orc, v ** (2 / p), list(range(lp + 1)), 1)
        worst = min(worst, est ** (p / 2))
    assert worst >= bound * (1 - 1e-12)
    grid = np.linspace(0.0, 1.0, 2001)
    vals = []
    for lam in grid:
        est, _ = _row_product(orc, [1.0] + [lam ** (2 / p)] * (n - 1), list(range(lp + 1)), 1)
        vals.append(est ** (p / 2))
    vals = np.array(vals)
    assert vals.min() >= bound * (1 - 1e-12)
    np.testing.assert_allclose(vals.min(), bound, rtol=1e-5)
    assert abs(grid[np.argmin(vals)] - 1 / (math.sqrt(n) + 1)) <= 1e-3


def test_projection_general_r_matches_and_recovers_multisets(orc):
    """The Hankel null-space construction (Sec. 2.1): r = 1 agrees with the
    oracle's estimator; r = 2 recovers both values of a two-valued multiset and
    r = 1 the value of a one-valued one."""
    g = workloads.rng(1610)
    for _ in range(20):
        u = g.random(int(g.integers(2, 30)))
        lp = int(g.integers(1, 6))
        p = 2.0 ** lp
        est, _ = _row_product(orc, u / u.max(), list(range(lp + 1)), 1)
        half = p / 2
        sums = [np.sum((u / u.max()) ** (m * half)) for m in (1, 2)]
        np.testing.assert_allclose(orc.project(sums, half, 1)[-1], est, rtol=1e-12)
    for b1, h1, b2, h2 in ((0.9, 1, 0.4, 5), (0.8, 3, 0.2, 2), (0.55, 2, 0.5, 7)):
        u = np.array([b1] * h1 + [b2] * h2)
        pp = 4.0
        sums = [np.sum(u ** (m * pp)) for m in (1, 2, 3, 4)]
        np.testing.assert_allclose(orc.project(sums, pp, 2), sorted([b1, b2]), rtol=1e-7)
    sums = [5 * 0.6 ** (m * 8.0) for m in (1, 2)]
    np.testing.assert_allclose(orc.project(sums, 8.0, 1), [0.6], rtol=1e-14)


def test_projection_r1_envelope_on_products(orc):
    """Every entry of a product: exact * (2/(sqrt(K)+1))^(2/p*) <= estimate <= exact."""
    for seed, (M, N, K) in ((1620, (9, 11, 40)), (1621, (13, 7, 300))):
        A, B = workloads.wide_range_pair(M, N, K, seed=seed)
        A, B = A.astype(np.float64), B.astype(np.float64)
        exact = orc.maxprod(A, B)
        out = orc.pnorm(A, B, list(range(7)), tau=orc.default_tau(K, orc.F32_EXACT), estimator=1)
        pstar = 2.0 ** (out["p_sel"] & 0x7F)
        low = exact * (2 / (math.sqrt(K) + 1)) ** (2 / pstar)
        assert np.all(out["C"] <= exact * (1 + 1e-12))
        assert np.all(out["C"] >= low * (1 - 1e-12))


def test_projection_r1_fallbacks_to_plain(orc):
    """No p* / 2 in P (non-consecutive P, or p* = min P), or no stable p: the
    plain estimate."""
    A, B = workloads.uniform_pair(6, 5, 30, seed=1630, dtype=np.float64)
    for pl in ([0, 2, 5], [3]):
        a = orc.pnorm(A, B, pl, tau=1e-300, estimator=0)
        b = orc.pnorm(A, B, pl, tau=1e-300, estimator=1)
        np.testing.assert_array_equal(a["C"], b["C"])
    a = orc.pnorm(A, B, [0, 1, 2], tau=1e300, estimator=0)
    b = orc.pnorm(A, B, [0, 1, 2], tau=1e300, estimator=1)
    assert np.all(b["p_sel"] == 0x80)
    np.testing.assert_array_equal(a["C"], b["C"])


# ------------------------------------------------------ r = 2 projection ---
# Sec. 2.1 with r = 2: the four evenly spaced sums at p*/4, p*/2, 3p*/4, p*
# are the moments m_0..m_3 of the measure with mass w_i x_i at each value
# x_i = u_i^(p*/4); the projection's two values are that measure's 2-point
# Gauss nodes.  Hence the projection recovers any two-valued multiset
# exactly, and its larger node lies between the 1-point node (the r = 1
# estimate) and max u.
@pytest.mark.parametrize("lp", [2, 3, 6])
def test_projection_r2_recovers_two_valued_rows(orc, lp):
    """u with exactly two distinct values: the r = 2 estimate is max u (the
    r = 1 estimate is not, while the low value still carries weight)."""
    pl = list(range(lp + 1))
    for hi, n_hi, lo, n_lo in ((1.0, 1, 0.5, 7), (0.8, 3, 0.79, 40), (0.9, 2, 0.05, 900),
                               (0.37, 5, 0.2, 1)):
        u = [hi] * n_hi + [lo] * n_lo
        est2, ps = _row_product(orc, u, pl, 2)
        est1, _ = _row_product(orc, u, pl, 1)
        assert ps == lp
        np.testing.assert_allclose(est2, hi, rtol=1e-9)
        if n_lo * (lo / hi) ** (2.0 ** lp / 2) > 1e-3 * n_hi:  # the low value still counts
            assert abs(est1 - hi) > 1e-6 * hi


def test_projection_r2_single_valued_rows_keep_r1(orc):
    """One value: s1 s3 = s2^2, the degenerate reading returns the r = 1
    projection, which is exact here."""
    for beta, K in ((0.3, 7), (0.71, 40), (1.0, 3)):
        c2, ps = _row_product(orc, [beta] * K, [0, 1, 2, 3, 4], 2)
        assert ps == 4
        np.testing.assert_allclose(c2, beta, rtol=1e-13)


def test_projection_r2_between_r1_and_exact(orc):
    """Every stable entry of a product: r1 <= r2 <= exact (node interlacing and
    the nodes' support)."""
    for seed, (M, N, K) in ((1640, (9, 11, 40)), (1641, (13, 7, 300)), (1642, (5, 6, 2000))):
        A, B = workloads.wide_range_pair(M, N, K, seed=seed)
        A, B = A.astype(np.float64), B.astype(np.float64)
        exact = orc.maxprod(A, B)
        tau = orc.default_tau(K, orc.F32_EXACT)
        o1 = orc.pnorm(A, B, list(range(7)), tau=tau, estimator=1)
        o2 = orc.pnorm(A, B, list(range(7)), tau=tau, estimator=2)
        assert np.array_equal(o1["p_sel"], o2["p_sel"])
        assert np.all(o2["C"] <= exact * (1 + 1e-12))
        assert np.all(o2["C"] >= o1["C"] * (1 - 1e-12))
        assert np.mean(o2["C"] > o1["C"] * (1 + 1e-9)) > 0.5


def test_projection_r2_matches_general_construction(orc):
    """The closed-form r = 2 (cross product of the Hankel rows) against the
    oracle's SVD null-space construction on random rows."""
    g = workloads.rng(1650)
    for _ in range(30):
        u = g.random(int(g.integers(3, 60)))
        u = u / u.max()
        pp = float(2 ** int(g.integers(0, 4)))
        sums = [np.sum(u ** (m * pp)) for m in (1, 2, 3, 4)]
        np.testing.assert_allclose(orc.project_r2(*sums, pp)[0], orc.project(sums, pp, 2)[-1],
                                   rtol=1e-6)


def test_projection_r2_guard_and_clamp(orc):
    """Exact sums of n ones and one value y^(1/p'): t3 - 1 = s1 s3 / s2^2 - 1 is
    about y / n.  Below the oracle's margin 1e-6 (no second value resolved by
    FP64 sums) the result is the r = 1 value; above it the two values are
    recovered and the estimate is the max, 1.  Perturbed sums (up to 5 %, no
    longer a moment sequence) still give a value between the r = 1 value and
    the plain norm, the interval of the larger Gauss node."""
    g = workloads.rng(1670)
    pp = 4.0
    for n in (1, 3, 17):
        for y, resolved in ((1e-9, False), (1e-7, False), (1e-3, True), (0.3, True)):
            u = np.concatenate([np.ones(n), [y ** (1 / pp)]])
            s = np.array([np.sum(u ** (m * pp)) for m in (1, 2, 3, 4)])
            t = s[2] * s[0] / s[1] ** 2 - 1
            assert (t > 1e-6) == resolved, (n, y, t)
            r1 = (s[1] / s[0]) ** (1 / pp)
            want = 1.0 if resolved else r1
            np.testing.assert_allclose(orc.project_r2(*s, pp)[0], want, rtol=1e-9)
    for _ in range(200):
        u = g.random(int(g.integers(2, 40)))
        u = u / u.max()
        s = np.array([np.sum(u ** (m * pp)) for m in (1, 2, 3, 4)])
        sp = s * (1 + 0.05 * g.uniform(-1, 1, 4))
        v = orc.project_r2(*sp, pp)[0]
        lo, hi = (sp[1] / sp[0]) ** (1 / pp), sp[3] ** (1 / (4 * pp))
        assert min(lo, hi) * (1 - 1e-12) <= v <= max(hi, lo) * (1 + 1e-12)


def test_projection_r2_fallbacks(orc):
    """p*/4 not in P (non-consecutive P, p* among the two smallest p), or no
    stable p: the plain estimate; the 3p/4 sums are the real-power sums."""
    A, B = workloads.uniform_pair(6, 5, 30, seed=1660, dtype=np.float64)
    for pl in ([0, 2, 5], [3], [0, 1]):
        a = orc.pnorm(A, B, pl, tau=1e-300, estimator=0)
        b = orc.pnorm(A, B, pl, tau=1e-300, estimator=2)
        np.testing.assert_array_equal(a["C"], b["C"])
    a = orc.pnorm(A, B, [0, 1, 2], tau=1e300, estimator=0)
    b = orc.pnorm(A, B, [0, 1, 2], tau=1e300, estimator=2)
    assert np.all(b["p_sel"] == 0x80)
    np.testing.assert_array_equal(a["C"], b["C"])
    r, c = orc.row_scales(A), orc.col_scales(B)
    np.testing.assert_allclose(orc.psums_real(A, B, [1.0, 4.0], r, c), orc.psums(A, B, [0, 2], r, c),
                               rtol=1e-14)


# ----------------------------------------------------------- corrections ---
# Sec. 2.1 (dividing by the envelope's upper end K^(1/p*)) and the Discussion
# (an affine model fitted to a few exact sub-solutions), both applied in the
# scaled space where the exact value lies in (0, 1].
def test_affine_fit_is_least_squares(orc):
    """Per class: numpy's degree-1 polyfit; degenerate classes as documented."""
    g = workloads.rng(1800)
    x = g.random(300) + 0.5
    y = 0.7 * x + 0.1 + 0.01 * g.standard_normal(300)
    cls = g.integers(0, 3, 300).astype(np.int32)
    cls[:5] = 4        # class 4: five samples with one x value -> ratio fit
    x[:5] = 1.25
    cls[5] = 5         # class 5: one sample -> ratio fit
    coef = orc.affine_fit(x, y, cls, 7)
    for q in range(3):
        m = cls == q
        a, b = np.polyfit(x[m], y[m], 1)
        np.testing.assert_allclose(coef[q], [a, b], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(coef[4], [y[:5].sum() / x[:5].sum(), 0.0], rtol=1e-12)
    np.testing.assert_allclose(coef[5], [y[5] / x[5], 0.0], rtol=1e-12)
    assert list(coef[3]) == [1.0, 0.0] and list(coef[6]) == [1.0, 0.0]


def test_divide_by_K_envelope(orc):
    """Correction 1: K^(-1/p*) C <= Chat <= C, and all-ones becomes exact."""
    A, B = workloads.uniform_pair(11, 13, 70, seed=1801, dtype=np.float64)
    C = orc.maxprod(A, B)
    out = orc.pnorm(A, B, [0, 1, 2, 3, 4], tau=1e-300, correction=1)
    pstar = 2.0 ** (out["p_sel"] & 0x7F)
    assert np.all(out["C"] <= C * (1 + 1e-13))
    assert np.all(out["C"] >= C * 70 ** (-1 / pstar) * (1 - 1e-13))
    ones = orc.pnorm(np.ones((3, 9)), np.ones((9, 4)), [0, 1, 2], tau=1e-300, correction=1)
    np.testing.assert_allclose(ones["C"], 1.0, rtol=1e-14)


def test_affine_correction_recovers_an_affine_relation(orc):
    """Every u has m equal maxima v (and zeros): the plain estimate is
    m^(1/p*) v, an exactly linear function of the exact value v, so a fit on a
    few samples makes every entry exact."""
    m, K = 6, 40
    g = workloads.rng(1802)
    A = np.zeros((10, K))
    A[:, :m] = 1.0
    B = np.zeros((K, 12))
    B[:m, :] = 0.3 + 0.7 * g.random(12)  # column j: m copies of v_j
    ii, jj = np.array([0, 3, 7]), np.array([1, 5, 11])
    out = orc.pnorm(A, B, list(range(5)), tau=1e-300, correction=2, fit_ij=(ii, jj))
    np.testing.assert_allclose(out["C"], orc.maxprod(A, B), rtol=1e-12)
    np.testing.assert_allclose(out["coef"][4], [m ** (-1 / 16), 0.0], atol=1e-12)


def test_affine_correction_normal_equations(orc):
    """Samples = every entry: per class the residuals of the corrected scaled
    estimate sum to zero and are orthogonal to the uncorrected estimate."""
    A, B = workloads.wide_range_pair(24, 20, 300, seed=1803)
    A, B = A.astype(np.float64), B.astype(np.float64)
    pl = list(range(7))
    tau = orc.default_tau(300, orc.BF16)
    ii, jj = np.meshgrid(np.arange(24), np.arange(20), indexing="ij")
    plain = orc.pnorm(A, B, pl, tau)
    corr = orc.pnorm(A, B, pl, tau, correction=2, fit_ij=(ii.ravel(), jj.ravel()))
    rc = plain["r"][:, None] * plain["c"][None, :]
    x, z, e = plain["C"] / rc, corr["C"] / rc, orc.maxprod(A, B) / rc
    for lp in np.unique(plain["p_sel"] & 0x7F):
        msk = (plain["p_sel"] & 0x7F) == lp
        res = e[msk] - z[msk]
        assert abs(res.sum()) <= 1e-10 * msk.sum()
        assert abs((res * x[msk]).sum()) <= 1e-10 * msk.sum()


def test_affine_correction_reduces_error(orc):
    """Wide-range entries (K = 2000, BF16 threshold): 256 exact samples bring
    the median relative error of both estimators down by more than 5x."""
    A, B = workloads.wide_range_pair(120, 110, 2000, seed=1804)
    A, B = A.astype(np.float64), B.astype(np.float64)
    g = workloads.rng(1805)
    ii, jj = g.integers(0, 120, 256), g.integers(0, 110, 256)
    tau = orc.default_tau(2000, orc.BF16)
    exact = orc.maxprod(A, B)
    for est in (0, 1):
        e0 = np.median(np.abs(orc.pnorm(A, B, list(range(7)), tau, estimator=est)["C"] - exact)
                       / exact)
        c2 = orc.pnorm(A, B, list(range(7)), tau, estimator=est, correction=2, fit_ij=(ii, jj))
        e2 = np.median(np.abs(c2["C"] - exact) / exact)
        assert e2 < e0 / 5, (est, e0, e2)


# ------------------------------------------------------- max-convolution ---
# Sec. 1: z_m = max_i x_i y_(m-i) and its p-norm estimate from ring
# convolutions of the powered, max-scaled vectors.
def _toeplitz(x, ny):
    nz = len(x) + ny - 1
    T = np.zeros((nz, ny))
    for m in range(nz):
        for t in range(ny):
            if 0 <= m - t < len(x):
                T[m, t] = x[m - t]
    return T


def test_maxconv_equals_maxprod_with_toeplitz(orc):
    """max_i x_i y_(m-i) is the (x,max) product of the Toeplitz matrix of x
    with y (Alg. 2 on a structured operand)."""
    g = workloads.rng(2000)
    for nx, ny in ((1, 1), (5, 3), (17, 29)):
        x, y = g.random(nx), g.random(ny)
        T = _toeplitz(x, ny)
        np.testing.assert_array_equal(orc.maxconv(x, y)[0], orc.maxprod(T, y[:, None])[:, 0])


def test_maxconv_pnorm_equals_pnorm_with_toeplitz(orc):
    """The p-norm max-convolution is the p-norm product of the Toeplitz matrix of
    x with the column y (Sec. 1 and Alg. 5 on a structured operand), computed by
    independent code.  With max x = max y = 1 the vector scaling and the
    product's global power-of-two scaling (scaling = 1) both leave the values
    unchanged, so the sums, p* and the estimate agree at a binding tau; with
    other maxima and every p stable the estimate, which does not depend on the
    scales, still agrees."""
    g = workloads.rng(2002)
    pl = list(range(7))
    seen = set()
    for nx, ny in ((1, 1), (6, 4), (40, 33), (200, 170)):
        x, y = g.random(nx), g.random(ny)
        x[g.integers(nx)] = 1.0
        y[g.integers(ny)] = 1.0
        T = _toeplitz(x, ny)
        mc = orc.maxconv_pnorm(x, y, pl, tau=1e-3, want_S=True)
        pr = orc.pnorm(T, y[:, None], pl, tau=1e-3, scaling=1, want_S=True)
        assert np.array_equal(mc["p_sel"][0], pr["p_sel"][:, 0])
        np.testing.assert_allclose(mc["S"][0], pr["S"][:, :, 0], rtol=1e-13, atol=1e-300)
        np.testing.assert_allclose(mc["z"][0], pr["C"][:, 0], rtol=1e-13)
        seen |= set(np.unique(mc["p_sel"][0] & 0x7F).tolist())
        x2, y2 = 3.7 * g.random(nx), 0.3 * g.random(ny)
        mc2 = orc.maxconv_pnorm(x2, y2, pl, tau=1e-300)
        pr2 = orc.pnorm(_toeplitz(x2, ny), y2[:, None], pl, tau=1e-300, scaling=1)
        assert np.all(mc2["p_sel"][0] == 6) and np.all(pr2["p_sel"][:, 0] == 6)
        np.testing.assert_allclose(mc2["z"][0], pr2["C"][:, 0], rtol=1e-13)
    assert len(seen) >= 3  # tau = 1e-3 selects several p*


def test_conv_matches_numpy(orc):
    g = workloads.rng(2001)
    x, y = g.random((3, 40)), g.random((3, 25))
    want = np.array([np.convolve(x[b], y[b]) for b in range(3)])
    np.testing.assert_allclose(orc.conv(x, y), want, rtol=1e-13)


def test_maxconv_pnorm_p1_is_convolution(orc):
    g = workloads.rng(2002)
    x, y = g.random((2, 30)) + 0.1, g.random((2, 20)) + 0.1
    out = orc.maxconv_pnorm(x, y, [0], tau=1e-300)
    want = np.array([np.convolve(x[b], y[b]) for b in range(2)])
    np.testing.assert_allclose(out["z"], want, rtol=1e-13)


def test_maxconv_pnorm_envelope_and_all_ones(orc):
    """z <= zhat <= L_m^(1/p*) z with L_m the number of terms of index m, and
    tight for all-ones vectors; zhat tends to z as p grows."""
    g = workloads.rng(2003)
    nx, ny = 50, 37
    x, y = g.random(nx), g.random(ny)
    z = orc.maxconv(x, y)[0]
    L = np.array([min(m, nx - 1) - max(0, m - ny + 1) + 1 for m in range(nx + ny - 1)])
    prev = None
    for lp in range(0, 9):
        zh = orc.maxconv_pnorm(x, y, [lp], tau=1e-300)["z"][0]
        assert np.all(zh >= z * (1 - 1e-13))
        assert np.all(zh <= z * L ** (1.0 / 2 ** lp) * (1 + 1e-13))
        if prev is not None:
            assert np.all(zh <= prev * (1 + 1e-13))
        prev = zh
    ones = orc.maxconv_pnorm(np.ones(nx), np.ones(ny), [0, 2, 4], tau=1e-12)
    assert np.all(ones["p_sel"] == 4)
    np.testing.assert_allclose(ones["z"][0], L ** (1 / 16), rtol=1e-14)


def test_maxconv_pnorm_selection_with_tau(orc):
    """The largest p with S >= tau is taken per index; a single-term index is
    exact at any p.  x = y = (1, 1e-3): S^(p)_0 = 1, S^(p)_1 = 2 (1e-3)^p,
    S^(p)_2 = (1e-6)^p; with tau = 0.9e-12 p* is 64, 4 and 2."""
    x = np.array([1.0, 1e-3])
    out = orc.maxconv_pnorm(x, x, [0, 1, 2, 3, 4, 5, 6], tau=0.9e-12, want_S=True)
    assert list(out["p_sel"][0]) == [6, 2, 1]
    np.testing.assert_allclose(out["z"][0], [1.0, 2 ** (1 / 4) * 1e-3, 1e-6], rtol=1e-12)
    out = orc.maxconv_pnorm(x, x, [0, 1, 2], tau=1e-3)
    assert out["p_sel"][0][2] == 0x80 | 0


def test_maxconv_pnorm_sums_match_fft_convolution(orc):
    """The p-sums are ring convolutions: numpy's FFT convolution of the
    powered scaled vectors agrees to FFT rounding (a few 1e-16 of the largest)."""
    g = workloads.rng(2004)
    x, y = g.random(300) ** 0.25, g.random(200) ** 0.25
    pl = [0, 2, 4, 6]
    out = orc.maxconv_pnorm(x, y, pl, tau=1e-300, want_S=True)
    nz = 499
    for q, lp in enumerate(pl):
        p = 2.0 ** lp
        a, b = (x / x.max()) ** p, (y / y.max()) ** p
        f = np.fft.irfft(np.fft.rfft(a, 512) * np.fft.rfft(b, 512), 512)[:nz]
        scale = np.sqrt(np.sum(a * a) * np.sum(b * b))
        assert np.max(np.abs(f - out["S"][0, q])) <= 1e-13 * scale


def test_maxconv_limit_of_ring_convolutions(orc):
    """log z_m = lim_p (1/p) log sum_i exp(p (log x_i + log y_(m-i))) by scipy's
    logsumexp at p = 2^12 (Sec. 1), independent of the oracle's loops."""
    from scipy.special import logsumexp
    g = workloads.rng(2005)
    x, y = g.random(23) + 0.05, g.random(31) + 0.05
    z = orc.maxconv(x, y)[0]
    p = 2.0 ** 12
    for m in range(53):
        terms = [p * (np.log(x[i]) + np.log(y[m - i])) for i in range(23) if 0 <= m - i < 31]
        est = np.exp(logsumexp(terms) / p)
        assert z[m] <= est * (1 + 1e-12) and est <= z[m] * len(terms) ** (1 / p) * (1 + 1e-12)


def test_maxconv_entries_match_full(orc):
    """Selected outputs equal the full oracle's (max and every p-sum)."""
    g = workloads.rng(2200)
    x, y = g.random(120) ** 0.25, g.random(90) ** 0.25
    pl = [0, 2, 4, 6]
    full = orc.maxconv_pnorm(x, y, pl, tau=1e-300, want_S=True)
    m = np.array([0, 1, 50, 118, 119, 150, 208])
    ex, S = orc.maxconv_entries(x, y, m, pl)
    np.testing.assert_array_equal(ex, orc.maxconv(x, y)[0][m])
    np.testing.assert_allclose(S, full["S"][0][:, m].T, rtol=1e-14)


# ------------------------------------------------------------ top-k of xy ---
def test_topk_recover_indices_brute_force(orc):
    """Every (i, j): m1 = i + j and m2 = i + n - 1 - j give back (i, j)."""
    n = 7
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    i, j = orc.recover_indices((ii + jj).ravel(), (ii + n - 1 - jj).ravel(), n)
    np.testing.assert_array_equal(i, ii.ravel())
    np.testing.assert_array_equal(j, jj.ravel())
    i, j = orc.recover_indices([3, 12, -1], [4, 12, 2], n)  # parity / range / missing
    assert list(i) == [-1, -1, -1] and list(j) == [-1, -1, -1]


def test_topk_single_term_diagonals_are_exact(orc):
    """Diagonals with one term are popped exactly, once, then exhausted; the
    two-term diagonal of n = 2 (0.27 and 0.2) gives estimates within its
    envelope (p* = 16: 0.3^16 >= 1e-12 > 0.3^32)."""
    v, d = orc.topk_xy([0.5], [0.8], 3, list(range(13)))
    np.testing.assert_allclose(v[0], 0.4, rtol=1e-14)
    assert d[0] == 0 and list(d[1:]) == [-1, -1]
    x, y = np.array([1.0, 0.3]), np.array([0.9, 0.2])
    v, d = orc.topk_xy(x, y, 5, list(range(13)))
    assert list(d) == [0, 1, 1, 2, -1]
    np.testing.assert_allclose(v[[0, 3]], [0.9, 0.06], rtol=1e-12)
    assert 0.27 <= v[1] <= 0.27 * 2 ** (1 / 16)
    assert abs(v[2] - 0.2) <= 0.02 * 0.2


def test_topk_monotone_and_close_to_exact(orc):
    """Emitted values never increase; with P = {1..4096} they match the exact
    top-k of x_i y_j within 0.5 %, and the first is within the
    L^(1/4096) envelope of the exact max."""
    g = workloads.rng(2400)
    n = 300
    x, y = g.random(n), g.random(n)
    exact = np.sort(np.outer(x, y).ravel())[::-1]
    v, d = orc.topk_xy(x, y, 150, list(range(13)))
    assert np.all(np.diff(v) <= 1e-15 * v[:-1])
    np.testing.assert_allclose(v, exact[:150], rtol=5e-3)
    assert exact[0] <= v[0] <= exact[0] * n ** (1 / 4096) * (1 + 1e-12)


def test_topk_recovered_indices_are_valid(orc):
    """The two calls (y and reversed y) give index pairs; the consistent ones
    (x_i y_j within 1 % of the estimate) are the top products themselves."""
    g = workloads.rng(2401)
    n = 400
    x, y = g.random(n), g.random(n)
    v, d1 = orc.topk_xy(x, y, 40, list(range(13)))
    _, d2 = orc.topk_xy(x, y, 40, list(range(13)), y_rev=True)
    i, j = orc.recover_indices(d1, d2, n)
    ok = i >= 0
    cons = ok.copy()
    cons[ok] = np.abs(x[i[ok]] * y[j[ok]] - v[ok]) <= 1e-2 * v[ok]
    assert cons.sum() >= 20
    exact = np.sort(np.outer(x, y).ravel())[::-1][:60]
    assert np.all(np.isin(np.round(x[i[cons]] * y[j[cons]], 14), np.round(exact, 14)))
