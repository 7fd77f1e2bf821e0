"""FP64 CPU oracle for the p-norm (x,max) semiring product (arXiv 1511.05690).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the GPU library (``paper_1511_05690_gb300``)
and never imports it.

The arithmetic lives in ``oracle.c`` (plain loops, FP64, OpenMP over output
rows); this module only loads it and marshals numpy arrays.  Functions and the
passages they follow:

* ``maxprod`` / ``maxprod_f32`` -- Alg. 2 (naive (x,max) product).
* ``minplus`` / ``minplus_f32`` -- Alg. 1 (naive (+,min) product).
* ``ringprod`` -- Alg. 3 (naive (x,+) product).
* ``row_scales`` / ``col_scales`` -- the scaled H' of Sec. 2.1 (power-of-two
  reading, see ``oracle.c``).
* ``psums`` -- Alg. 5 first loop: S^(p) = (A'^p)(B'^p) for every p in P.
* ``psums_real`` / ``entries_real`` -- the same sums at real exponents (the
  3p/4 family that the r = 2 projection of Sec. 2.1 needs), all entries /
  selected entries.
* ``estimate`` -- Alg. 5 second loop: estimateMaxFromNormPowerSequence in the
  plain form (largest stable p), or the multiset projection of Sec. 2.1 with
  r = 1 (estimator 1) or r = 2 (estimator 2).
* ``project`` -- the projection of Sec. 2.1 for any r from its Hankel matrix
  (a general construction the r = 1 and r = 2 paths are checked against).
* ``project_r2`` -- the r = 2 projection from its four sums (Sec. 2.1).
* ``pnorm`` -- scales, sums and estimate together.
* ``entries`` -- exact max and p-sums at selected entries only.
* ``affine_fit`` / ``fit_coefficients`` / ``apply_correction`` -- the bias
  corrections (Sec. 2.1 bound remark; Discussion): division by K^(1/p*), and
  a least-squares affine map per p* class from exactly solved samples.
* ``floyd_warshall`` -- exact APSP (the comparison of Sec. 3.1).
* ``apsp_pnorm`` -- Sec. 2.2: exp(-W), repeated p-norm squaring, -log.
* ``pnorm_grad`` / ``pnorm_grad_entries`` -- gradient of the p-norm product at
  fixed p per entry (all entries / selected entries); ``row_logloss`` /
  ``col_logloss`` are the losses its finite-difference pins use.
* ``maxconv`` / ``conv`` -- naive max-convolution (Sec. 1) and the naive ring
  convolution an FFT computes.
* ``maxconv_pnorm`` / ``maxconv_entries`` -- the p-norm estimate of the
  max-convolution (Sec. 1 with the scaling of Sec. 2.1), all outputs /
  selected outputs.
* ``topk_xy`` / ``recover_indices`` -- approximate top-k of x_i y_j (Alg. 9
  with the NormQueue) and the index recovery from two calls.
* ``default_tau`` -- the stability threshold reading (Sec. 2.1, tau).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# compute-mode numbers used by default_tau (same meaning as the library's
# pn_compute enum, written out here independently).
F32_EXACT, TF32, BF16, F16, E4M3 = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (OpenMP if available)."""
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-ffp-contract=off", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            i64, dbl, vp, ci = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_int
            for name in ("orc_maxprod_f64", "orc_maxprod_f32", "orc_minplus_f64",
                         "orc_minplus_f32", "orc_ringprod_f64"):
                getattr(lib, name).argtypes = [i64, i64, i64, vp, i64, vp, i64, vp, i64]
                getattr(lib, name).restype = None
            lib.orc_row_scales.argtypes = [i64, i64, vp, i64, ci, vp]
            lib.orc_col_scales.argtypes = [i64, i64, vp, i64, ci, vp]
            lib.orc_psums.argtypes = [i64, i64, i64, vp, i64, vp, i64, vp, vp, ci, vp, vp]
            lib.orc_estimate.argtypes = [i64, i64, ci, vp, vp, vp, vp, dbl, vp, vp, vp]
            lib.orc_estimate_ex.argtypes = [i64, i64, ci, vp, vp, vp, vp, dbl, ci, vp, vp, vp]
            lib.orc_estimate_ex2.argtypes = [i64, i64, ci, vp, vp, vp, vp, vp, dbl, ci, vp,
                                             vp, vp]
            lib.orc_pnorm_ex2.argtypes = [i64, i64, i64, vp, i64, vp, i64, ci, vp, dbl, ci, ci,
                                          vp, vp, vp, vp, vp, vp]
            lib.orc_pnorm_ex2.restype = ci
            lib.orc_psums_real.argtypes = [i64, i64, i64, vp, i64, vp, i64, vp, vp, ci, vp, vp]
            lib.orc_entries_real.argtypes = [i64, vp, i64, vp, i64, vp, vp, ci, vp, i64, vp, vp,
                                             vp]
            lib.orc_project_r2.argtypes = [dbl, dbl, dbl, dbl, dbl]
            lib.orc_project_r2.restype = dbl
            lib.orc_project_r2_batch.argtypes = [i64, vp, vp, vp, vp, dbl, vp]
            lib.orc_pnorm.argtypes = [i64, i64, i64, vp, i64, vp, i64, ci, vp, dbl, ci,
                                      vp, vp, vp, vp, vp, vp]
            lib.orc_pnorm.restype = ci
            lib.orc_pnorm_ex.argtypes = [i64, i64, i64, vp, i64, vp, i64, ci, vp, dbl, ci, ci,
                                         vp, vp, vp, vp, vp, vp]
            lib.orc_pnorm_ex.restype = ci
            lib.orc_maxconv.argtypes = [i64, i64, vp, i64, vp, vp]
            lib.orc_topk_xy.argtypes = [i64, vp, vp, ci, ci, vp, dbl, i64, vp, vp]
            lib.orc_maxconv_entries.argtypes = [i64, vp, i64, vp, ci, vp, i64, vp, vp, vp]
            lib.orc_conv.argtypes = [i64, i64, vp, i64, vp, vp]
            lib.orc_maxconv_pnorm.argtypes = [i64, i64, vp, i64, vp, ci, vp, dbl, vp, vp, vp]
            lib.orc_affine_fit.argtypes = [i64, vp, vp, vp, ci, vp]
            lib.orc_apply_correction.argtypes = [i64, i64, i64, ci, vp, ci, vp, vp, vp, vp, vp]
            lib.orc_entries.argtypes = [i64, i64, i64, vp, i64, vp, i64, vp, vp, ci, vp,
                                        i64, vp, vp, vp, vp]
            lib.orc_floyd_warshall.argtypes = [i64, vp, i64]
            lib.orc_apsp_pnorm.argtypes = [i64, vp, i64, ci, ci, vp, dbl, ci, ci, vp, i64, vp]
            lib.orc_apsp_pnorm.restype = ci
            lib.orc_pnorm_grad.argtypes = [i64, i64, i64, vp, vp, vp, vp, vp, vp, vp, vp]
            lib.orc_pnorm_grad_entries.argtypes = [i64, i64, i64, vp, vp, vp, vp, vp, vp, i64, vp,
                                                   vp, vp, i64, vp, vp, vp]
            lib.orc_row_logloss.argtypes = [i64, i64, vp, vp, vp]
            lib.orc_row_logloss.restype = dbl
            lib.orc_col_logloss.argtypes = [i64, i64, vp, vp, vp]
            lib.orc_col_logloss.restype = dbl
            lib.orc_default_tau.argtypes = [i64, ci]
            lib.orc_default_tau.restype = dbl
            lib.orc_num_threads.restype = ci
            lib.orc_set_num_threads.argtypes = [ci]
            _lib = lib
    return _lib


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def _f32(x):
    return np.ascontiguousarray(x, dtype=np.float32)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _plog(p_log2):
    return np.ascontiguousarray(p_log2, dtype=np.int32)


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_num_threads(n: int) -> None:
    _load().orc_set_num_threads(int(n))


def default_tau(K: int, compute: int) -> float:
    return float(_load().orc_default_tau(int(K), int(compute)))


def _prod(fn, A, B, conv, out_dtype):
    A, B = conv(A), conv(B)
    M, K = A.shape
    K2, N = B.shape
    assert K == K2
    C = np.empty((M, N), dtype=out_dtype)
    fn(M, N, K, _p(A), K, _p(B), N, _p(C), N)
    return C


def maxprod(A, B):
    """Alg. 2 in FP64: C_ij = max_k a_ik b_kj."""
    return _prod(_load().orc_maxprod_f64, A, B, _f64, np.float64)


def maxprod_f32(A, B):
    """Alg. 2 with FP32 products (bit-exact reference for the GPU exact kernel)."""
    return _prod(_load().orc_maxprod_f32, A, B, _f32, np.float32)


def minplus(A, B):
    """Alg. 1 in FP64: C_ij = min_k a_ik + b_kj."""
    return _prod(_load().orc_minplus_f64, A, B, _f64, np.float64)


def minplus_f32(A, B):
    return _prod(_load().orc_minplus_f32, A, B, _f32, np.float32)


def ringprod(A, B):
    """Alg. 3 in FP64: C_ij = sum_k a_ik b_kj (plain triple loop)."""
    return _prod(_load().orc_ringprod_f64, A, B, _f64, np.float64)


def row_scales(A, mode: int = 2):
    A = _f64(A)
    M, K = A.shape
    r = np.empty(M, dtype=np.float64)
    _load().orc_row_scales(M, K, _p(A), K, int(mode), _p(r))
    return r


def col_scales(B, mode: int = 2):
    B = _f64(B)
    K, N = B.shape
    c = np.empty(N, dtype=np.float64)
    _load().orc_col_scales(K, N, _p(B), N, int(mode), _p(c))
    return c


def psums(A, B, p_log2, r=None, c=None, scaling: int = 2):
    """S[q] = sum_k (a_ik/r_i * b_kj/c_j)^(2^p_log2[q]); shape (n_p, M, N)."""
    A, B = _f64(A), _f64(B)
    M, K = A.shape
    _, N = B.shape
    r = row_scales(A, scaling) if r is None else _f64(r)
    c = col_scales(B, scaling) if c is None else _f64(c)
    pl = _plog(p_log2)
    S = np.empty((len(pl), M, N), dtype=np.float64)
    _load().orc_psums(M, N, K, _p(A), K, _p(B), N, _p(r), _p(c), len(pl), _p(pl), _p(S))
    return S


def estimate(S, p_log2, r, c, tau: float, estimator: int = 0, S34=None):
    """Largest stable p per entry; returns (Chat, p_sel, S_sel).  estimator 1
    replaces the root by the r = 1 projection from S^(p*/2) and S^(p*);
    estimator 2 by the r = 2 projection, which also needs S34[q] = the sums
    at 3 p_q / 4 (same shape as S)."""
    S = _f64(S)
    n_p, M, N = S.shape
    pl = _plog(p_log2)
    assert len(pl) == n_p
    r, c = _f64(r), _f64(c)
    if estimator == 2:
        S34 = _f64(S34)
        assert S34.shape == S.shape
    Chat = np.empty((M, N), dtype=np.float64)
    psel = np.empty((M, N), dtype=np.uint8)
    Ssel = np.empty((M, N), dtype=np.float64)
    _load().orc_estimate_ex2(M, N, n_p, _p(pl), _p(S), _p(S34) if S34 is not None else None,
                             _p(r), _p(c), float(tau), int(estimator), _p(Chat),
                             _p(psel), _p(Ssel))
    return Chat, psel, Ssel


def project_r2(s1, s2, s3, s4, p_prime: float):
    """The r = 2 multiset projection (Sec. 2.1) of the four evenly spaced
    power sums s_m = sum_i u_i^(m p'), elementwise over arrays (see oracle.c):
    sums with s1 s3 - s2^2 <= 1e-6 s2^2 (no second value resolved by exact
    sums) give the r = 1 value."""
    s1, s2, s3, s4 = np.broadcast_arrays(*(np.asarray(x, dtype=np.float64) for x in (s1, s2, s3, s4)))
    s1, s2, s3, s4 = (np.ascontiguousarray(x).ravel() for x in (s1, s2, s3, s4))
    out = np.empty(len(s1), dtype=np.float64)
    _load().orc_project_r2_batch(len(s1), _p(s1), _p(s2), _p(s3), _p(s4), float(p_prime),
                                 _p(out))
    return out


def psums_real(A, B, powers, r, c):
    """S[q] = sum_k (a_ik/r_i * b_kj/c_j)^powers[q] for real powers; (n_p, M, N)."""
    A, B = _f64(A), _f64(B)
    M, K = A.shape
    _, N = B.shape
    pw = _f64(np.asarray(powers, dtype=np.float64))
    r, c = _f64(r), _f64(c)
    S = np.empty((len(pw), M, N), dtype=np.float64)
    _load().orc_psums_real(M, N, K, _p(A), K, _p(B), N, _p(r), _p(c), len(pw), _p(pw), _p(S))
    return S


def entries_real(A, B, ii, jj, powers, r, c):
    """p-sums at real powers at the entries (ii[e], jj[e]); shape (n_e, n_p)."""
    A, B = _f64(A), _f64(B)
    M, K = A.shape
    _, N = B.shape
    ii = np.ascontiguousarray(ii, dtype=np.int64)
    jj = np.ascontiguousarray(jj, dtype=np.int64)
    pw = _f64(np.asarray(powers, dtype=np.float64))
    r, c = _f64(r), _f64(c)
    S = np.empty((len(ii), len(pw)), dtype=np.float64)
    _load().orc_entries_real(K, _p(A), K, _p(B), N, _p(r), _p(c), len(pw), _p(pw), len(ii),
                             _p(ii), _p(jj), _p(S))
    return S


def affine_fit(est, exact, cls, n_cls: int):
    """Least-squares exact = a_q est + b_q per class q (Discussion); (n_cls, 2)."""
    est, exact = _f64(est), _f64(exact)
    cls = np.ascontiguousarray(cls, dtype=np.int32)
    coef = np.empty((n_cls, 2), dtype=np.float64)
    _load().orc_affine_fit(len(est), _p(est), _p(exact), _p(cls), int(n_cls), _p(coef))
    return coef


def pnorm(A, B, p_log2, tau: float, scaling: int = 2, want_S: bool = False,
          estimator: int = 0, correction: int = 0, fit_ij=None):
    """Full p-norm estimate of the (x,max) product (Alg. 5 with H = Alg. 3).
    estimator 0 is the plain largest-stable-p norm, 1 the r = 1 projection,
    2 the r = 2 projection (with the sums at 3p/4, computed here).
    correction 1 divides by K^(1/p*); correction 2 fits the affine model of
    the Discussion on the sample entries fit_ij = (ii, jj) and applies it.

    Returns a dict with Chat, p_sel, S_sel, r, c, coef (correction 2) and
    (if want_S) S_all; Chat is the corrected estimate.
    """
    A, B = _f64(A), _f64(B)
    M, K = A.shape
    K2, N = B.shape
    assert K == K2
    if estimator == 2 and correction == 2:
        raise ValueError("the affine correction is defined for estimators 0 and 1")
    pl = _plog(p_log2)
    Chat = np.empty((M, N), dtype=np.float64)
    psel = np.empty((M, N), dtype=np.uint8)
    Ssel = np.empty((M, N), dtype=np.float64)
    r = np.empty(M, dtype=np.float64)
    c = np.empty(N, dtype=np.float64)
    S = np.empty((len(pl), M, N), dtype=np.float64) if want_S else None
    rc = _load().orc_pnorm_ex2(M, N, K, _p(A), K, _p(B), N, len(pl), _p(pl), float(tau),
                               int(scaling), int(estimator), _p(Chat), _p(psel),
                               _p(Ssel), _p(S) if S is not None else None, _p(r), _p(c))
    if rc:
        raise MemoryError("oracle pnorm allocation failed")
    coef = None
    if correction == 2:
        ii, jj = (np.asarray(x, dtype=np.int64) for x in fit_ij)
        coef = fit_coefficients(A, B, ii, jj, pl, r, c, tau, estimator)
    if correction:
        apply_correction(Chat, psel, pl, K, r, c, correction, coef)
    out = dict(C=Chat, p_sel=psel, S_sel=Ssel, r=r, c=c, coef=coef)
    if want_S:
        out["S"] = S
    return out


def project(sums, p_prime: float, r: int):
    """Multiset projection of Sec. 2.1 for one vector u.

    sums[m-1] = ||u||_{m p'}^{m p'} = sum_i u_i^(m p') for m = 1 .. 2r.  The
    r x (r+1) Hankel matrix H[i][j] = sums[i + j] (the paper's matrix of
    power sums at p', 2p', ...) has a null vector gamma; the roots a of
    sum_i gamma_i a^i are the projected values alpha^p', and the estimate of
    max_i u_i is max alpha = max a^(1/p').  Returns all alpha (ascending).
    """
    sums = np.asarray(sums, dtype=np.float64)
    assert len(sums) >= 2 * r
    H = np.array([[sums[i + j] for j in range(r + 1)] for i in range(r)])
    _, _, vt = np.linalg.svd(H)
    gamma = vt[-1]                        # spans the null space when rank(H) = r
    roots = np.roots(gamma[::-1])         # np.roots wants the highest power first
    roots = np.real(roots[np.abs(np.imag(roots)) <= 1e-9 * np.maximum(1.0, np.abs(roots))])
    roots = roots[roots > 0]
    return np.sort(roots ** (1.0 / p_prime))


def fit_coefficients(A, B, ii, jj, p_log2, r, c, tau: float, estimator: int = 0):
    """The affine model's (a_q, b_q) from the exact values at the sample
    entries (ii, jj): scaled estimate and scaled exact value per sample, each
    sample in the class of its own p*."""
    pl = _plog(p_log2)
    exact, S = entries(A, B, ii, jj, pl, r, c)
    est, ps, _ = estimate(S.T[:, None, :], pl, np.ones(1), np.ones(len(ii)), tau, estimator)
    idx = {int(v): q for q, v in enumerate(pl)}
    cls = np.array([idx[int(b) & 0x7F] for b in ps[0]], dtype=np.int32)
    return affine_fit(est[0], exact / (r[ii] * c[jj]), cls, len(pl))


def apply_correction(Chat, psel, p_log2, K: int, r, c, correction: int, coef=None):
    """Correction 1 or 2 applied to Chat in place (see oracle.c)."""
    pl = _plog(p_log2)
    M, N = Chat.shape
    coef = np.zeros((len(pl), 2)) if coef is None else _f64(coef)
    psel = np.ascontiguousarray(psel, dtype=np.uint8)
    _load().orc_apply_correction(M, N, int(K), len(pl), _p(pl), int(correction), _p(coef),
                                 _p(psel), _p(_f64(r)), _p(_f64(c)), _p(Chat))
    return Chat


def entries(A, B, ii, jj, p_log2, r, c):
    """Exact max and all p-sums at the entries (ii[e], jj[e])."""
    A, B = _f64(A), _f64(B)
    M, K = A.shape
    _, N = B.shape
    ii = np.ascontiguousarray(ii, dtype=np.int64)
    jj = np.ascontiguousarray(jj, dtype=np.int64)
    pl = _plog(p_log2)
    r, c = _f64(r), _f64(c)
    ex = np.empty(len(ii), dtype=np.float64)
    S = np.empty((len(ii), len(pl)), dtype=np.float64)
    _load().orc_entries(M, N, K, _p(A), K, _p(B), N, _p(r), _p(c), len(pl), _p(pl), len(ii),
                        _p(ii), _p(jj), _p(ex), _p(S))
    return ex, S


def floyd_warshall(W):
    """Exact APSP distances; W uses +inf for missing edges."""
    D = np.array(W, dtype=np.float64, copy=True, order="C")
    n = D.shape[0]
    _load().orc_floyd_warshall(n, _p(D), n)
    return D


def apsp_pnorm(W, p_log2, tau: float, n_squarings: int = 0, scaling: int = 2,
               diag_policy: int = 2):
    W = _f64(W)
    n = W.shape[0]
    D = np.empty((n, n), dtype=np.float64)
    psel = np.empty((n, n), dtype=np.uint8)
    pl = _plog(p_log2)
    rc = _load().orc_apsp_pnorm(n, _p(W), n, int(n_squarings), len(pl), _p(pl), float(tau),
                                int(scaling), int(diag_policy), _p(D), n, _p(psel))
    if rc:
        raise MemoryError("oracle apsp allocation failed")
    return D, psel


def pnorm_grad(A, B, plog, G, scaling: int = 2):
    """dL/dA, dL/dB for L with dL/dC = G, p per entry = 2^plog (flag bits masked)."""
    A, B, G = _f64(A), _f64(B), _f64(G)
    M, K = A.shape
    _, N = B.shape
    r = row_scales(A, scaling)
    c = col_scales(B, scaling)
    pl = np.ascontiguousarray(np.asarray(plog) & 0x7F, dtype=np.uint8)
    dA = np.empty((M, K), dtype=np.float64)
    dB = np.empty((K, N), dtype=np.float64)
    _load().orc_pnorm_grad(M, N, K, _p(A), _p(B), _p(r), _p(c), _p(pl), _p(G), _p(dA), _p(dB))
    return dA, dB


def pnorm_grad_entries(A, B, plog, G, ia, ka, kb, jb, scaling: int = 2):
    """Sampled entries dA[ia, ka] and dB[kb, jb] of pnorm_grad (same definitions)."""
    A, B, G = _f64(A), _f64(B), _f64(G)
    M, K = A.shape
    _, N = B.shape
    r = row_scales(A, scaling)
    c = col_scales(B, scaling)
    pl = np.ascontiguousarray(np.asarray(plog) & 0x7F, dtype=np.uint8)
    ia, ka = np.ascontiguousarray(ia, np.int64), np.ascontiguousarray(ka, np.int64)
    kb, jb = np.ascontiguousarray(kb, np.int64), np.ascontiguousarray(jb, np.int64)
    dA = np.empty(len(ia), dtype=np.float64)
    dB = np.empty(len(kb), dtype=np.float64)
    _load().orc_pnorm_grad_entries(M, N, K, _p(A), _p(B), _p(r), _p(c), _p(pl), _p(G), len(ia),
                                   _p(ia), _p(ka), _p(dA), len(kb), _p(kb), _p(jb), _p(dB))
    return dA, dB


def row_logloss(arow, B, plog_row):
    arow, B = _f64(arow), _f64(B)
    K, N = B.shape
    pl = np.ascontiguousarray(np.asarray(plog_row) & 0x7F, dtype=np.uint8)
    return float(_load().orc_row_logloss(N, K, _p(arow), _p(B), _p(pl)))


def col_logloss(A, bcol, plog_col):
    A, bcol = _f64(A), _f64(bcol)
    M, K = A.shape
    pl = np.ascontiguousarray(np.asarray(plog_col) & 0x7F, dtype=np.uint8)
    return float(_load().orc_col_logloss(M, K, _p(A), _p(bcol), _p(pl)))


# ------------------------------------------------------- max-convolution ---
def _batch(x):
    x = _f64(x)
    return x[None, :] if x.ndim == 1 else x


def maxconv(x, y):
    """Exact max-convolution z_m = max_i x_i y_(m-i) (Sec. 1), per batch row."""
    x, y = _batch(x), _batch(y)
    b, nx = x.shape
    ny = y.shape[1]
    z = np.empty((b, nx + ny - 1), dtype=np.float64)
    _load().orc_maxconv(b, nx, _p(x), ny, _p(y), _p(z))
    return z


def conv(x, y):
    """Naive ring convolution w_m = sum_i x_i y_(m-i), per batch row."""
    x, y = _batch(x), _batch(y)
    b, nx = x.shape
    ny = y.shape[1]
    w = np.empty((b, nx + ny - 1), dtype=np.float64)
    _load().orc_conv(b, nx, _p(x), ny, _p(y), _p(w))
    return w


def maxconv_pnorm(x, y, p_log2, tau: float, want_S: bool = False):
    """p-norm estimate of the max-convolution from naive-convolution p-sums of
    the vectors scaled by their maxima (Sec. 1, Sec. 2.1).  Returns a dict with
    z, p_sel and (if want_S) S of shape (batch, n_p, nz)."""
    x, y = _batch(x), _batch(y)
    b, nx = x.shape
    ny = y.shape[1]
    nz = nx + ny - 1
    pl = _plog(p_log2)
    z = np.empty((b, nz), dtype=np.float64)
    psel = np.empty((b, nz), dtype=np.uint8)
    S = np.empty((b, len(pl), nz), dtype=np.float64) if want_S else None
    _load().orc_maxconv_pnorm(b, nx, _p(x), ny, _p(y), len(pl), _p(pl), float(tau), _p(z),
                              _p(psel), _p(S) if S is not None else None)
    out = dict(z=z, p_sel=psel)
    if want_S:
        out["S"] = S
    return out


def maxconv_entries(x, y, m, p_log2):
    """Exact max and every p-sum at the outputs m of one max-convolution."""
    x, y = _f64(x).ravel(), _f64(y).ravel()
    m = np.ascontiguousarray(m, dtype=np.int64)
    pl = _plog(p_log2)
    ex = np.empty(len(m), dtype=np.float64)
    S = np.empty((len(m), len(pl)), dtype=np.float64)
    _load().orc_maxconv_entries(len(x), _p(x), len(y), _p(y), len(pl), _p(pl), len(m), _p(m),
                                _p(ex), _p(S))
    return ex, S


def topk_xy(x, y, k, p_log2, tau: float = 1e-12, y_rev: bool = False):
    """Approximate top-k of x_i y_j (Alg. 9 with the NormQueue, plain
    estimator); returns (values, diagonals m = i + j, -1 when exhausted)."""
    x, y = _f64(x).ravel(), _f64(y).ravel()
    assert len(x) == len(y)
    pl = _plog(p_log2)
    vals = np.empty(k, dtype=np.float64)
    diag = np.empty(k, dtype=np.int64)
    _load().orc_topk_xy(len(x), _p(x), _p(y), int(bool(y_rev)), len(pl), _p(pl), float(tau),
                        int(k), _p(vals), _p(diag))
    return vals, diag


def recover_indices(d1, d2, n):
    """Index recovery of Alg. 9's discussion: the k-th result of the call on y
    lies on diagonal m1 = i + j, of the call on reversed y on m2 = i + (n-1-j);
    i = (m1 + m2 - n + 1) / 2, j = m1 - i.  Pairs whose parity or range is
    impossible give (-1, -1)."""
    d1, d2 = np.asarray(d1, dtype=np.int64), np.asarray(d2, dtype=np.int64)
    t = d1 + d2 - n + 1
    i = np.where((t % 2 == 0) & (d1 >= 0) & (d2 >= 0), t // 2, -1)
    j = np.where(i >= 0, d1 - i, -1)
    bad = (i < 0) | (i >= n) | (j < 0) | (j >= n)
    return np.where(bad, -1, i), np.where(bad, -1, j)
