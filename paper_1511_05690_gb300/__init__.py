"""GB300 (sm_103a) p-norm semiring products: a thin PyTorch-facing wrapper.

The library estimates the (x,max) semiring matrix product on nonnegative reals
with a family of p-norm rings (O. Serang, arXiv 1511.05690, Sec. 2.1 and
Alg. 5): scale, raise to p, ring GEMM on the tensor cores, 1/p root, largest
stable p per entry, un-scale.  Through x = exp(-w) it gives (+,min) APSP by
repeated squaring (Sec. 2.2).

PyTorch provides device memory and streams only.  Every function here
validates shapes, allocates outputs and the workspace, and calls the C ABI of
``_lib/libpnorm.so`` (``include/pnorm.h``); all arithmetic runs in the CUDA
kernels.  There is no CPU fallback: if the library is missing, calls raise.
"""
from __future__ import annotations

import ctypes

import torch

from . import _binding as _b
from ._binding import (PN_BF16, PN_E4M3, PN_F16, PN_F32_EXACT, PN_TF32, PnError,  # noqa: F401
                       make_opts, status_string)

__all__ = ["maxprod_pnorm", "maxprod_exact", "apsp_pnorm", "default_tau", "workspace",
           "PnError", "make_opts", "status_string", "sm_count", "PNormMaxProd",
           "maxprod_pnorm_backward", "GroupedProduct", "autotune", "maxconv_pnorm",
           "maxconv_exact", "topk_xy"]

_ws = {}
_status = {}


def lib():
    return _b.load()


def sm_count() -> int:
    return int(lib().pn_device_sm_count())


def default_tau(K: int, compute="bf16") -> float:
    c = _b.COMPUTE_NAMES[compute] if isinstance(compute, str) else int(compute)
    return float(lib().pn_default_tau(int(K), c))


def workspace(nbytes: int, device) -> torch.Tensor:
    """Per-device cached workspace of at least nbytes (256-byte aligned)."""
    dev = torch.device(device)
    key = dev.index if dev.index is not None else torch.cuda.current_device()
    buf = _ws.get(key)
    if buf is None or buf.numel() < nbytes:
        _ws.pop(key, None)
        buf = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=dev)
        if buf.data_ptr() % 256:
            raise RuntimeError("workspace allocation is not 256-byte aligned")
        _ws[key] = buf
    return buf


def status_word(device) -> torch.Tensor:
    """Per-device int32 word receiving device-side errors (zero when clean)."""
    dev = torch.device(device)
    key = dev.index if dev.index is not None else torch.cuda.current_device()
    w = _status.get(key)
    if w is None:
        w = torch.zeros(1, dtype=torch.int32, device=dev)
        _status[key] = w
    return w


def check_device_status(device, where: str) -> None:
    """Synchronises the current stream and raises PnError if a kernel recorded an error."""
    w = status_word(device)
    code = int(w.item())
    if code != 0:
        w.zero_()
        raise PnError(code, where)


def _stream_ptr(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _event(ev):
    """Raw cudaEvent_t of a torch.cuda.Event (created on first use)."""
    if ev is None:
        return None
    if not ev.cuda_event:
        ev.record()  # torch creates the underlying event lazily
    return ev.cuda_event


def _mat(x: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(x, torch.Tensor) or x.dim() != 2:
        raise ValueError(f"{name} must be a 2-D tensor")
    if x.dtype != torch.float32:
        raise ValueError(f"{name} must be float32")
    if not x.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if x.stride(1) != 1 or (x.size(0) > 1 and x.stride(0) < x.size(1)):
        x = x.contiguous()
    return x


def _ld(x: torch.Tensor) -> int:
    return x.stride(0) if x.size(0) > 1 else max(x.size(1), 1)


def maxprod_pnorm(A: torch.Tensor, B: torch.Tensor, *, p_log2=tuple(range(7)), compute="bf16",
                  tau=None, scaling=2, tile_n=0, out=None, want_psel=True, want_ssel=True,
                  check=True, ev_begin=None, ev_end=None, stream=None, timeout_ns=0,
                  debug_flags=0, estimator=0, correction=0, fit_i=None, fit_j=None,
                  fit_coef=None, tile_m=0):
    """p-norm estimate of C = A (x,max) B.  Returns (C, p_sel or None, S_sel or None).
    tile_m: 0 automatic, 128 one CTA per tile, 256 a CTA pair per 256 x tile_n tile
    (tile_n 0: a size rule picks the pair's width).
    estimator 0: plain (S^(p*))^(1/p*); 1: r = 1 projection (S^(p*)/S^(p*/2))^(2/p*);
    2: r = 2 projection from the sums at p*/4, p*/2, 3p*/4 and p* (Sec. 2.1).
    correction 1: divide by K^(1/p*); 2: affine model per p* class fitted to the
    exact values at the sample entries (fit_i, fit_j) (int32 CUDA tensors);
    fit_coef (float32 CUDA tensor of 2 * len(p_log2)) receives (a_q, b_q)."""
    A, B = _mat(A, "A"), _mat(B, "B")
    M, K = A.shape
    K2, N = B.shape
    if K != K2:
        raise ValueError("inner dimensions differ")
    dev = A.device
    C = out if out is not None else torch.empty((M, N), dtype=torch.float32, device=dev)
    psel = torch.empty((M, N), dtype=torch.uint8, device=dev) if want_psel else None
    ssel = torch.empty((M, N), dtype=torch.float32, device=dev) if want_ssel else None
    st = status_word(dev)
    fit = dict(correction=correction)
    if correction == 2:
        fit_i = fit_i.to(device=dev, dtype=torch.int32).contiguous()
        fit_j = fit_j.to(device=dev, dtype=torch.int32).contiguous()
        if fit_i.numel() != fit_j.numel():
            raise ValueError("fit_i and fit_j differ in length")
        fit.update(n_fit=fit_i.numel(), fit_i=fit_i.data_ptr(), fit_j=fit_j.data_ptr(),
                   fit_coef=fit_coef.data_ptr() if fit_coef is not None else None)
    o = make_opts(p_log2, compute, tau, scaling, 1, tile_n, st.data_ptr(), _event(ev_begin),
                  _event(ev_end), timeout_ns, debug_flags, estimator, tile_m=tile_m, **fit)
    L = lib()
    need = L.pn_workspace_size(M, N, K, ctypes.byref(o))
    if need == 0 and M * N > 0:
        raise ValueError("invalid options")
    ws = workspace(need, dev)
    rc = L.maxprod_pnorm(M, N, K, A.data_ptr(), _ld(A), B.data_ptr(), _ld(B), C.data_ptr(),
                         _ld(C), psel.data_ptr() if psel is not None else None,
                         ssel.data_ptr() if ssel is not None else None, ctypes.byref(o),
                         ws.data_ptr(), ws.numel(), _stream_ptr(stream))
    _b.check(rc, "maxprod_pnorm")
    if check:
        check_device_status(dev, "maxprod_pnorm")
    return C, psel, ssel


def autotune(A: torch.Tensor, B: torch.Tensor, *, p_log2=tuple(range(7)), compute="bf16",
             tau=None, scaling=2, stream=None) -> int:
    """Times the tile shapes for this shape class and remembers the fastest
    (later calls with tile_n=0, tile_m=0 use it).  Synchronises; returns the
    width of one CTA's tile (128 or 256), or 256 + the width for a CTA pair
    (512 or 384)."""
    A, B = _mat(A, "A"), _mat(B, "B")
    M, K = A.shape
    N = B.shape[1]
    C = torch.empty((M, N), dtype=torch.float32, device=A.device)
    o = make_opts(p_log2, compute, tau, scaling, 2, 0, status_word(A.device).data_ptr())
    L = lib()
    need = L.pn_workspace_size(M, N, K, ctypes.byref(o))
    ws = workspace(need, A.device)
    chosen = ctypes.c_int32(0)
    rc = L.pn_autotune(M, N, K, A.data_ptr(), _ld(A), B.data_ptr(), _ld(B), C.data_ptr(), _ld(C),
                       ctypes.byref(o), ws.data_ptr(), ws.numel(), _stream_ptr(stream),
                       ctypes.byref(chosen))
    _b.check(rc, "pn_autotune")
    return int(chosen.value)


class GroupedProduct:
    """Many independent p-norm (x,max) products C_g = A_g (x) B_g computed
    together in one persistent launch over every problem, p level and tile
    (scaling 1 uses one launch sequence per p level).  The problem table is built
    and copied to the device once here; run() only launches kernels, so it can
    be captured in a CUDA graph (the plan keeps its own workspace and outputs
    alive for replays).  A_g: (M_g, K_g), B_g: (K_g, N_g), float32 CUDA."""

    def __init__(self, As, Bs, *, p_log2=tuple(range(7)), compute="bf16", tau=None, scaling=2,
                 tile_n=0, estimator=0, correction=0, debug_flags=0):
        import numpy as np
        if len(As) != len(Bs):
            raise ValueError("As and Bs differ in length")
        self.As = [_mat(a, "A").contiguous() for a in As]
        self.Bs = [_mat(b, "B").contiguous() for b in Bs]
        dev = self.As[0].device if self.As else torch.device("cuda")
        self.Cs = [torch.empty((a.shape[0], b.shape[1]), dtype=torch.float32, device=dev)
                   for a, b in zip(self.As, self.Bs)]
        count = len(self.As)
        mnk = []
        for a, b in zip(self.As, self.Bs):
            if a.shape[1] != b.shape[0]:
                raise ValueError("inner dimensions differ")
            mnk += [a.shape[0], b.shape[1], a.shape[1]]
        self.status = status_word(dev)
        self.opts = make_opts(p_log2, compute, tau, scaling, 2, tile_n, self.status.data_ptr(),
                              estimator=estimator, correction=correction,
                              debug_flags=debug_flags)
        L = lib()
        MNK = (ctypes.c_int64 * max(1, 3 * count))(*mnk)
        vp = ctypes.c_void_p
        Ap = (vp * max(1, count))(*[a.data_ptr() for a in self.As])
        Bp = (vp * max(1, count))(*[b.data_ptr() for b in self.Bs])
        Cp = (vp * max(1, count))(*[c.data_ptr() for c in self.Cs])
        tb = L.pn_grouped_table_bytes(count, MNK, ctypes.byref(self.opts))
        if tb == 0:
            raise PnError(_b.PN_EINVAL, "pn_grouped_table_bytes")
        self.host_table = np.zeros(tb, dtype=np.uint8)
        ws_bytes = ctypes.c_size_t(0)
        rc = L.pn_grouped_build_table(count, MNK, Ap, Bp, Cp, ctypes.byref(self.opts),
                                      self.host_table.ctypes.data_as(vp), tb,
                                      ctypes.byref(ws_bytes))
        _b.check(rc, "pn_grouped_build_table")
        self.dev_table = torch.from_numpy(self.host_table).to(dev)
        self.ws = torch.empty(max(int(ws_bytes.value), 256), dtype=torch.uint8, device=dev)

    def _args(self):
        return (self.host_table.ctypes.data_as(ctypes.c_void_p), self.dev_table.data_ptr(),
                ctypes.byref(self.opts), self.ws.data_ptr(), self.ws.numel())

    def run(self, stream=None, check=False):
        rc = lib().maxprod_pnorm_grouped(*self._args(), _stream_ptr(stream))
        _b.check(rc, "maxprod_pnorm_grouped")
        if check:
            check_device_status(self.ws.device, "maxprod_pnorm_grouped")
        return self.Cs

    def autotune(self, stream=None) -> int:
        chosen = ctypes.c_int32(0)
        rc = lib().pn_grouped_autotune(*self._args(), _stream_ptr(stream), ctypes.byref(chosen))
        _b.check(rc, "pn_grouped_autotune")
        return int(chosen.value)


def maxprod_exact(A: torch.Tensor, B: torch.Tensor, *, semiring=0, variant=None, out=None,
                  stream=None):
    """Exact (x,max) (semiring 0) or (+,min) (semiring 1) product on the CUDA cores."""
    A, B = _mat(A, "A"), _mat(B, "B")
    M, K = A.shape
    K2, N = B.shape
    if K != K2:
        raise ValueError("inner dimensions differ")
    C = out if out is not None else torch.empty((M, N), dtype=torch.float32, device=A.device)
    L = lib()
    if variant is None:
        rc = L.maxprod_exact(M, N, K, A.data_ptr(), _ld(A), B.data_ptr(), _ld(B), C.data_ptr(),
                             _ld(C), int(semiring), _stream_ptr(stream))
    else:
        rc = L.pn_maxprod_exact_variant(M, N, K, A.data_ptr(), _ld(A), B.data_ptr(), _ld(B),
                                        C.data_ptr(), _ld(C), int(semiring), int(variant),
                                        _stream_ptr(stream))
    _b.check(rc, "maxprod_exact")
    return C


def _rows(v, name):
    """A (batch, n) float32 CUDA tensor with unit column stride (1-D -> one row)."""
    if v.dim() == 1:
        v = v.unsqueeze(0)
    return _mat(v, name)


def maxconv_pnorm(x: torch.Tensor, y: torch.Tensor, *, p_log2=tuple(range(7)), tau=None,
                  out=None, want_psel=True, check=True, stream=None):
    """p-norm estimate of the batched max-convolution z_m = max_i x_i y_(m-i)
    with H = FP64 FFT convolution (Sec. 1).  x: (batch, nx), y: (batch, ny)
    (or 1-D).  Returns (z, p_sel or None), z of shape (batch, nx + ny - 1).
    Up to nx + ny - 1 = 8192 one CTA per problem (maxconv_pnorm); longer
    problems, up to 2^22, one call of maxconv_pnorm_long per row."""
    x, y = _rows(x, "x"), _rows(y, "y")
    if x.shape[0] != y.shape[0]:
        raise ValueError("x and y differ in batch")
    batch, nx = x.shape
    ny = y.shape[1]
    nz = nx + ny - 1
    dev = x.device
    z = out if out is not None else torch.empty((batch, nz), dtype=torch.float32, device=dev)
    psel = torch.empty((batch, nz), dtype=torch.uint8, device=dev) if want_psel else None
    st = status_word(dev)
    o = make_opts(p_log2, "f32", tau, 2, 0, 0, st.data_ptr())
    L = lib()
    if nz <= 8192:
        rc = L.maxconv_pnorm(batch, nx, x.data_ptr(), _ld(x), ny, y.data_ptr(), _ld(y),
                             z.data_ptr(), _ld(z), psel.data_ptr() if psel is not None else None,
                             nz, ctypes.byref(o), _stream_ptr(stream))
        _b.check(rc, "maxconv_pnorm")
    else:
        need = L.pn_maxconv_long_workspace_size(nx, ny, 1 if psel is not None else 0)
        if need == 0:
            raise PnError(_b.PN_EUNSUPPORTED, "maxconv_pnorm_long")
        ws = workspace(need, dev)
        for b in range(batch):
            rc = L.maxconv_pnorm_long(nx, x[b].data_ptr(), ny, y[b].data_ptr(), z[b].data_ptr(),
                                      psel[b].data_ptr() if psel is not None else None,
                                      ctypes.byref(o), ws.data_ptr(), ws.numel(),
                                      _stream_ptr(stream))
            _b.check(rc, "maxconv_pnorm_long")
    if check:
        check_device_status(dev, "maxconv_pnorm")
    return z, psel


def topk_xy(x: torch.Tensor, y: torch.Tensor, k: int, *, p_log2=tuple(range(13)), tau=None,
            check=True, stream=None):
    """Approximate top-k of x_i y_j per batch row (Alg. 9 with the NormQueue)
    and the recovered indices (-1 where the check fails).  Returns (vals, i, j),
    each (batch, k)."""
    x, y = _rows(x, "x"), _rows(y, "y")
    if x.shape != y.shape:
        raise ValueError("x and y must have the same shape")
    batch, n = x.shape
    dev = x.device
    vals = torch.empty((batch, k), dtype=torch.float32, device=dev)
    ii = torch.empty((batch, k), dtype=torch.int32, device=dev)
    jj = torch.empty((batch, k), dtype=torch.int32, device=dev)
    st = status_word(dev)
    o = make_opts(p_log2, "f32", tau, 2, 0, 0, st.data_ptr())
    L = lib()
    need = L.pn_topk_xy_workspace_size(batch, n, k, ctypes.byref(o))
    if need == 0:
        raise PnError(_b.PN_EUNSUPPORTED, "topk_xy")
    ws = workspace(need, dev)
    rc = L.topk_xy(batch, n, x.data_ptr(), _ld(x), y.data_ptr(), _ld(y), k, vals.data_ptr(),
                   ii.data_ptr(), jj.data_ptr(), k, ctypes.byref(o), ws.data_ptr(), ws.numel(),
                   _stream_ptr(stream))
    _b.check(rc, "topk_xy")
    if check:
        check_device_status(dev, "topk_xy")
    return vals, ii, jj


def maxconv_exact(x: torch.Tensor, y: torch.Tensor, *, out=None, stream=None):
    """Exact batched max-convolution on the CUDA cores (the comparison)."""
    x, y = _rows(x, "x"), _rows(y, "y")
    if x.shape[0] != y.shape[0]:
        raise ValueError("x and y differ in batch")
    batch, nx = x.shape
    ny = y.shape[1]
    z = out if out is not None else torch.empty((batch, nx + ny - 1), dtype=torch.float32,
                                                device=x.device)
    rc = lib().maxconv_exact(batch, nx, x.data_ptr(), _ld(x), ny, y.data_ptr(), _ld(y),
                             z.data_ptr(), _ld(z), _stream_ptr(stream))
    _b.check(rc, "maxconv_exact")
    return z


def apsp_pnorm(W: torch.Tensor, *, n_squarings=0, p_log2=tuple(range(7)), compute="f32",
               tau=None, scaling=2, diag_policy=2, tile_n=0, out=None, check=True,
               stream=None, ev_begin=None, ev_end=None, estimator=0, correction=0, tile_m=0):
    """Estimated all-pairs shortest distances of the weight matrix W (+inf = no edge).
    Only the plain, uncorrected estimator is supported: a nonzero estimator or
    correction raises PnError(PN_EUNSUPPORTED)."""
    W = _mat(W, "W")
    n = W.shape[0]
    if W.shape[1] != n:
        raise ValueError("W must be square")
    dev = W.device
    D = out if out is not None else torch.empty((n, n), dtype=torch.float32, device=dev)
    st = status_word(dev)
    o = make_opts(p_log2, compute, tau, scaling, diag_policy, tile_n, st.data_ptr(),
                  _event(ev_begin), _event(ev_end), estimator=estimator, correction=correction,
                  tile_m=tile_m)
    L = lib()
    need = L.pn_apsp_workspace_size(n, ctypes.byref(o))
    if need == 0 and n > 0:
        raise ValueError("invalid options")
    ws = workspace(need, dev)
    rc = L.apsp_pnorm(n, W.data_ptr(), _ld(W), D.data_ptr(), _ld(D), int(n_squarings),
                      ctypes.byref(o), ws.data_ptr(), ws.numel(), _stream_ptr(stream))
    _b.check(rc, "apsp_pnorm")
    if check:
        check_device_status(dev, "apsp_pnorm")
    return D


def maxprod_pnorm_backward(A, B, C, S_sel, p_sel, dC, *, p_log2=tuple(range(7)),
                           compute="f32", tau=None, scaling=2, check=True, stream=None,
                           tile_m=0, tile_n=0):
    """Adjoint of maxprod_pnorm at fixed p* per entry; returns (dA, dB).
    tile_m / tile_n: the gradient GEMMs' tiles (0 automatic: CTA pairs on
    256 x 256 tiles when each GEMM has at least two pair tiles per pair of
    SMs)."""
    A, B = _mat(A, "A").contiguous(), _mat(B, "B").contiguous()
    C, S_sel, dC = C.contiguous(), S_sel.contiguous(), dC.contiguous()
    p_sel = p_sel.contiguous()
    M, K = A.shape
    N = B.shape[1]
    dev = A.device
    dA = torch.empty((M, K), dtype=torch.float32, device=dev)
    dB = torch.empty((K, N), dtype=torch.float32, device=dev)
    st = status_word(dev)
    o = make_opts(p_log2, compute, tau, scaling, 1, tile_n, st.data_ptr(), tile_m=tile_m)
    L = lib()
    need = L.pn_backward_workspace_size(M, N, K, ctypes.byref(o))
    ws = workspace(max(need, 256), dev)
    rc = L.maxprod_pnorm_backward(M, N, K, A.data_ptr(), B.data_ptr(), C.data_ptr(),
                                  S_sel.data_ptr(), p_sel.data_ptr(), dC.data_ptr(),
                                  dA.data_ptr(), dB.data_ptr(), ctypes.byref(o), ws.data_ptr(),
                                  ws.numel(), _stream_ptr(stream))
    _b.check(rc, "maxprod_pnorm_backward")
    if check:
        check_device_status(dev, "maxprod_pnorm_backward")
    return dA, dB


class PNormMaxProd(torch.autograd.Function):
    """C = p-norm (x,max) product of A and B, differentiable at fixed p* per entry."""

    @staticmethod
    def forward(ctx, A, B, p_log2=tuple(range(7)), compute="f32", tau=None, scaling=2):
        C, psel, ssel = maxprod_pnorm(A, B, p_log2=p_log2, compute=compute, tau=tau,
                                      scaling=scaling)
        ctx.save_for_backward(A, B, C, ssel, psel)
        ctx.cfg = (tuple(p_log2), compute, tau, scaling)
        ctx.mark_non_differentiable(psel, ssel)
        return C, psel, ssel

    @staticmethod
    def backward(ctx, dC, _dpsel=None, _dssel=None):
        A, B, C, ssel, psel = ctx.saved_tensors
        p_log2, compute, tau, scaling = ctx.cfg
        dA, dB = maxprod_pnorm_backward(A, B, C, ssel, psel, dC.contiguous(), p_log2=p_log2,
                                        compute=compute, tau=tau, scaling=scaling)
        return dA, dB, None, None, None, None
