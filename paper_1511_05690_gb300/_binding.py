"""ctypes binding of ``libpnorm.so`` (the C ABI in ``include/pnorm.h``).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Loading fails loudly if the library has not been built; there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpnorm.so")

PN_MAX_P = 16
PN_OK, PN_EINVAL, PN_EALIGN, PN_EWORKSPACE, PN_EDOMAIN, PN_ECUDA, PN_ETIMEOUT, PN_EUNSUPPORTED = range(8)
PN_F32_EXACT, PN_TF32, PN_BF16, PN_F16, PN_E4M3 = range(5)

COMPUTE_NAMES = {"f32": PN_F32_EXACT, "fp32": PN_F32_EXACT, "3xtf32": PN_F32_EXACT,
                 "tf32": PN_TF32, "bf16": PN_BF16, "f16": PN_F16, "fp16": PN_F16,
                 "e4m3": PN_E4M3, "fp8": PN_E4M3}

# Every symbol include/pnorm.h declares.
EXPORTS = (
    "pn_status_string", "pn_default_opts", "pn_default_tau", "pn_device_sm_count",
    "pn_workspace_size", "maxprod_pnorm", "maxprod_exact", "pn_maxprod_exact_variant",
    "pn_apsp_workspace_size", "apsp_pnorm", "pn_backward_workspace_size",
    "maxprod_pnorm_backward", "pn_grouped_table_bytes", "pn_grouped_build_table",
    "maxprod_pnorm_grouped", "maxprod_pnorm_static", "pn_autotune", "pn_grouped_autotune",
    "maxconv_pnorm", "maxconv_exact", "pn_maxconv_default_tau", "maxconv_pnorm_long",
    "pn_maxconv_long_workspace_size", "topk_xy", "pn_topk_xy_workspace_size",
)


class PnOpts(ctypes.Structure):
    _fields_ = [
        ("n_p", ctypes.c_int32),
        ("p_log2", ctypes.c_int32 * PN_MAX_P),
        ("tau", ctypes.c_double),
        ("compute", ctypes.c_int32),
        ("scaling", ctypes.c_int32),
        ("diag_policy", ctypes.c_int32),
        ("tile_n", ctypes.c_int32),
        ("dev_status", ctypes.c_void_p),
        ("ev_gemm_begin", ctypes.c_void_p),
        ("ev_gemm_end", ctypes.c_void_p),
        ("timeout_ns", ctypes.c_int64),
        ("debug_flags", ctypes.c_int32),
        ("estimator", ctypes.c_int32),
        ("correction", ctypes.c_int32),
        ("n_fit", ctypes.c_int32),
        ("fit_i", ctypes.c_void_p),
        ("fit_j", ctypes.c_void_p),
        ("fit_coef", ctypes.c_void_p),
        ("tile_m", ctypes.c_int32),
    ]


class PnError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = int(status)
        super().__init__(f"{where}: {status_string(status)}" if where else status_string(status))


_lib = None
_lock = threading.Lock()


def load():
    """Loads libpnorm.so; raises if it is missing (build it with build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"CUDA library not built: {LIB_PATH} is missing "
                "(run paper_1511_05690_gb300.build.build() or __graft_entry__.build())")
        lib = ctypes.CDLL(LIB_PATH)
        i64, i32, vp, sz, dbl = (ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                                 ctypes.c_size_t, ctypes.c_double)
        optp = ctypes.POINTER(PnOpts)
        lib.pn_status_string.argtypes = [i32]
        lib.pn_status_string.restype = ctypes.c_char_p
        lib.pn_default_opts.argtypes = [optp]
        lib.pn_default_opts.restype = None
        lib.pn_default_tau.argtypes = [i64, i32]
        lib.pn_default_tau.restype = dbl
        lib.pn_device_sm_count.argtypes = []
        lib.pn_device_sm_count.restype = i32
        lib.pn_workspace_size.argtypes = [i64, i64, i64, optp]
        lib.pn_workspace_size.restype = sz
        lib.maxprod_pnorm.argtypes = [i64, i64, i64, vp, i64, vp, i64, vp, i64, vp, vp, optp,
                                      vp, sz, vp]
        lib.maxprod_pnorm.restype = i32
        lib.maxprod_pnorm_static.argtypes = [i64, i64, i64, vp, i64, vp, i64, vp, i64, vp, vp,
                                             optp, vp]
        lib.maxprod_pnorm_static.restype = i32
        lib.maxprod_exact.argtypes = [i64, i64, i64, vp, i64, vp, i64, vp, i64, i32, vp]
        lib.maxprod_exact.restype = i32
        lib.pn_maxprod_exact_variant.argtypes = [i64, i64, i64, vp, i64, vp, i64, vp, i64, i32,
                                                 i32, vp]
        lib.pn_maxprod_exact_variant.restype = i32
        lib.maxconv_pnorm.argtypes = [i64, i64, vp, i64, i64, vp, i64, vp, i64, vp, i64, optp, vp]
        lib.maxconv_pnorm.restype = i32
        lib.maxconv_exact.argtypes = [i64, i64, vp, i64, i64, vp, i64, vp, i64, vp]
        lib.maxconv_exact.restype = i32
        lib.maxconv_pnorm_long.argtypes = [i64, vp, i64, vp, vp, vp, optp, vp, ctypes.c_size_t, vp]
        lib.maxconv_pnorm_long.restype = i32
        lib.pn_maxconv_long_workspace_size.argtypes = [i64, i64, i32]
        lib.pn_maxconv_long_workspace_size.restype = ctypes.c_size_t
        lib.topk_xy.argtypes = [i64, i64, vp, i64, vp, i64, i64, vp, vp, vp, i64, optp, vp,
                                ctypes.c_size_t, vp]
        lib.topk_xy.restype = i32
        lib.pn_topk_xy_workspace_size.argtypes = [i64, i64, i64, optp]
        lib.pn_topk_xy_workspace_size.restype = ctypes.c_size_t
        lib.pn_maxconv_default_tau.argtypes = []
        lib.pn_maxconv_default_tau.restype = ctypes.c_double
        lib.pn_apsp_workspace_size.argtypes = [i64, optp]
        lib.pn_apsp_workspace_size.restype = sz
        lib.apsp_pnorm.argtypes = [i64, vp, i64, vp, i64, i32, optp, vp, sz, vp]
        lib.apsp_pnorm.restype = i32
        lib.pn_backward_workspace_size.argtypes = [i64, i64, i64, optp]
        lib.pn_backward_workspace_size.restype = sz
        lib.maxprod_pnorm_backward.argtypes = [i64, i64, i64, vp, vp, vp, vp, vp, vp, vp, vp,
                                               optp, vp, sz, vp]
        lib.maxprod_pnorm_backward.restype = i32
        lib.pn_grouped_table_bytes.argtypes = [i32, vp, optp]
        lib.pn_grouped_table_bytes.restype = sz
        lib.pn_grouped_build_table.argtypes = [i32, vp, vp, vp, vp, optp, vp, sz,
                                               ctypes.POINTER(sz)]
        lib.pn_grouped_build_table.restype = i32
        lib.maxprod_pnorm_grouped.argtypes = [vp, vp, optp, vp, sz, vp]
        lib.maxprod_pnorm_grouped.restype = i32
        lib.pn_autotune.argtypes = [i64, i64, i64, vp, i64, vp, i64, vp, i64, optp, vp, sz, vp,
                                    ctypes.POINTER(i32)]
        lib.pn_autotune.restype = i32
        lib.pn_grouped_autotune.argtypes = [vp, vp, optp, vp, sz, vp, ctypes.POINTER(i32)]
        lib.pn_grouped_autotune.restype = i32
        _lib = lib
        return lib


def status_string(status: int) -> str:
    return load().pn_status_string(int(status)).decode()


def check(status: int, where: str = "") -> None:
    if int(status) != PN_OK:
        raise PnError(status, where)


def make_opts(p_log2=tuple(range(7)), compute="bf16", tau=None, scaling=2, diag_policy=2,
              tile_n=0, dev_status=None, ev_begin=None, ev_end=None, timeout_ns=0,
              debug_flags=0, estimator=0, correction=0, n_fit=0, fit_i=None, fit_j=None,
              fit_coef=None, tile_m=0) -> PnOpts:
    o = PnOpts()
    load().pn_default_opts(ctypes.byref(o))
    pl = [int(x) for x in p_log2]
    if not 1 <= len(pl) <= PN_MAX_P:
        raise ValueError("p family must have 1..16 entries")
    o.n_p = len(pl)
    for q, v in enumerate(pl):
        o.p_log2[q] = v
    o.tau = 0.0 if tau is None else float(tau)
    o.compute = COMPUTE_NAMES[compute] if isinstance(compute, str) else int(compute)
    o.scaling = int(scaling)
    o.diag_policy = int(diag_policy)
    o.tile_n = int(tile_n)
    o.dev_status = dev_status
    o.ev_gemm_begin = ev_begin
    o.ev_gemm_end = ev_end
    o.timeout_ns = int(timeout_ns)
    o.debug_flags = int(debug_flags)
    o.estimator = int(estimator)
    o.correction = int(correction)
    o.n_fit = int(n_fit)
    o.fit_i = fit_i
    o.fit_j = fit_j
    o.fit_coef = fit_coef
    o.tile_m = int(tile_m)
    return o
