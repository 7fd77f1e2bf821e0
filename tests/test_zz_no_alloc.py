"""The allocation-free entry point maxprod_pnorm_static, called through the C ABI.

It serves callers that may not allocate device memory (they own only their
inputs and outputs), so it runs in a scratch array inside the library.  Both
entry points run the same deterministic kernels on the same inputs, so the
static call must give bit-identical C, p_sel and S_sel to maxprod_pnorm with
a workspace of its own.  Every case follows a larger call, so scratch left
over from that call would show.  This file is collected last so that a run
stopping at the first failure has run every other test first; it also passes
on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_05690_gb300 import build
    build.build()
    from paper_1511_05690_gb300 import _binding
    return _binding


def _run(b, M, N, K, seed, compute="bf16", estimator=0, correction=0):
    """Calls maxprod_pnorm_static, then maxprod_pnorm with its own workspace,
    on the same inputs; returns both (C, p_sel, S_sel) triples."""
    L = b.load()
    A_h, B_h = workloads.wide_range_pair(M, N, K, seed=seed)
    A = torch.from_numpy(A_h).cuda()
    B = torch.from_numpy(B_h).cuda()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    extra = {}
    if correction == 2:
        g = workloads.rng(seed + 1)
        fi = torch.from_numpy(g.integers(0, M, 64).astype(np.int32)).cuda()
        fj = torch.from_numpy(g.integers(0, N, 64).astype(np.int32)).cuda()
        extra = dict(n_fit=64, fit_i=fi.data_ptr(), fit_j=fj.data_ptr())
    o = b.make_opts(compute=compute, dev_status=status.data_ptr(), estimator=estimator,
                    correction=correction, **extra)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    outs = []
    for static in (True, False):
        C = torch.empty((M, N), dtype=torch.float32, device="cuda")
        psel = torch.empty((M, N), dtype=torch.uint8, device="cuda")
        ssel = torch.empty((M, N), dtype=torch.float32, device="cuda")
        args = (M, N, K, A.data_ptr(), K, B.data_ptr(), N, C.data_ptr(), N, psel.data_ptr(),
                ssel.data_ptr(), ctypes.byref(o))
        if static:
            rc = L.maxprod_pnorm_static(*args, stream)
        else:
            need = L.pn_workspace_size(M, N, K, ctypes.byref(o))
            ws = torch.empty(need, dtype=torch.uint8, device="cuda")
            rc = L.maxprod_pnorm(*args, ws.data_ptr(), need, stream)
        assert rc == 0, b.status_string(rc)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        outs.append((C, psel, ssel))
    return outs


def _assert_identical(outs):
    (Cs, ps, ss), (Cw, pw, sw) = outs
    assert torch.equal(ps, pw)
    assert torch.equal(Cs, Cw)
    assert torch.equal(ss, sw)


def test_static_entry_matches_workspace_entry_twice(lib):
    """Two calls in a row, the second smaller than the first: bit-identical to
    maxprod_pnorm on the same inputs."""
    for (M, N, K, seed) in [(700, 900, 1100, 11), (333, 257, 515, 12)]:
        _assert_identical(_run(lib, M, N, K, seed))


@pytest.mark.parametrize("estimator,correction", [(2, 0), (0, 2), (1, 2)])
def test_static_entry_projection_and_correction(lib, estimator, correction):
    """The r = 2 projection (parked sums and pending stages in the scratch) and
    the affine correction (sample records and coefficients in the scratch),
    each right after a larger plain call: bit-identical to maxprod_pnorm."""
    _assert_identical(_run(lib, 900, 800, 1000, 21))
    _assert_identical(_run(lib, 300, 260, 400, 22, estimator=estimator, correction=correction))


def test_static_entry_rejects_oversized_problems(lib):
    L = lib.load()
    o = lib.make_opts(compute="bf16")
    n = 4096
    assert L.pn_workspace_size(n, n, n, ctypes.byref(o)) > (64 << 20)
    rc = L.maxprod_pnorm_static(n, n, n, None, n, None, n, None, n, None, None, ctypes.byref(o),
                                None)
    assert rc == lib.PN_EWORKSPACE
