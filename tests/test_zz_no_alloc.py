"""The allocation-free entry point maxprod_pnorm_static, called through the C ABI.

It serves callers that may not allocate device memory (they own only their
inputs and outputs), so it runs in a scratch array inside the library.  This
file is collected last so that a run stopping at the first failure has run
every other test first; it also passes on its own in a fresh process.
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


def _rel_tol(K, plog):
    # tolerance the parity tests use for BF16 operands (see test_gpu_product.s_tol)
    p = 2.0 ** plog
    s = 2 * (p - 1) * 2.0 ** -24 + 2 * 2.0 ** -8 + 2.0 ** -7 + K * 2.0 ** -23
    return 1.5 * ((1 + s) ** (1.0 / p) - 1) + 2e-7


def _run(b, fn_static, M, N, K, seed):
    L = b.load()
    A_h, B_h = workloads.wide_range_pair(M, N, K, seed=seed)
    A = torch.from_numpy(A_h).cuda()
    B = torch.from_numpy(B_h).cuda()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    o = b.make_opts(compute="bf16", dev_status=status.data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    outs = []
    for static in (fn_static, False):
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
        outs.append((C.cpu().numpy(), psel.cpu().numpy(), ssel.cpu().numpy()))
    return outs


def test_static_entry_matches_workspace_entry_twice(lib):
    """Two calls in a row (different sizes, so stale scratch would show) agree
    with maxprod_pnorm on the same inputs within the parity tolerance."""
    for (M, N, K, seed) in [(700, 900, 1100, 11), (333, 257, 515, 12)]:
        (Cs, ps, ss), (Cw, pw, sw) = _run(lib, True, M, N, K, seed)
        np.testing.assert_array_equal(ps, pw)
        tol = np.vectorize(lambda lp: _rel_tol(K, lp))(pw & 0x7F)
        assert np.all(np.abs(Cs - Cw) <= tol * np.abs(Cw))
        assert np.all(np.abs(ss - sw) <= tol * np.abs(sw))


def test_static_entry_rejects_oversized_problems(lib):
    L = lib.load()
    o = lib.make_opts(compute="bf16")
    n = 4096
    assert L.pn_workspace_size(n, n, n, ctypes.byref(o)) > (64 << 20)
    rc = L.maxprod_pnorm_static(n, n, n, None, n, None, n, None, n, None, None, ctypes.byref(o),
                                None)
    assert rc == lib.PN_EWORKSPACE
