"""Failure detection without a GPU fault: a bounded device-side wait runs out.

The host sets a test flag that makes the copy producer of the tensor-core
kernel skip one stage, so the MMA issuer's wait for it can never complete.
The wait gives up after `timeout_ns`, the kernel records PN_ETIMEOUT in the
status word, lets its copies land, frees TMEM and returns; the host reads the
status and the context stays usable for the next call.  Nothing traps, asserts
or hangs.
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


def test_bounded_wait_reports_timeout_and_context_survives(pn):
    A, B = workloads.uniform_pair(512, 512, 512, seed=31)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    with pytest.raises(pn.PnError) as ei:
        pn.maxprod_pnorm(dA, dB, compute="bf16", timeout_ns=200_000_000, debug_flags=1)
    assert ei.value.status == 6  # PN_ETIMEOUT
    # the next call on the same context works and matches a clean run
    C1, _, _ = pn.maxprod_pnorm(dA, dB, compute="bf16")
    C2, _, _ = pn.maxprod_pnorm(dA, dB, compute="bf16")
    assert torch.equal(C1, C2)
    assert torch.isfinite(C1).all()


def test_image_kernel_wait_reports_timeout_and_context_survives(pn):
    """The tensor-copy image kernel (16-byte aligned rows) waits, bounded, for a
    tile whose bytes are announced but never copied: PN_ETIMEOUT, the copies in
    flight land, and the next call works."""
    A, B = workloads.uniform_pair(512, 512, 512, seed=32)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    with pytest.raises(pn.PnError) as ei:
        pn.maxprod_pnorm(dA, dB, compute="bf16", timeout_ns=200_000_000, debug_flags=2)
    assert ei.value.status == 6  # PN_ETIMEOUT
    C1, _, _ = pn.maxprod_pnorm(dA, dB, compute="bf16")
    C2, _, _ = pn.maxprod_pnorm(dA, dB, compute="bf16")
    assert torch.equal(C1, C2)
    assert torch.isfinite(C1).all()
