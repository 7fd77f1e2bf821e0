"""The host-buffer pipeline (copy-in / compute / copy-out overlapped across
independent products) gives exactly the products of direct calls."""
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


@pytest.mark.parametrize("mode", ["bf16", "f32"])
def test_host_pipeline_matches_direct_calls(pn, mode):
    from paper_1511_05690_gb300.pipeline import HostPipeline
    M, N, K = 700, 520, 900
    items, ref = [], []
    for i in range(5):
        A, B = workloads.wide_range_pair(M, N, K, seed=1000 + i)
        Ah = torch.from_numpy(A).pin_memory()
        Bh = torch.from_numpy(B).pin_memory()
        Ch = torch.full((M, N), -1.0).pin_memory()
        items.append((Ah, Bh, Ch))
        C, _, _ = pn.maxprod_pnorm(Ah.cuda(), Bh.cuda(), compute=mode)
        ref.append(C.cpu())
    pipe = HostPipeline(M, N, K, compute=mode)
    pipe.run(items)
    for (_, _, Ch), C in zip(items, ref):
        assert torch.equal(Ch, C)
