"""GPU parity of the grouped launch (many products, one launch per p level),
its CUDA-graph capture and the tile-width autotuner."""
import ctypes

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


_U = {"f32": 2.0 ** -21, "bf16": 2.0 ** -8, "e4m3": 2.0 ** -4}
_M = {"f32": 21, "bf16": 7, "e4m3": 3}
_CODE = {"f32": 0, "bf16": 2, "e4m3": 4}


def _tol(mode, K, plog):
    p = 2.0 ** plog
    s = 2 * (p - 1) * 2.0 ** -24 + 2 * _U[mode] + 2.0 ** -_M[mode] + K * 2.0 ** -23
    return 1.5 * ((1 + s) ** (1.0 / p) - 1) + 2e-7


def _problems(seed, count=40, cap=300):
    sizes = np.minimum(workloads.grouped_sizes(count, seed=seed), cap)
    probs = workloads.grouped_problems(sizes, seed=seed)
    # a few non-square and ragged shapes, and an empty one
    g = workloads.rng(seed + 5)
    probs.append(((1 - g.random((37, 129))).astype(np.float32),
                  (1 - g.random((129, 5))).astype(np.float32)))
    probs.append((np.zeros((0, 7), np.float32), np.zeros((7, 9), np.float32)))
    probs.append(((1 - g.random((130, 1))).astype(np.float32),
                  (1 - g.random((1, 260))).astype(np.float32)))
    return probs


@pytest.mark.parametrize("mode,tile_n", [("bf16", 128), ("bf16", 256), ("f32", 128),
                                          ("e4m3", 256)])
def test_grouped_matches_oracle(pn, orc, mode, tile_n):
    probs = _problems(800 + tile_n)
    plan = pn.GroupedProduct([_dev(a) for a, _ in probs], [_dev(b) for _, b in probs],
                             compute=mode, tile_n=tile_n)
    Cs = [c.cpu().numpy() for c in plan.run(check=True)]
    pl = list(range(7))
    for (A, B), C in zip(probs, Cs):
        if A.shape[0] == 0:
            assert C.shape == (0, B.shape[1])
            continue
        K = A.shape[1]
        tau = orc.default_tau(K, _CODE[mode])
        ref = orc.pnorm(A.astype(np.float64), B.astype(np.float64), pl, tau, want_S=True)
        q = ref["p_sel"] & 0x7F
        tol = np.vectorize(lambda lp: _tol(mode, K, lp))(q)
        # entries whose S is within the error band of tau may take another p*
        near = np.zeros(C.shape, bool)
        for qq in range(7):
            near |= np.abs(ref["S"][qq] / tau - 1) < 4 * 1.5 * _tol(mode, K, 0)
        err = np.abs(C - ref["C"]) / ref["C"]
        assert np.all((err <= tol) | near), (A.shape, B.shape, float(err.max()))


def test_grouped_equals_single_products(pn):
    probs = _problems(811)
    for tile_n in (128, 256):
        plan = pn.GroupedProduct([_dev(a) for a, _ in probs], [_dev(b) for _, b in probs],
                                 compute="bf16", tile_n=tile_n)
        Cs = plan.run(check=True)
        for (A, B), C in zip(probs, Cs):
            if A.shape[0] == 0:
                continue
            C1, _, _ = pn.maxprod_pnorm(_dev(A), _dev(B), compute="bf16", tile_n=tile_n)
            assert torch.equal(C, C1)


def test_grouped_cuda_graph_replay(pn):
    """The run step is captured once and replayed on new input values."""
    probs = _problems(812, count=24)
    As = [_dev(a) for a, _ in probs]
    Bs = [_dev(b) for _, b in probs]
    plan = pn.GroupedProduct(As, Bs, compute="bf16", tile_n=256)
    plan.run(check=True)  # warm-up outside the capture (kernel attributes)
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            plan.run(stream=s)
    torch.cuda.current_stream().wait_stream(s)
    for rep in range(2):
        g = workloads.rng(900 + rep)
        for a in plan.As:
            a.copy_(torch.from_numpy((1 - g.random(tuple(a.shape))).astype(np.float32)))
        graph.replay()
        torch.cuda.synchronize()
        for a, b, c in zip(plan.As, plan.Bs, plan.Cs):
            if a.shape[0] == 0:
                continue
            c1, _, _ = pn.maxprod_pnorm(a, b, compute="bf16", tile_n=256)
            assert torch.equal(c, c1)


def test_grouped_autotune_and_untuned_rule(pn):
    probs = _problems(813, count=32, cap=1024)
    plan = pn.GroupedProduct([_dev(a) for a, _ in probs], [_dev(b) for _, b in probs],
                             compute="bf16", tile_n=0)
    ref = [c.clone() for c in plan.run(check=True)]
    chosen = plan.autotune()
    assert chosen in (128, 256)
    Cs = plan.run(check=True)
    plan256 = pn.GroupedProduct(plan.As, plan.Bs, compute="bf16", tile_n=chosen)
    for c, c2 in zip(Cs, plan256.run(check=True)):
        assert torch.equal(c, c2)
    del ref


def test_single_autotune(pn):
    A, B = workloads.uniform_pair(1024, 1536, 800, seed=9)
    chosen = pn.autotune(_dev(A), _dev(B), compute="bf16")
    assert chosen in (128, 256)
    C, _, _ = pn.maxprod_pnorm(_dev(A), _dev(B), compute="bf16")
    C2, _, _ = pn.maxprod_pnorm(_dev(A), _dev(B), compute="bf16", tile_n=chosen)
    assert torch.equal(C, C2)


def test_grouped_rejects_empty_contraction(pn):
    with pytest.raises(pn.PnError) as ei:
        pn.GroupedProduct([torch.zeros((4, 0), device="cuda")],
                          [torch.zeros((0, 3), device="cuda")])
    assert ei.value.status == 1
