"""GPU parity of the grouped call (many products in one persistent launch over
every problem, p level and tile), its per-level launch sequence, its CUDA-graph
capture and the tile-width autotuner."""
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


@pytest.mark.parametrize("scaling", [0, 1])
def test_grouped_scaling_modes_equal_single_products(pn, scaling):
    """Scaling 0 (no scales; the strip kernel and the persistent launch) and
    scaling 1 (one global scale per problem; the per-level launches) give the
    single products' results bit for bit, over ragged and empty problems."""
    probs = _problems(815, count=24)
    As = [_dev(a) for a, _ in probs]
    Bs = [_dev(b) for _, b in probs]
    for tile_n in (128, 256):
        plan = pn.GroupedProduct(As, Bs, compute="bf16", tile_n=tile_n, scaling=scaling)
        Cs = plan.run(check=True)
        for A, B, C in zip(As, Bs, Cs):
            if A.shape[0] == 0:
                continue
            C1, _, _ = pn.maxprod_pnorm(A, B, compute="bf16", tile_n=tile_n, scaling=scaling)
            assert torch.equal(C, C1), (tuple(A.shape), tuple(B.shape), tile_n)


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
    assert chosen in (128, 256, 384, 512)
    C, _, _ = pn.maxprod_pnorm(_dev(A), _dev(B), compute="bf16")
    shape = (dict(tile_n=chosen - 256, tile_m=256) if chosen > 256
             else dict(tile_n=chosen, tile_m=128))
    C2, _, _ = pn.maxprod_pnorm(_dev(A), _dev(B), compute="bf16", **shape)
    assert torch.equal(C, C2)


def test_grouped_rejects_empty_contraction(pn):
    with pytest.raises(pn.PnError) as ei:
        pn.GroupedProduct([torch.zeros((4, 0), device="cuda")],
                          [torch.zeros((0, 3), device="cuda")])
    assert ei.value.status == 1


def _multilevel_problems(seed, count=12):
    """Square problems whose entries spread p* over several levels: small
    cross terms and one large product per row (as in the product tests)."""
    g = workloads.rng(seed)
    out = []
    for n in [int(x) for x in g.integers(20, 300, count)] + [129, 257]:
        A = (0.05 * (0.5 + 0.5 * g.random((n, n)))).astype(np.float32)
        B = (0.05 * (0.5 + 0.5 * g.random((n, n)))).astype(np.float32)
        A[np.arange(n), np.arange(n)] = 1.0
        B[(np.arange(n) + 1) % n, np.arange(n)] = 1.0
        out.append((A, B))
    return out


@pytest.mark.parametrize("mode,tile_n,estimator,correction",
                         [("bf16", 128, 0, 0), ("bf16", 256, 0, 0), ("f32", 128, 0, 0),
                          ("tf32", 256, 0, 0), ("f16", 128, 0, 0), ("e4m3", 256, 0, 0),
                          ("bf16", 256, 1, 0), ("f32", 128, 0, 1)])
def test_grouped_persistent_equals_level_launches(pn, mode, tile_n, estimator, correction):
    """The single persistent launch (top-level images written before it, or
    by its own block builders) and the per-level launch sequence run the
    same arithmetic: bit-identical results, here with entries resolving at
    several levels (work lists carried between levels inside the launch), the
    r = 1 projection and the K^(1/p*) correction."""
    probs = _multilevel_problems(830) + _problems(831, count=16)
    As = [_dev(a) for a, _ in probs]
    Bs = [_dev(b) for _, b in probs]
    kw = dict(compute=mode, tile_n=tile_n, estimator=estimator, correction=correction)
    tau = 1.0 if mode == "f16" else None  # FP16 operands: a tau the data clears at low p
    persist = pn.GroupedProduct(As, Bs, tau=tau, **kw)
    inside = pn.GroupedProduct(As, Bs, tau=tau, debug_flags=8, **kw)
    levels = pn.GroupedProduct(As, Bs, tau=tau, debug_flags=4, **kw)
    C1 = persist.run(check=True)
    C2 = levels.run(check=True)
    C3 = inside.run(check=True)
    for a, c1, c2, c3 in zip(As, C1, C2, C3):
        assert torch.equal(c1, c2), (tuple(a.shape), mode)
        assert torch.equal(c3, c2), (tuple(a.shape), mode)
    # several levels took part
    C, psel, _ = pn.maxprod_pnorm(As[0], Bs[0], compute=mode, tile_n=tile_n, tau=tau)
    assert len(torch.unique(psel & 0x7F)) >= 2


def test_grouped_persistent_multilevel_matches_oracle(pn, orc):
    probs = _multilevel_problems(840, count=6)
    plan = pn.GroupedProduct([_dev(a) for a, _ in probs], [_dev(b) for _, b in probs],
                             compute="f32", tile_n=128)
    Cs = [c.cpu().numpy() for c in plan.run(check=True)]
    pl = list(range(7))
    levels = set()
    for (A, B), C in zip(probs, Cs):
        K = A.shape[1]
        tau = orc.default_tau(K, 0)
        ref = orc.pnorm(A.astype(np.float64), B.astype(np.float64), pl, tau)
        levels |= set(np.unique(ref["p_sel"] & 0x7F).tolist())
        err = np.abs(C - ref["C"]) / ref["C"]
        assert err.max() <= 1e-5, float(err.max())
    assert len(levels) >= 2  # tiles carried to a lower level inside the launch


@pytest.mark.parametrize("flags", [0, 8])
def test_grouped_persistent_domain_error(pn, flags):
    """A negative value in one problem of the group raises PN_EDOMAIN (from
    the maxima kernel, or with flag 8 from the block builders of the
    persistent launch), and the context stays usable."""
    probs = _problems(850, count=10)
    As = [_dev(a) for a, _ in probs]
    Bs = [_dev(b) for _, b in probs]
    As[3][2, 1] = -1.0
    plan = pn.GroupedProduct(As, Bs, compute="bf16", debug_flags=flags)
    with pytest.raises(pn.PnError) as ei:
        plan.run(check=True)
    assert ei.value.status == 4
    As[3][2, 1] = 0.5
    Bs[5][0, 0] = float("nan")
    plan = pn.GroupedProduct(As, Bs, compute="bf16", debug_flags=flags)
    with pytest.raises(pn.PnError) as ei:
        plan.run(check=True)
    assert ei.value.status == 4
    Bs[5][0, 0] = 0.5
    pn.GroupedProduct(As, Bs, compute="bf16", debug_flags=flags).run(check=True)


def test_grouped_bench_configuration_sampled(pn, orc):
    """The grouped configuration the bench times, at full size: 4096 square
    problems of n = round(16 * 64^U) with entries 1 - U[0,1), BF16 operands,
    P = {1..64}, the tile width the autotuner picks and the launches the bench
    replays (the strip kernel, then the persistent launch).  In 48 problems
    (the largest, the smallest and 46 drawn at random) 32 sampled entries each
    against the FP64 oracle at the oracle's own p*, entries within the error
    band of tau excepted."""
    sizes = workloads.grouped_sizes(4096)
    g = torch.Generator(device="cuda")
    g.manual_seed(workloads.SEED_BASE + 3)
    As = [1 - torch.rand((int(m), int(m)), generator=g, device="cuda") for m in sizes]
    Bs = [1 - torch.rand((int(m), int(m)), generator=g, device="cuda") for m in sizes]
    plan = pn.GroupedProduct(As, Bs, compute="bf16")
    assert plan.autotune() in (128, 256)
    Cs = plan.run(check=True)
    h = workloads.rng(None, 140)
    pick = set(h.choice(len(sizes), 46, replace=False).tolist())
    pick |= {int(np.argmax(sizes)), int(np.argmin(sizes))}
    pl = list(range(7))
    checked = 0
    for gi in sorted(pick):
        A = As[gi].double().cpu().numpy()
        B = Bs[gi].double().cpu().numpy()
        n = A.shape[0]
        ii, jj = h.integers(0, n, 32), h.integers(0, n, 32)
        r, c = orc.row_scales(A), orc.col_scales(B)
        _, S = orc.entries(A, B, ii, jj, pl, r, c)
        tau = orc.default_tau(n, orc.BF16)
        stable = S >= tau
        q = np.where(stable.any(axis=1), len(pl) - 1 - np.argmax(stable[:, ::-1], axis=1), 0)
        lp = np.array(pl)[q]
        expect = r[ii] * c[jj] * np.power(S[np.arange(len(ii)), q], 1.0 / 2.0 ** lp)
        got = Cs[gi][torch.from_numpy(ii).cuda(), torch.from_numpy(jj).cuda()].double().cpu().numpy()
        tol = np.array([_tol("bf16", n, int(x)) for x in lp])
        near = (np.abs(S / tau - 1) < 4 * 1.5 * _tol("bf16", n, 0)).any(axis=1)
        err = np.abs(got - expect) / expect
        assert np.all((err <= tol) | near), (n, float(err.max()))
        checked += int((~near).sum())
    assert checked >= 48 * 32 // 2
