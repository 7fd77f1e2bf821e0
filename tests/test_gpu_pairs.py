"""GPU parity of the CTA-pair tensor-core path (tile_m = 256: two SMs of a
cluster share one 256 x 256 or 256 x 128 tile through cta_group::2 MMAs, each
loading one 128-row half of A and one half of the B^T column tile: a whole
128-row image block, or 64 rows of one).  The arithmetic per entry is that of the
single-CTA path, so the oracle tolerances of the product tests apply, and the
pair and single-CTA results are held to each other within them.  Shapes with
an odd number of 128-row tiles use the padded zero block of A; several-level
data exercise the per-tile push that either half of a pair may make."""
import numpy as np
import pytest

import workloads
from test_gpu_product import _compare, _multilevel_inputs, pnorm_tol

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


@pytest.mark.parametrize("width", [256, 128])
@pytest.mark.parametrize("mode", ["f32", "bf16", "tf32", "f16", "e4m3"])
@pytest.mark.parametrize("shape", [(256, 256, 300), (300, 520, 257), (640, 384, 1000),
                                   (100, 300, 64)])
def test_pairs_match_oracle(pn, orc, mode, shape, width):
    """Every format and both pair widths, ragged shapes, an odd count of
    128-row tiles (300, 640 rows: 3 and 5 tile rows) and a product smaller
    than one pair tile."""
    M, N, K = shape
    A, B = workloads.wide_range_pair(M, N, K, seed=4000 + M + K)
    tau = orc.default_tau(K, 3) if mode == "f16" else None
    C, psel, ssel, err = _compare(pn, orc, A, B, mode, list(range(7)), tau=tau,
                                  tile_n=width, tile_m=256)
    Cs, ps, ss = pn.maxprod_pnorm(_dev(A), _dev(B), compute=mode, tau=tau, tile_n=256,
                                  tile_m=128)
    Cs, ps = Cs.cpu().numpy(), ps.cpu().numpy()
    agree = ps == psel
    tol = np.vectorize(lambda lp: pnorm_tol(mode, K, lp))(psel & 0x7F)
    rel = np.abs(C - Cs) / np.maximum(np.abs(Cs), 1e-30)
    assert np.all(rel[agree] <= 2 * tol[agree])


@pytest.mark.parametrize("width", [256, 128])
@pytest.mark.parametrize("mode", ["f32", "bf16"])
def test_pairs_lower_levels(pn, orc, mode, width):
    """Entries resolving at several levels: a pair tile goes down when either
    half has entries left, each half keeps its own resolved bits."""
    A, B = _multilevel_inputs(520, 700, 256, seed=4100)
    C, psel, _, _ = _compare(pn, orc, A, B, mode, list(range(7)), tile_n=width, tile_m=256)
    assert len(set(np.unique(psel & 0x7F).tolist())) >= 2


def test_pairs_projection_r1(pn, orc):
    """The r = 1 projection over several levels with pairs equals the
    single-CTA result within the projection's tolerance."""
    from test_gpu_projection import proj_tol
    A, B = _multilevel_inputs(384, 520, 200, seed=4200)
    dA, dB = _dev(A), _dev(B)
    tau = orc.default_tau(200, 0)
    C2, p2, _ = pn.maxprod_pnorm(dA, dB, compute="f32", tau=tau, estimator=1, tile_m=256)
    C1, p1, _ = pn.maxprod_pnorm(dA, dB, compute="f32", tau=tau, estimator=1, tile_m=128)
    assert torch.equal(p1, p2)
    ref = orc.pnorm(A.astype(np.float64), B.astype(np.float64), list(range(7)), tau,
                    estimator=1)
    C2 = C2.cpu().numpy()
    q = (p2.cpu().numpy() & 0x7F).astype(int)
    tol = np.vectorize(lambda lp: proj_tol("f32", 200, lp))(q)
    err = np.abs(C2 - ref["C"]) / ref["C"]
    assert np.all(err <= tol), float(err.max())


@pytest.mark.parametrize("width", [256, 128])
@pytest.mark.parametrize("mode", ["f32", "bf16"])
def test_pairs_projection_r2_equals_single(pn, mode, width):
    """The r = 2 projection with pairs: the two halves of a pair tile decide
    together whether it visits the half level (either half started a chain),
    and the results equal the single-CTA run bit for bit over several levels
    (a half without chains at a half level parks nothing)."""
    A, B = _multilevel_inputs(384, 520, 200, seed=4300)
    dA, dB = _dev(A), _dev(B)
    r2 = pn.maxprod_pnorm(dA, dB, compute=mode, estimator=2, tile_m=256, tile_n=width)
    r1 = pn.maxprod_pnorm(dA, dB, compute=mode, estimator=2, tile_m=128)
    for x2, x1 in zip(r2, r1):
        assert torch.equal(x2, x1)
    assert len(torch.unique(r2[1] & 0x7F)) >= 2


@pytest.mark.parametrize("width,n", [(256, 5120), (128, 3584)])
def test_pairs_tile_per_epilogue_group(pn, width, n):
    """Short contractions over many tiles (K = 256, at least four pair tiles
    per cluster): each epilogue group of a pair's CTAs finishes whole tiles
    in turn instead of all groups sharing every tile.  Entries spread over
    several levels; C, p_sel and S_sel equal the single-CTA run bit for bit."""
    A, B = _multilevel_inputs(n, n, 256, seed=4500 + width)
    dA, dB = _dev(A), _dev(B)
    r2 = pn.maxprod_pnorm(dA, dB, compute="bf16", tile_m=256, tile_n=width)
    r1 = pn.maxprod_pnorm(dA, dB, compute="bf16", tile_m=128, tile_n=width)
    for x2, x1 in zip(r2, r1):
        assert torch.equal(x2, x1)
    assert len(torch.unique(r2[1] & 0x7F)) >= 2


@pytest.mark.parametrize("width", [256, 128])
def test_pairs_apsp_matches_single(pn, orc, width):
    """APSP squarings (diagonal reset and clamp in the epilogue) with pairs:
    the same distances as with single CTAs within the per-squaring bar."""
    n = 700
    W = workloads.apsp_weights(n, density=0.1, seed=4300)
    tau = orc.default_tau(n, orc.F32_EXACT)
    dW = torch.from_numpy(W).cuda()
    D2 = pn.apsp_pnorm(dW, compute="f32", tau=tau, tile_m=256, tile_n=width).cpu().numpy()
    D1 = pn.apsp_pnorm(dW, compute="f32", tau=tau, tile_m=128).cpu().numpy()
    fin = np.isfinite(D1)
    assert np.array_equal(np.isfinite(D2), fin)
    assert np.abs(D2[fin] - D1[fin]).max() <= (2 ** 10 - 1) * 1e-5
    assert np.all(np.diag(D2) == 0)


def test_pairs_cuda_graph(pn):
    """A pair launch (a cluster launch) captured in a CUDA graph and replayed."""
    A, B = workloads.uniform_pair(512, 512, 384, seed=4400)
    dA, dB = _dev(A), _dev(B)
    C0, _, _ = pn.maxprod_pnorm(dA, dB, compute="bf16", tile_m=256)
    out = torch.empty_like(C0)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            pn.maxprod_pnorm(dA, dB, compute="bf16", tile_m=256, out=out, check=False,
                             stream=s)
    torch.cuda.current_stream().wait_stream(s)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, C0)
