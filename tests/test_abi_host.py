"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every symbol include/pnorm.h declares, and its host logic (options, status
strings, workspace sizes, defaults, argument validation) behaves as documented.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def binding():
    from paper_1511_05690_gb300 import build
    build.build()
    from paper_1511_05690_gb300 import _binding
    _binding.load()
    return _binding


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^PN_API\s+[\w\s\*]+?\b(\w+)\s*\(", text, flags=re.M))
    return names


def test_library_exports_every_declared_symbol(binding):
    declared = _declared_symbols()
    assert len(declared) >= 15
    lib = binding.load()
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(binding.EXPORTS)


def test_status_strings(binding):
    lib = binding.load()
    for code in range(8):
        assert lib.pn_status_string(code).decode().startswith("PN_")
    assert lib.pn_status_string(99) == b"unknown pn_status"


def test_default_opts(binding):
    o = binding.make_opts()
    assert o.n_p == 7 and list(o.p_log2[:7]) == list(range(7))
    assert o.compute == binding.PN_BF16 and o.scaling == 2 and o.diag_policy == 2


def test_default_tau_matches_oracle_reading(binding, orc):
    lib = binding.load()
    for K in (1, 256, 4096, 16384):
        for mode in range(5):
            assert lib.pn_default_tau(K, mode) == orc.default_tau(K, mode)
    assert lib.pn_default_tau(10, 9) < 0


def test_workspace_sizes(binding):
    lib = binding.load()
    o = binding.make_opts(compute="bf16")
    s1 = lib.pn_workspace_size(1000, 1000, 1000, ctypes.byref(o))
    s2 = lib.pn_workspace_size(2000, 1000, 1000, ctypes.byref(o))
    assert 0 < s1 < s2 and s1 % 256 == 0
    # the operand images dominate: one level's (A + B) at 2 bytes per element
    # (every p level reuses the same image buffers)
    assert 2 * 1024 * 1024 * 2 <= s1 < 2 * 2 * 1024 * 1024 * 2
    o32 = binding.make_opts(compute="f32")
    assert lib.pn_workspace_size(1000, 1000, 1000, ctypes.byref(o32)) > 3 * s1
    bad = binding.make_opts()
    bad.n_p = 17
    assert lib.pn_workspace_size(10, 10, 10, ctypes.byref(bad)) == 0
    bad = binding.make_opts()
    bad.p_log2[3] = bad.p_log2[2]
    assert lib.pn_workspace_size(10, 10, 10, ctypes.byref(bad)) == 0
    assert lib.pn_workspace_size(-1, 10, 10, ctypes.byref(o)) == 0
    assert lib.pn_apsp_workspace_size(100, ctypes.byref(o)) > lib.pn_workspace_size(
        100, 100, 100, ctypes.byref(o))
    # the r = 1 projection keeps a second word of state per 32 entries (M N / 8 bytes)
    oproj = binding.make_opts(compute="bf16", estimator=1)
    s1p = lib.pn_workspace_size(1000, 1000, 1000, ctypes.byref(oproj))
    assert s1 + 1000 * 1024 // 8 <= s1p <= s1 + 1000 * 1024 // 8 + 4096
    # the r = 2 projection: two words of stage per 32 entries, two parked sums
    # per entry (2 M N floats) and the extra half levels' work lists
    o2 = binding.make_opts(compute="bf16", estimator=2)
    s2p = lib.pn_workspace_size(1000, 1000, 1000, ctypes.byref(o2))
    assert s1p + 1000 * 1024 // 8 + 8 * 1000 * 1000 <= s2p <= s1p + 1000 * 1024 // 8 + 8 * 1000 * 1000 + 65536
    bad = binding.make_opts(estimator=3)
    assert lib.pn_workspace_size(10, 10, 10, ctypes.byref(bad)) == 0
    bad = binding.make_opts(estimator=2, correction=2, n_fit=4, fit_i=16, fit_j=16)
    assert lib.pn_workspace_size(10, 10, 10, ctypes.byref(bad)) == 0
    bad = binding.make_opts(estimator=2, correction=1)
    assert lib.pn_workspace_size(10, 10, 10, ctypes.byref(bad)) == 0
    # corrections: division only with the plain estimator; the affine model
    # needs its sample entries
    assert lib.pn_workspace_size(10, 10, 10, ctypes.byref(binding.make_opts(correction=1))) > 0
    bad = binding.make_opts(correction=1, estimator=1)
    assert lib.pn_workspace_size(10, 10, 10, ctypes.byref(bad)) == 0
    bad = binding.make_opts(correction=2)
    assert lib.pn_workspace_size(10, 10, 10, ctypes.byref(bad)) == 0
    good = binding.make_opts(correction=2, n_fit=4, fit_i=16, fit_j=16)
    assert lib.pn_workspace_size(10, 10, 10, ctypes.byref(good)) > 0
    bad = binding.make_opts(correction=3)
    assert lib.pn_workspace_size(10, 10, 10, ctypes.byref(bad)) == 0


def test_argument_validation_before_any_device_call(binding):
    """Invalid options and shapes are rejected on the host (PN_EINVAL) before the
    library looks for a device; empty problems succeed without touching it."""
    lib = binding.load()
    o = binding.make_opts()
    bad = binding.make_opts()
    bad.compute = 9
    z = None
    assert lib.maxprod_pnorm(4, 4, 4, z, 4, z, 4, z, 4, z, z, ctypes.byref(bad), z, 0, z) == 1
    assert lib.maxprod_pnorm(4, 4, 4, 16, 2, 16, 4, 16, 4, z, z, ctypes.byref(o), z, 0, z) == 1
    assert lib.maxprod_pnorm(0, 4, 4, z, 4, z, 4, z, 4, z, z, ctypes.byref(o), z, 0, z) == 0
    assert lib.maxprod_exact(4, 4, 4, z, 4, z, 4, z, 4, 5, z) == 1
    assert lib.maxprod_exact(0, 4, 4, z, 4, z, 4, z, 4, 0, z) == 0
    assert lib.pn_maxprod_exact_variant(4, 4, 4, z, 4, z, 4, z, 4, 0, 3, z) == 1
    # the projection estimator: APSP and the adjoint refuse it (PN_EUNSUPPORTED)
    proj = binding.make_opts(compute="f32", estimator=1)
    assert lib.apsp_pnorm(4, 16, 4, 16, 4, 0, ctypes.byref(proj), z, 0, z) == 7
    assert lib.maxprod_pnorm_backward(4, 4, 4, 16, 16, 16, 16, 16, 16, 16, 16,
                                      ctypes.byref(proj), z, 0, z) == 7
    div = binding.make_opts(compute="f32", correction=1)
    assert lib.apsp_pnorm(4, 16, 4, 16, 4, 0, ctypes.byref(div), z, 0, z) == 7
    # max-convolution: shapes and limits are checked on the host
    assert lib.maxconv_pnorm(0, 4, z, 4, 4, z, 4, z, 7, z, 7, ctypes.byref(o), z) == 0
    assert lib.maxconv_pnorm(2, 0, z, 4, 4, z, 4, z, 7, z, 7, ctypes.byref(o), z) == 1
    assert lib.maxconv_pnorm(2, 5000, 16, 5000, 4000, 16, 4000, 16, 8999, z, 0,
                             ctypes.byref(o), z) == 7
    assert lib.maxconv_pnorm(2, 4, 16, 4, 4, 16, 4, 16, 7, z, 0, ctypes.byref(proj), z) == 7
    assert lib.maxconv_pnorm(2, 4, 16, 3, 4, 16, 4, 16, 7, z, 0, ctypes.byref(o), z) == 1
    assert lib.maxconv_exact(2, 4, 16, 4, 0, 16, 4, 16, 7, z) == 1
    assert lib.maxconv_exact(1, 1 << 30, 16, 1 << 30, 1, 16, 1, 16, 1 << 30, z) == 7
    assert lib.pn_maxconv_default_tau() == 1e-12
    # long max-convolution: workspace size and checks before any device call
    w1 = lib.pn_maxconv_long_workspace_size(6000, 5000, 1)
    w0 = lib.pn_maxconv_long_workspace_size(6000, 5000, 0)
    assert w1 >= 16384 * 16 and w0 >= w1 + 10999
    assert lib.pn_maxconv_long_workspace_size(1 << 22, 2, 1) == 0
    assert lib.maxconv_pnorm_long(6000, 16, 5000, 16, 16, z, ctypes.byref(o), 256, 100, z) == 3
    assert lib.maxconv_pnorm_long(6000, 16, 5000, 16, 16, 16, ctypes.byref(o), 264, w1, z) == 2
    assert lib.maxconv_pnorm_long(1 << 22, 16, 2, 16, 16, 16, ctypes.byref(o), 256, w1, z) == 7
    assert lib.pn_maxprod_exact_variant(4, 4, 4, z, 4, z, 4, z, 4, 0, -1, z) == 1
    assert lib.apsp_pnorm(0, z, 0, z, 0, 0, ctypes.byref(o), z, 0, z) == 0
    assert lib.apsp_pnorm(4, z, 4, z, 4, 0, ctypes.byref(o), z, 0, z) == 1


def test_missing_library_fails_loudly(binding, monkeypatch):
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "LIB_PATH", "/nonexistent/libpnorm.so")
    with pytest.raises(RuntimeError, match="not built"):
        binding.load()


def _group_args(sizes, ptr=0x10000):
    """ctypes arguments of a group: MNK and distinct 256-byte-aligned placeholder
    addresses (the table builder stores them and reads their alignment only)."""
    vp = ctypes.c_void_p
    n = len(sizes)
    MNK = (ctypes.c_int64 * max(1, 3 * n))(*[v for s in sizes for v in s])
    mk = lambda k: (vp * max(1, n))(*[None if 0 in s[:2] else ptr + 256 * (3 * g + k)  # noqa: E731
                                       for g, s in enumerate(sizes)])
    return n, MNK, mk(0), mk(1), mk(2)


def _build(lib, binding, sizes, o, short=0):
    import numpy as np
    n, MNK, A, B, C = _group_args(sizes)
    tb = lib.pn_grouped_table_bytes(n, MNK, ctypes.byref(o))
    assert tb > 0
    table = np.zeros(tb, dtype=np.uint8)
    ws = ctypes.c_size_t(0)
    rc = lib.pn_grouped_build_table(n, MNK, A, B, C, ctypes.byref(o),
                                    table.ctypes.data_as(ctypes.c_void_p), tb - short,
                                    ctypes.byref(ws))
    return rc, table, ws.value


def test_grouped_table_builder_on_the_host(binding):
    """pn_grouped_build_table runs on the host only: deterministic bytes, a
    workspace that holds every problem's operand images, empty problems
    without pointers or tiles, and PN_EINVAL for every invalid argument."""
    import numpy as np
    lib = binding.load()
    o = binding.make_opts(compute="bf16")
    sizes = [(16, 16, 16), (300, 200, 1000), (129, 1, 77), (1, 700, 5)]
    rc, t1, ws = _build(lib, binding, sizes, o)
    assert rc == 0 and ws > 0 and ws % 256 == 0
    rc2, t2, ws2 = _build(lib, binding, sizes, o)
    assert rc2 == 0 and ws2 == ws and np.array_equal(t1, t2)
    # the 128-wide layout alone needs every A and B^T image tile: 16 KB per
    # 128 rows (columns) x 64 values of K in BF16
    img = sum((-(-m // 128) + -(-n // 128)) * -(-k // 64) for m, n, k in sizes) * 16384
    assert ws >= img
    # more work, larger table and workspace
    rc3, t3, ws3 = _build(lib, binding, sizes + [(512, 512, 512)], o)
    assert rc3 == 0 and len(t3) > len(t1) and ws3 > ws
    # empty problems take no pointers and no tiles (only their scale words)
    rc4, t4, ws4 = _build(lib, binding, sizes + [(0, 50, 50), (50, 0, 50), (0, 0, 0)], o)
    assert rc4 == 0 and ws <= ws4 <= ws + 4096
    # 3xTF32: two planes of 4-byte values, 32 per 128-byte image row
    o32 = binding.make_opts(compute="f32")
    rc5, _, ws5 = _build(lib, binding, sizes, o32)
    img32 = 2 * sum((-(-m // 128) + -(-n // 128)) * -(-k // 32) for m, n, k in sizes) * 16384
    assert rc5 == 0 and ws5 >= img32 > 3 * img
    # invalid arguments
    assert _build(lib, binding, sizes, o, short=1)[0] == 1            # table too small
    n, MNK, A, B, C = _group_args([(4, 4, 0)])                       # empty contraction
    assert lib.pn_grouped_table_bytes(n, MNK, ctypes.byref(o)) > 0
    tab = np.zeros(1 << 16, dtype=np.uint8)
    vpt = tab.ctypes.data_as(ctypes.c_void_p)
    assert lib.pn_grouped_build_table(n, MNK, A, B, C, ctypes.byref(o), vpt, tab.size, None) == 1
    n, MNK, A, B, C = _group_args([(4, 4, 4)])
    A[0] = None                                                       # missing operand
    assert lib.pn_grouped_build_table(n, MNK, A, B, C, ctypes.byref(o), vpt, tab.size, None) == 1
    for bad in ([(-1, 4, 4)], [(4, 1 << 30, 4)]):                     # size out of range
        n, MNK, A, B, C = _group_args(bad)
        assert lib.pn_grouped_table_bytes(n, MNK, ctypes.byref(o)) == 0
        assert lib.pn_grouped_build_table(n, MNK, A, B, C, ctypes.byref(o), vpt, tab.size,
                                          None) == 1
    badopt = binding.make_opts(compute="bf16")
    badopt.n_p = 0
    n, MNK, A, B, C = _group_args(sizes)
    assert lib.pn_grouped_table_bytes(n, MNK, ctypes.byref(badopt)) == 0
    assert lib.pn_grouped_build_table(n, MNK, A, B, C, ctypes.byref(badopt), vpt, tab.size,
                                      None) == 1
    assert lib.pn_grouped_build_table(-1, MNK, A, B, C, ctypes.byref(o), vpt, tab.size, None) == 1


def test_python_layer_has_no_cpu_path(binding):
    """Every entry point of the Python layer refuses host tensors (and other
    dtypes or ranks) before any work: there is no CPU fallback."""
    torch = pytest.importorskip("torch")
    import paper_1511_05690_gb300 as pn
    a = torch.rand(8, 8)
    calls = [lambda: pn.maxprod_pnorm(a, a), lambda: pn.maxprod_exact(a, a),
             lambda: pn.apsp_pnorm(a), lambda: pn.GroupedProduct([a], [a]),
             lambda: pn.maxconv_pnorm(a, a), lambda: pn.maxconv_exact(a, a),
             lambda: pn.topk_xy(a, a, 3)]
    for call in calls:
        with pytest.raises(ValueError, match="CUDA"):
            call()
    with pytest.raises(ValueError, match="float32"):
        pn.maxprod_pnorm(a.double(), a.double())
    with pytest.raises(ValueError, match="2-D"):
        pn.maxprod_pnorm(torch.rand(8), a)
