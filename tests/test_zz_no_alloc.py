"""lsp_periodogram_noalloc: the allocation-free entry point.

It is meant for callers that cannot allocate device memory while they run
(for instance an application whose own pool owns the GPU); its scratch is a
fixed file-scope device array.  Here it is called through the C ABI twice in a
row on different inputs, and each result must match lsp_periodogram (the
context-based entry point) within the parity tolerance of the other tests:
|dP| <= 1e-4 max P.  The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-4


@pytest.fixture(scope="module")
def lsp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1007_1658_gb300 import build, lsp as L
    build.build()
    return L


def _inputs():
    from paper_1007_1658_gb300 import synth
    a = synth.plain_1k()
    rng = np.random.default_rng(77)
    t = np.sort(rng.uniform(0.0, 300.0, 20011))
    X = 4.0 + rng.normal(size=t.size) + 0.3 * np.sin(2 * np.pi * 1.234 * t)
    df = 1.0 / (4.0 * (t.max() - t.min()))
    b = (t, X, df, df, 30001)
    return [(a.t, a.X, a.f0, a.df, a.nf), b]


def test_noalloc_matches_context_path_twice_in_a_row(lsp):
    lib = lsp.load()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    cases = _inputs()
    dev_in = [(torch.from_numpy(t).to(dev), torch.from_numpy(X).to(dev), f0, df, nf) for t, X, f0, df, nf in cases]
    outs = []
    for t, X, f0, df, nf in dev_in:
        out = torch.full((nf,), -1.0, dtype=torch.float32, device=dev)
        st = lib.lsp_periodogram_noalloc(ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(X.data_ptr()), t.numel(),
                                         f0, df, nf, ctypes.c_void_p(out.data_ptr()),
                                         ctypes.c_void_p(stream.cuda_stream))
        assert st == lsp.OK
        outs.append(out)
    torch.cuda.synchronize()
    with lsp.Context(0) as ctx:
        for (t, X, f0, df, nf), out in zip(dev_in, outs):
            ref = ctx.periodogram(t, X, f0, df, nf)
            ctx.sync(60.0)
            got = out.cpu().numpy().astype(np.float64)
            exp = ref.cpu().numpy().astype(np.float64)
            assert np.all(np.isfinite(got))
            assert np.max(np.abs(got - exp)) <= TOL * exp.max()


def test_noalloc_rejects_oversize_and_host_pointers(lsp):
    lib = lsp.load()
    dev = torch.device("cuda:0")
    t = torch.zeros(16, dtype=torch.float64, device=dev)
    out = torch.empty(4, dtype=torch.float32, device=dev)
    too_many = (1 << 19) + 1
    st = lib.lsp_periodogram_noalloc(ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(t.data_ptr()), too_many,
                                     0.1, 0.1, 4, ctypes.c_void_p(out.data_ptr()), None)
    assert st == lsp.ERR_INVALID_ARG
    h = np.zeros(16)
    st = lib.lsp_periodogram_noalloc(ctypes.c_void_p(h.ctypes.data), ctypes.c_void_p(h.ctypes.data), 16,
                                     0.1, 0.1, 4, ctypes.c_void_p(out.data_ptr()), None)
    assert st == lsp.ERR_INVALID_ARG
