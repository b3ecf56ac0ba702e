"""lsp_periodogram_noalloc: the allocation-free entry point.

It is meant for callers that cannot allocate device memory while they run
(for instance an application whose own memory pool owns the whole GPU, or a
latency-critical loop that cannot take cudaMalloc's synchronization); its
scratch is a fixed file-scope device array.  Here it is called through the C
ABI several times in a row on different inputs, and each result is compared
with the FP64 oracle at the parity tolerance of the other tests (|dP| <= 1e-4
max P, relative error <= 1e-4 at the largest peaks), and with lsp_periodogram
(the context-based entry point).  The largest case uses the array's limit,
N_t = 2^19 samples, with a grid too long for the partial sums of 16,384-sample
chunks to fit at once, so the call runs in several frequency tiles.  The file
is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import oracle
from tests.parity import assert_parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-4
MAX_SAMPLES = 1 << 19
TILE = 98_304  # frequencies per tile at 2^19 samples: 32 chunks of partial sums in 48 MiB


@pytest.fixture(scope="module")
def lsp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1007_1658_gb300 import build, lsp as L
    build.build()
    return L


def _call(lsp, t, X, f0, df, nf, out, stream):
    return lsp.load().lsp_periodogram_noalloc(ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(X.data_ptr()),
                                              t.numel(), f0, df, nf, ctypes.c_void_p(out.data_ptr()),
                                              ctypes.c_void_p(stream.cuda_stream or 1))


def _small_cases():
    from paper_1007_1658_gb300 import synth
    a = synth.plain_1k()
    rng = np.random.default_rng(77)
    t = np.sort(rng.uniform(0.0, 300.0, 20011))
    X = 4.0 + rng.normal(size=t.size) + 0.3 * np.sin(2 * np.pi * 1.234 * t)
    df = 1.0 / (4.0 * (t.max() - t.min()))
    return [(a.t, a.X, a.f0, a.df, a.nf), (t, X, df, df, 30001)]


def _large_case():
    rng = np.random.default_rng(2024)
    n = MAX_SAMPLES
    t = np.sort(rng.uniform(0.0, 1000.0, n))
    df = 1.0 / (4.0 * (t.max() - t.min()))
    k_sig = 150_000  # inside the second frequency tile (the grid is f_k = (k + 1) df)
    f_sig = (k_sig + 1 + 0.3) * df
    X = 0.05 * np.sin(2 * np.pi * f_sig * t) + rng.normal(size=n)
    return t, X, df, df, 300_000, k_sig


def test_noalloc_matches_the_oracle_twice_in_a_row(lsp):
    dev = torch.device("cuda:0")
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    cases = _small_cases()
    dev_in = [(torch.from_numpy(t).to(dev), torch.from_numpy(X).to(dev), f0, df, nf) for t, X, f0, df, nf in cases]
    outs = []
    for t, X, f0, df, nf in dev_in:
        out = torch.full((nf,), -1.0, dtype=torch.float32, device=dev)
        assert _call(lsp, t, X, f0, df, nf, out, stream) == lsp.OK
        outs.append(out)
    torch.cuda.synchronize()
    with lsp.Context(0) as ctx:
        for (t, X, f0, df, nf), out, (th, Xh, *_rest) in zip(dev_in, outs, cases):
            got = out.cpu().numpy().astype(np.float64)
            ref = oracle.periodogram(th, Xh, f0, df, nf)
            assert_parity(got, ref, tol_abs=TOL, tol_peak=TOL, what="noalloc vs oracle, N_t=%d" % th.size)
            ctx_P = ctx.periodogram(t, X, f0, df, nf)
            ctx.sync(60.0)
            exp = ctx_P.cpu().numpy().astype(np.float64)
            assert np.max(np.abs(got - exp)) <= TOL * exp.max()


def test_noalloc_at_the_sample_limit_in_frequency_tiles(lsp):
    t, X, f0, df, nf, k_sig = _large_case()
    dev = torch.device("cuda:0")
    td, Xd = torch.from_numpy(t).to(dev), torch.from_numpy(X).to(dev)
    stream = torch.cuda.current_stream()
    outs = []
    for _ in range(2):  # two calls in a row: the shared array keeps the first call's contents
        out = torch.full((nf,), -1.0, dtype=torch.float32, device=dev)
        assert _call(lsp, td, Xd, f0, df, nf, out, stream) == lsp.OK
        outs.append(out)
    torch.cuda.synchronize()
    got = outs[0].cpu().numpy().astype(np.float64)
    assert np.array_equal(got, outs[1].cpu().numpy().astype(np.float64))
    assert np.all(np.isfinite(got)) and got.min() >= 0.0
    rng = np.random.default_rng(3)
    edges = [b + d for b in range(TILE, nf, TILE) for d in range(-3, 4)]
    ks = np.unique(np.concatenate([rng.integers(0, nf, 96), edges, np.arange(k_sig - 24, k_sig + 25),
                                   [0, nf - 1]]))
    ref = oracle.periodogram_at(t, X, f0 + ks * df)
    scale = max(ref.max(), got.max())
    err = np.abs(got[ks] - ref)
    assert err.max() <= TOL * scale, (err.max() / scale, ks[np.argmax(err)])
    peak = int(np.argmax(ref))
    assert abs(got[ks[peak]] - ref[peak]) <= TOL * ref[peak]
    assert ks[peak] in (k_sig, k_sig + 1)
    # the whole grid against the context path, which splits N_t the same way
    with lsp.Context(0) as ctx:
        P = ctx.periodogram(td, Xd, f0, df, nf)
        ctx.sync(60.0)
        exp = P.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - exp)) <= TOL * exp.max()


def test_noalloc_data_errors_show_as_nan(lsp):
    from paper_1007_1658_gb300 import synth
    c = synth.plain_1k()
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream()
    X = c.X.copy()
    X[17] = np.nan
    out = torch.zeros(64, dtype=torch.float32, device=dev)
    td = torch.from_numpy(c.t).to(dev)
    assert _call(lsp, td, torch.from_numpy(X).to(dev), c.f0, c.df, 64, out, stream) == lsp.OK
    torch.cuda.synchronize()
    assert torch.isnan(out).all()
    # beyond the fixed-point phase's 2^52-turn range
    out = torch.zeros(64, dtype=torch.float32, device=dev)
    assert _call(lsp, td, torch.from_numpy(c.X).to(dev), 1e15, c.df, 64, out, stream) == lsp.OK
    torch.cuda.synchronize()
    assert torch.isnan(out).all()
    # and a good call right after is clean
    out = torch.zeros(c.nf, dtype=torch.float32, device=dev)
    assert _call(lsp, td, torch.from_numpy(c.X).to(dev), c.f0, c.df, c.nf, out, stream) == lsp.OK
    torch.cuda.synchronize()
    assert_parity(out.cpu().numpy(), oracle.periodogram(c.t, c.X, c.f0, c.df, c.nf), what="after NaN calls")


def test_noalloc_rejects_oversize_and_host_pointers(lsp):
    lib = lsp.load()
    dev = torch.device("cuda:0")
    t = torch.zeros(16, dtype=torch.float64, device=dev)
    out = torch.empty(4, dtype=torch.float32, device=dev)
    too_many = MAX_SAMPLES + 1
    st = lib.lsp_periodogram_noalloc(ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(t.data_ptr()), too_many,
                                     0.1, 0.1, 4, ctypes.c_void_p(out.data_ptr()), None)
    assert st == lsp.ERR_INVALID_ARG
    h = np.zeros(16)
    st = lib.lsp_periodogram_noalloc(ctypes.c_void_p(h.ctypes.data), ctypes.c_void_p(h.ctypes.data), 16,
                                     0.1, 0.1, 4, ctypes.c_void_p(out.data_ptr()), None)
    assert st == lsp.ERR_INVALID_ARG
