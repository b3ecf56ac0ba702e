"""Mixed host/device pointers, user streams and small edge grids across the
entry points (each argument's side is detected on its own)."""
import numpy as np
import pytest

import oracle
from oracle import press_rybicki as pr
from tests.parity import assert_parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lsp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1007_1658_gb300 import build, lsp as L
    build.build()
    return L


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def test_mixed_pointer_sides_agree(lsp):
    from paper_1007_1658_gb300 import synth
    c = synth.with_errors(synth.plain_1k)
    with lsp.Context(0) as ctx:
        ref = ctx.periodogram(c.t, c.X, c.f0, c.df, c.nf)
        a = np.empty(c.nf, np.float32)
        ctx.periodogram(_dev(c.t), c.X, c.f0, c.df, c.nf, out=a)            # t device, X host, P host
        out = torch.empty(c.nf, dtype=torch.float32, device="cuda")
        ctx.periodogram(c.t, _dev(c.X), c.f0, c.df, c.nf, out=out)          # t host, X device, P device
        ctx.sync(30.0)
        assert np.array_equal(ref, a) and np.array_equal(ref, out.cpu().numpy())
        g_ref = ctx.periodogram_gls(c.t, c.X, c.f0, c.df, c.nf, dy=c.dy)
        g = ctx.periodogram_gls(_dev(c.t), _dev(c.X), c.f0, c.df, c.nf, dy=c.dy)  # dy host, rest device
        ctx.sync(30.0)
        assert np.array_equal(g_ref, g.cpu().numpy())
        p_ref = ctx.press_rybicki(c.t, c.X, c.f0, c.df, c.nf)
        p = np.empty(c.nf, np.float32)
        ctx.press_rybicki(_dev(c.t), c.X, c.f0, c.df, c.nf, out=p)
        assert np.max(np.abs(p_ref - p)) <= 1e-6 * p_ref.max()


def test_user_stream_and_asynchronous_results(lsp):
    from paper_1007_1658_gb300 import synth
    c = synth.plain_1k()
    s = torch.cuda.Stream()
    with lsp.Context(0, stream=s) as ctx:
        t, X = _dev(c.t), _dev(c.X)
        P = torch.empty(c.nf, dtype=torch.float32, device="cuda")
        G = torch.empty(c.nf, dtype=torch.float32, device="cuda")
        Q = torch.empty(c.nf, dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            ctx.periodogram(t, X, c.f0, c.df, c.nf, out=P)
            ctx.periodogram_gls(t, X, c.f0, c.df, c.nf, out=G)
            ctx.press_rybicki(t, X, c.f0, c.df, c.nf, out=Q)
        s.synchronize()
        ref = oracle.periodogram(c.t, c.X, c.f0, c.df, c.nf)
        assert_parity(P.cpu().numpy().astype(np.float64), ref, what="user stream")
        gref = oracle.gls_at(c.t, c.X, c.f0 + np.arange(c.nf) * c.df)
        assert_parity(G.cpu().numpy().astype(np.float64), gref, what="user stream gls")
        pref = pr.periodogram(c.t, c.X, 1, c.nf, c.df, 4)
        assert_parity(Q.cpu().numpy().astype(np.float64), pref, what="user stream press-rybicki")


def test_small_edge_grids(lsp):
    rng = np.random.default_rng(4)
    t = np.sort(rng.uniform(0, 20.0, 300))
    X = rng.normal(size=300) + np.cos(2 * np.pi * 0.6 * t)
    df = 1.0 / 80.0
    with lsp.Context(0) as ctx:
        # Press-Rybicki from f = 0 with a single bin, and from f = 0 on a short grid
        p1 = ctx.press_rybicki(t, X, 0.0, df, 1)
        assert p1.shape == (1,) and abs(float(p1[0])) <= 1e-3 * t.size
        p = ctx.press_rybicki(t, X, 0.0, df, 97, macc=6)
        ref = pr.periodogram(t, X, 0, 97, df, 6)
        assert np.max(np.abs(p[1:] - ref[1:])) <= 1e-4 * ref.max()
        # one-bin exact and floating-mean periodograms at the injected line
        P = ctx.periodogram(t, X, 0.6, df, 1)
        assert abs(P[0] - oracle.periodogram_at(t, X, [0.6])[0]) <= 1e-4 * t.size
        G = ctx.periodogram_gls(t, X, 0.6, df, 1)
        assert abs(G[0] - oracle.gls_at(t, X, [0.6])[0]) <= 1e-4 * t.size


def test_batch_outputs_on_mixed_sides(lsp):
    from paper_1007_1658_gb300 import synth
    b = synth.noise_batch(n_curves=6, seed=9, nt_min=50, nt_max=600, t_min=5.0, t_max=50.0)
    P_off = np.zeros(b.n + 1, np.int64)
    P_off[1:] = np.cumsum(b.nf)
    with lsp.Context(0) as ctx:
        P_h = np.empty(int(P_off[-1]), np.float32)
        m_d = torch.empty(b.n, dtype=torch.float32, device="cuda")
        a_d = torch.empty(b.n, dtype=torch.int32, device="cuda")
        ctx.batch(b.t_off, b.t, b.f0, b.df, b.nf, seed=3, P_out=P_h, P_off=P_off, maxP=m_d, argmax=a_d)
        ctx.sync(30.0)
        m = m_d.cpu().numpy()
        a = a_d.cpu().numpy()
        for c in range(b.n):
            seg = P_h[P_off[c]:P_off[c + 1]]
            assert m[c] == seg.max() and seg[a[c]] == m[c]
