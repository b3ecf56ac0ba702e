"""GPU parity of the floating-mean (generalized, weighted) periodogram
(lsp_periodogram_gls) against the FP64 oracle, element by element.

Tolerance as for the classic periodogram: |dP| <= 1e-4 max P over the grid and
relative error <= 1e-4 at the ten largest peaks.  Small cases on the whole
grid (several strips, tiles and chunks, ragged tails); the full-size gapped
workload with per-sample errors in the benchmark's launch configuration on
sampled bins.  Degenerate frequencies (f = 0, Nyquist of an even grid,
two-phase sampling) and the exact Beta(1, (N-3)/2) noise law are checked too.
"""
import numpy as np
import pytest
from scipy import stats

import oracle
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


@pytest.fixture(scope="module")
def ctx(lsp):
    c = lsp.Context(0)
    yield c
    c.close()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _gls(ctx, t, X, f0, df, nf, dy=None, **opts):
    ctx.set_options(**opts)
    P = ctx.periodogram_gls(_dev(t), _dev(X), f0, df, nf, dy=None if dy is None else _dev(dy))
    ctx.sync(60.0)
    return P.cpu().numpy().astype(np.float64)


def _grid(f0, df, nf):
    return f0 + np.arange(int(nf), dtype=np.float64) * df


OPTS = [dict(sincos_mode=3), dict(sincos_mode=2), dict(sincos_mode=1), dict(sincos_mode=4),
        dict(sincos_mode=3, freqs_per_thread=8), dict(sincos_mode=4, freqs_per_thread=8),
        dict(sincos_mode=4, freqs_per_thread=12),
        dict(sincos_mode=1, freqs_per_thread=16), dict(sincos_mode=3, split=1), dict(sincos_mode=3, split=5)]


@pytest.mark.parametrize("weighted", [True, False])
@pytest.mark.parametrize("opts", OPTS)
def test_plain_1k_with_errors_full_grid(ctx, opts, weighted):
    from paper_1007_1658_gb300 import synth
    c = synth.with_errors(synth.plain_1k)
    dy = c.dy if weighted else None
    ref = oracle.gls_at(c.t, c.X, _grid(c.f0, c.df, c.nf), dy)
    got = _gls(ctx, c.t, c.X, c.f0, c.df, c.nf, dy, **opts)
    assert_parity(got, ref, what="plain_1k gls %s weighted=%s" % (opts, weighted))
    assert int(np.argmax(got)) == int(np.argmax(ref))


@pytest.mark.parametrize("n,nf", [(3, 1), (5, 64), (255, 511), (257, 513), (1000, 2049), (4099, 2048),
                                  (1023, 4097)])
@pytest.mark.parametrize("mode", [1, 3, 4])
def test_ragged_sizes(ctx, n, nf, mode):
    rng = np.random.default_rng(n * 31 + nf)
    t = np.sort(rng.uniform(0, 37.0, n))
    dy = rng.uniform(0.2, 2.0, n)
    X = 3.0 + dy * rng.normal(size=n) + 0.8 * np.sin(2 * np.pi * 1.7 * t)
    df = 1.0 / (4 * (t.max() - t.min()))
    ref = oracle.gls_at(t, X, _grid(df, df, nf), dy)
    got = _gls(ctx, t, X, df, df, nf, dy, sincos_mode=mode)
    assert_parity(got, ref, what="ragged n=%d nf=%d mode=%d" % (n, nf, mode))


def test_full_size_gapped_100k_with_errors_sampled(ctx):
    """The benchmark's floating-mean workload (gapped_100k with per-sample
    errors, 100,000 x 200,000, default launch shape) on sampled bins."""
    from paper_1007_1658_gb300 import synth
    c = synth.with_errors(synth.gapped_100k)
    got = _gls(ctx, c.t, c.X, c.f0, c.df, c.nf, c.dy, sincos_mode=0)
    rng = np.random.default_rng(5)
    idx = set(rng.choice(c.nf, 200, replace=False).tolist())
    for f in c.signal_freqs:
        k = int(round((f - c.f0) / c.df))
        idx.update(range(max(0, k - 3), min(c.nf, k + 4)))
    top = np.argsort(-got)[:20]
    idx.update(top.tolist())
    idx = np.array(sorted(idx))
    ref = oracle.gls_at(c.t, c.X, c.f0 + idx * c.df, c.dy)
    scale = max(ref.max(), got.max())
    assert np.max(np.abs(got[idx] - ref)) <= 1e-4 * scale
    pk = np.argsort(-ref)[:5]
    assert np.max(np.abs(got[idx[pk]] - ref[pk]) / ref[pk]) <= 1e-4


@pytest.mark.parametrize("F", [8, 16])
def test_packed_recurrence_is_bit_identical_to_scalar(ctx, F):
    from paper_1007_1658_gb300 import synth
    c = synth.with_errors(synth.gapped_100k)
    outs = [_gls(ctx, c.t, c.X, c.f0, c.df, 30_000, c.dy, sincos_mode=m, freqs_per_thread=F, split=sp)
            for m in (3, 4) for sp in (1, 5)]
    assert np.array_equal(outs[0], outs[2]) and np.array_equal(outs[1], outs[3])


def test_even_grid_agrees_with_classic_and_handles_degenerate_bins(ctx):
    # equal weights, t_j = j dt: at Fourier frequencies the fitted offset is the
    # mean, so both periodograms agree; f = 0 gives 0; Nyquist keeps the cosine
    N, dt = 256, 0.25
    rng = np.random.default_rng(3)
    t = 100.0 + dt * np.arange(N)
    X = 5.0 + rng.normal(size=N) + np.cos(2 * np.pi * 0.8 * t)
    df = 1.0 / (N * dt)
    nf = N // 2 + 1  # f = 0 .. Nyquist
    got = _gls(ctx, t, X, 0.0, df, nf, sincos_mode=3)
    ref = oracle.gls_at(t, X, _grid(0.0, df, nf))
    assert_parity(got, ref, what="even grid")
    assert got[0] == 0.0
    ctx.set_options(sincos_mode=3)
    cls = ctx.periodogram(_dev(t), _dev(X), df, df, nf - 1)
    ctx.sync(60.0)
    cls = cls.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(cls - got[1:])) <= 1e-4 * got.max()


def test_two_phase_sampling_rank_one(ctx):
    rng = np.random.default_rng(21)
    t = np.sort(rng.integers(0, 400, 300) + 0.3 * rng.integers(0, 2, 300)).astype(np.float64)
    dy = rng.uniform(0.5, 1.5, t.size)
    X = rng.normal(size=t.size) + 0.8 * (np.abs(t - np.round(t)) > 0.1)
    got = _gls(ctx, t, X, 1.0, 0.5, 3, dy, sincos_mode=3)  # f = 1, 1.5, 2: rank 1 at 1 and 2
    for k, f in enumerate((1.0, 1.5, 2.0)):
        ref = oracle.gls_lsq(t, X, f, dy)
        assert abs(got[k] - ref) <= 1e-4 * max(ref, 1.0), (f, got[k], ref)


def test_host_and_device_pointers_agree(ctx):
    from paper_1007_1658_gb300 import synth
    c = synth.with_errors(synth.plain_1k)
    ctx.set_options(sincos_mode=3)
    dev = ctx.periodogram_gls(_dev(c.t), _dev(c.X), c.f0, c.df, c.nf, dy=_dev(c.dy))
    ctx.sync(60.0)
    host = ctx.periodogram_gls(c.t, c.X, c.f0, c.df, c.nf, dy=c.dy)
    assert np.array_equal(dev.cpu().numpy(), host)


def test_errors(ctx, lsp):
    t = np.linspace(0.0, 10.0, 50)
    X = np.sin(t)
    dy = np.ones(50)
    bad = dy.copy()
    bad[7] = 0.0
    ctx.set_options(sincos_mode=3)
    with pytest.raises(lsp.LspError) as e:
        ctx.periodogram_gls(t, X, 0.1, 0.1, 10, dy=bad)
    assert e.value.status == lsp.ERR_INVALID_ARG
    with pytest.raises(lsp.LspError) as e:
        ctx.periodogram_gls(t, np.full(50, 2.0), 0.1, 0.1, 10, dy=dy)
    assert e.value.status == lsp.ERR_DEGENERATE
    with pytest.raises(lsp.LspError) as e:
        ctx.periodogram_gls(t[:2], X[:2], 0.1, 0.1, 10)
    assert e.value.status == lsp.ERR_INVALID_ARG
    ctx.set_options(phase_mode=1)
    with pytest.raises(lsp.LspError) as e:
        ctx.periodogram_gls(t, X, 0.1, 0.1, 10)
    assert e.value.status == lsp.ERR_UNSUPPORTED
    ctx.set_options(sincos_mode=3)
    # the context is still usable
    P = ctx.periodogram_gls(t, X, 0.1, 0.1, 10, dy=dy)
    assert np.all(np.isfinite(P))


def test_noise_power_follows_the_exact_beta_law(ctx):
    """Gaussian noise with sigma_j = dy_j on uneven times, weights 1/dy^2 and a
    fitted mean: 2P/N at a fixed frequency is Beta(1, (N-3)/2) exactly."""
    n, R = 25, 2000
    rng = np.random.default_rng(12)
    t = np.sort(rng.uniform(0, 3.0, n))
    dy = rng.uniform(0.2, 3.0, n)
    dy[::6] = 20.0
    ctx.set_options(sincos_mode=3)
    z = np.empty(R)
    for r in range(R):
        X = 4.0 + dy * rng.normal(size=n)
        z[r] = 2 * float(ctx.periodogram_gls(t, X, 1.37, 1.0, 1, dy=dy)[0]) / n
    assert stats.kstest(z, stats.beta(1, (n - 3) / 2).cdf).pvalue > 1e-3


def _err_batch(n_curves=9, seed=41):
    from paper_1007_1658_gb300 import synth
    b = synth.noise_batch(n_curves=n_curves, seed=seed, nt_min=30, nt_max=1500, t_min=5.0, t_max=60.0)
    rng = np.random.default_rng(seed)
    dy = rng.uniform(0.3, 3.0, b.t.size)
    X = 7.0 + dy * rng.normal(size=b.t.size)
    for c in range(b.n):  # a line in every curve
        s = slice(b.t_off[c], b.t_off[c + 1])
        X[s] += 1.5 * np.sin(2 * np.pi * (0.4 + 0.07 * c) * b.t[s])
    return b, X, dy


@pytest.mark.parametrize("weighted", [True, False])
def test_batch_matches_the_oracle_curve_by_curve(ctx, lsp, weighted):
    b, X, dy = _err_batch()
    d = dy if weighted else None
    P_off = np.zeros(b.n + 1, np.int64)
    P_off[1:] = np.cumsum(b.nf)
    P = np.empty(int(P_off[-1]), np.float32)
    mx = np.empty(b.n, np.float32)
    am = np.empty(b.n, np.int32)
    ctx.set_options()
    ctx.batch_gls(b.t_off, b.t, X, b.f0, b.df, b.nf, dy=d, P_out=P, P_off=P_off, maxP=mx, argmax=am)
    for c in range(b.n):
        s = slice(b.t_off[c], b.t_off[c + 1])
        ref = oracle.gls_at(b.t[s], X[s], _grid(b.f0[c], b.df[c], b.nf[c]), None if d is None else d[s])
        got = P[P_off[c]:P_off[c + 1]].astype(np.float64)
        assert_parity(got, ref, what="batch curve %d" % c)
        assert mx[c] == P[P_off[c] + am[c]] and mx[c] == P[P_off[c]:P_off[c + 1]].max()
    # the single-curve entry point gives the same values
    c = 3
    s = slice(b.t_off[c], b.t_off[c + 1])
    one = ctx.periodogram_gls(b.t[s], X[s], b.f0[c], b.df[c], b.nf[c], dy=None if d is None else d[s])
    assert np.max(np.abs(one - P[P_off[c]:P_off[c + 1]])) <= 1e-5 * one.max()


def test_batch_device_pointers_and_errors(ctx, lsp):
    b, X, dy = _err_batch(n_curves=5, seed=7)
    mx, am = ctx.batch_gls(torch.from_numpy(b.t_off).cuda(), _dev(b.t), _dev(X), _dev(b.f0), _dev(b.df),
                           torch.from_numpy(b.nf).cuda(), dy=_dev(dy))
    ctx.sync(30.0)
    mh, ah = ctx.batch_gls(b.t_off, b.t, X, b.f0, b.df, b.nf, dy=dy)
    assert np.array_equal(mx.cpu().numpy(), mh) and np.array_equal(am.cpu().numpy(), ah)
    bad = dy.copy()
    bad[3] = -1.0
    with pytest.raises(lsp.LspError) as e:
        ctx.batch_gls(b.t_off, b.t, X, b.f0, b.df, b.nf, dy=bad)
    assert e.value.status == lsp.ERR_INVALID_ARG
    off2 = b.t_off.copy()
    off2[1] = 2  # a 2-sample curve
    with pytest.raises(lsp.LspError) as e:
        ctx.batch_gls(off2, b.t, X, b.f0, b.df, b.nf, dy=dy)
    assert e.value.status == lsp.ERR_INVALID_ARG
    # the plain batch still works on the same context afterwards
    m2, a2 = ctx.batch(b.t_off, b.t, b.f0, b.df, b.nf, X=X)
    assert np.all(np.isfinite(m2)) and np.all(a2 >= 0)
