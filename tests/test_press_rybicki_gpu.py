"""GPU parity of the Press-Rybicki fast approximation (lsp_press_rybicki).

Against the FP64 numpy oracle of the same approximation (same macc, same FFT
grid): |dP| <= 1e-4 max P and relative error <= 1e-4 at the ten largest peaks
(the GPU computes the FFT in FP32).  Against the direct periodogram: exact up
to FP32 when every sample sits on a grid node, within the extirpolation error
otherwise.  FFT grids with even and odd log2 sizes; the full paper-shape
workload (382,003 samples, 1,528,064 bins, a 2^24-point FFT) on every bin.
"""
import numpy as np
import pytest

import oracle
from oracle import press_rybicki as pr
from tests.parity import assert_parity, assert_parity_with_degenerate_band

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


def _pr(ctx, t, X, f0, df, nf, macc):
    P = ctx.press_rybicki(_dev(t), _dev(X), f0, df, nf, macc=macc)
    ctx.sync(60.0)
    return P.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("macc", [4, 6, 2, 10])
def test_plain_1k_matches_the_oracle_approximation(ctx, macc):
    from paper_1007_1658_gb300 import synth
    c = synth.plain_1k()
    j0 = int(round(c.f0 / c.df))
    ref = pr.periodogram(c.t, c.X, j0, c.nf, c.df, macc)
    got = _pr(ctx, c.t, c.X, c.f0, c.df, c.nf, macc)
    assert_parity(got, ref, what="plain_1k press-rybicki macc=%d" % macc)


@pytest.mark.parametrize("n,nf,j0", [(2, 5, 1), (37, 100, 0), (1000, 2049, 3), (4099, 8193, 1), (300, 1, 57)])
def test_ragged_sizes_and_offsets(ctx, n, nf, j0):
    rng = np.random.default_rng(n + nf)
    t = np.sort(rng.uniform(0, 50.0, n))
    X = rng.normal(size=n) + np.sin(2 * np.pi * 0.9 * t)
    df = 1.0 / (4 * (t.max() - t.min()))
    for macc in (4, 6):  # even and odd log2 FFT sizes
        ref = pr.periodogram(t, X, j0, nf, df, macc)
        got = _pr(ctx, t, X, j0 * df, df, nf, macc)
        if n <= 2:
            # the same bound away from the degenerate-term band (here the band is
            # wider: the extirpolated tau sums carry the approximation's error)
            assert_parity_with_degenerate_band(got, ref, t, X, (j0 + np.arange(nf)) * df, rel=2.0 ** -10,
                                               kept_tol=1e-3, what="n=%d nf=%d j0=%d macc=%d" % (n, nf, j0, macc))
        else:
            assert_parity(got, ref, what="n=%d nf=%d j0=%d macc=%d" % (n, nf, j0, macc))


def test_exact_on_grid_nodes_and_close_to_the_direct_periodogram(ctx):
    rng = np.random.default_rng(1)
    n, df = 2000, 1.0 / 4000.0
    nf = 4 * n
    n_fft = pr.fft_size(nf, 4)
    idx = np.sort(rng.choice(np.arange(0, n_fft // 4), n, replace=False))
    t = 3.0 + idx / (df * n_fft)
    X = rng.normal(size=n) + np.sin(2 * np.pi * 0.3 * t)
    ref = oracle.periodogram(t, X, df, df, nf)
    assert_parity(_pr(ctx, t, X, df, df, nf, 4), ref, what="on grid")
    from paper_1007_1658_gb300 import synth
    c = synth.plain_1k()
    ref = oracle.periodogram(c.t, c.X, c.f0, c.df, c.nf)
    for macc, bound in ((4, 1e-3), (10, 2e-5)):
        err = np.max(np.abs(_pr(ctx, c.t, c.X, c.f0, c.df, c.nf, macc) - ref)) / ref.max()
        assert err <= bound, (macc, err)


def test_full_paper_shape_every_bin(ctx):
    """382,003 samples, 1,528,064 bins, a 2^24-point FFT: the GPU result
    against the FP64 oracle of the same approximation on every bin, and the
    approximation against the direct periodogram on sampled bins."""
    from paper_1007_1658_gb300 import synth
    c = synth.corot_382k()
    j0 = int(round(c.f0 / c.df))
    got = _pr(ctx, c.t, c.X, c.f0, c.df, c.nf, 4)
    ref = pr.periodogram(c.t, c.X, j0, c.nf, c.df, 4)
    assert_parity(got, ref, what="corot_382k press-rybicki")
    rng = np.random.default_rng(2)
    ks = np.unique(np.concatenate([rng.integers(0, c.nf, 64), np.argsort(-ref)[:8]]))
    exact = oracle.periodogram_at(c.t, c.X, c.f0 + ks * c.df)
    assert np.max(np.abs(got[ks] - exact)) <= 1e-3 * exact.max()


def test_host_pointers_and_errors(ctx, lsp):
    from paper_1007_1658_gb300 import synth
    c = synth.plain_1k()
    dev = _pr(ctx, c.t, c.X, c.f0, c.df, c.nf, 4)
    host = ctx.press_rybicki(c.t, c.X, c.f0, c.df, c.nf, macc=4)
    # FP64 atomics may add in another order: equal to FP32 rounding
    assert np.max(np.abs(dev - host)) <= 1e-6 * dev.max()
    for kw in (dict(f0=0.37 * c.df), dict(macc=5), dict(macc=18)):
        args = dict(f0=c.f0, macc=4)
        args.update(kw)
        with pytest.raises(lsp.LspError) as e:
            ctx.press_rybicki(c.t, c.X, args["f0"], c.df, c.nf, macc=args["macc"])
        assert e.value.status == lsp.ERR_INVALID_ARG
    with pytest.raises(lsp.LspError) as e:
        ctx.press_rybicki(c.t, np.full(c.t.size, 3.0), c.f0, c.df, c.nf)
    assert e.value.status == lsp.ERR_DEGENERATE
