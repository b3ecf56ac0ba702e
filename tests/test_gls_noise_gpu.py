"""lsp_batch_gls_noise: Monte-Carlo noise periodograms in the floating-mean
form.  Realization r of curve c is X = dy z with z the oracle's Philox N(0,1)
stream for (seed, c, r) (the GPU generator is pinned to it bit for bit
elsewhere); every (curve, realization) periodogram is compared with the FP64
oracle's floating-mean periodogram of that X at the parity tolerance
(|dP| <= 1e-4 max P), with and without errors.  The noise peaks at a fixed
frequency must follow the exact Beta(1, (N-3)/2) law, realization 0 must agree
with lsp_batch_gls on the same X, groups of realizations sharing a pass must
give the one-at-a-time results bit for bit (groups of 8 are checked against
the oracle), and the refusals are checked.
"""
import numpy as np
import pytest
from scipy import stats

import oracle
from tests.parity import assert_parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CANARY = np.float32(-7.25)


@pytest.fixture(scope="module")
def lsp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1007_1658_gb300 import build, lsp as L
    build.build()
    return L


def _batch(n_curves=6, seed=91):
    from paper_1007_1658_gb300 import synth
    b = synth.noise_batch(n_curves=n_curves, seed=seed, nt_min=40, nt_max=900, t_min=5.0, t_max=60.0)
    rng = np.random.default_rng(seed)
    dy = np.exp(rng.uniform(np.log(0.2), np.log(3.0), b.t.size))
    return b, dy


def _grid(f0, df, nf):
    return f0 + np.arange(int(nf), dtype=np.float64) * df


@pytest.mark.parametrize("weighted,n_real", [(True, 5), (False, 5), (True, 1)])
def test_every_realization_matches_the_oracle(lsp, weighted, n_real):
    """Five realizations run as a group of 4 and a group of 1; a single one
    runs the one-at-a-time kernel with its default strips of 16."""
    b, dy = _batch()
    d = dy if weighted else None
    seed = 20260
    P_off = np.zeros(b.n + 1, np.int64)
    P_off[1:] = np.cumsum(b.nf + 3)  # 3 slots of slack after each curve
    stride = int(P_off[-1])
    P = np.full(n_real * stride, CANARY, np.float32)
    mx = np.empty(n_real * b.n, np.float32)
    am = np.empty(n_real * b.n, np.int32)
    ctx = lsp.Context(0)
    ctx.batch_gls_noise(b.t_off, b.t, b.f0, b.df, b.nf, dy=d, seed=seed, n_real=n_real, P_out=P, P_off=P_off,
                        maxP=mx, argmax=am)
    ctx.close()
    for r in range(n_real):
        for c in range(b.n):
            s = slice(b.t_off[c], b.t_off[c + 1])
            z = oracle.noise(seed, c, r, b.t_off[c + 1] - b.t_off[c])
            X = z * dy[s] if weighted else z
            ref = oracle.gls_at(b.t[s], X, _grid(b.f0[c], b.df[c], b.nf[c]), dy[s] if weighted else None)
            base = r * stride + int(P_off[c])
            got = P[base:base + b.nf[c]].astype(np.float64)
            assert_parity(got, ref, what="curve %d realization %d" % (c, r))
            i = r * b.n + c
            assert mx[i] == P[base + am[i]] and mx[i] == P[base:base + b.nf[c]].max()
            assert np.all(P[base + b.nf[c]:r * stride + int(P_off[c + 1])] == CANARY)


def test_noise_peaks_follow_the_exact_beta_law(lsp):
    """Heteroscedastic Gaussian noise X = dy z on uneven times, weights 1/dy^2,
    the mean fitted: 2P/N at a fixed frequency is Beta(1, (N-3)/2) exactly,
    over 4000 realizations of one curve drawn on the device."""
    n, R = 25, 4000
    rng = np.random.default_rng(12)
    t = np.sort(rng.uniform(0, 3.0, n))
    dy = rng.uniform(0.2, 3.0, n)
    dy[::6] = 20.0
    nf = 3
    ctx = lsp.Context(0)
    P = np.empty(R * nf, np.float32)
    ctx.batch_gls_noise(np.array([0, n], np.int64), t, np.array([1.37]), np.array([1.0]), np.array([nf], np.int64),
                        dy=dy, seed=5, n_real=R, P_out=P, P_off=np.array([0, nf], np.int64))
    ctx.close()
    z = 2 * P.reshape(R, nf)[:, 0].astype(np.float64) / n
    assert stats.kstest(z, stats.beta(1, (n - 3) / 2).cdf).pvalue > 1e-3


def test_realization_zero_agrees_with_the_measured_batch(lsp):
    b, dy = _batch(n_curves=4, seed=17)
    seed = 99
    X = np.concatenate([oracle.noise(seed, c, 0, b.t_off[c + 1] - b.t_off[c]) for c in range(b.n)]) * dy
    P_off = np.zeros(b.n + 1, np.int64)
    P_off[1:] = np.cumsum(b.nf)
    Pn = np.empty(int(P_off[-1]) * 2, np.float32)
    Pm = np.empty(int(P_off[-1]), np.float32)
    ctx = lsp.Context(0)
    ctx.batch_gls_noise(b.t_off, b.t, b.f0, b.df, b.nf, dy=dy, seed=seed, n_real=2, P_out=Pn, P_off=P_off,
                        maxP=np.empty(2 * b.n, np.float32), argmax=np.empty(2 * b.n, np.int32))
    ctx.batch_gls(b.t_off, b.t, X, b.f0, b.df, b.nf, dy=dy, P_out=Pm, P_off=P_off,
                  maxP=np.empty(b.n, np.float32), argmax=np.empty(b.n, np.int32))
    # the same X normalized by two reductions of different shape: FP32 rounding apart
    assert np.max(np.abs(Pn[:Pm.size] - Pm)) <= 1e-5 * float(Pm.max())
    ctx.close()


def test_refusals(lsp):
    b, dy = _batch(n_curves=3, seed=5)
    ctx = lsp.Context(0)
    with pytest.raises(lsp.LspError) as e:
        ctx.batch_gls_noise(b.t_off, b.t, b.f0, b.df, b.nf, dy=dy, n_real=0)
    assert e.value.status == lsp.ERR_INVALID_ARG
    ctx.set_options(sincos_mode=lsp.SINCOS_RECUR3)  # the scalar strip has no noise form
    with pytest.raises(lsp.LspError) as e:
        ctx.batch_gls_noise(b.t_off, b.t, b.f0, b.df, b.nf, dy=dy, n_real=2)
    assert e.value.status == lsp.ERR_UNSUPPORTED
    ctx.set_options(sincos_mode=lsp.SINCOS_AUTO)
    bad = dy.copy()
    bad[2] = -1.0
    with pytest.raises(lsp.LspError) as e:
        ctx.batch_gls_noise(b.t_off, b.t, b.f0, b.df, b.nf, dy=bad, n_real=2)
    assert e.value.status == lsp.ERR_INVALID_ARG
    # the context still computes afterwards
    mx, am = ctx.batch_gls_noise(b.t_off, b.t, b.f0, b.df, b.nf, dy=dy, n_real=2)
    assert np.all(np.isfinite(mx)) and np.all(am >= 0)
    ctx.close()


@pytest.mark.parametrize("R", [2, 4])
def test_realization_groups_match_one_at_a_time(lsp, R):
    """Groups of R realizations share the phase, the recurrence and the
    pattern sums; every (frequency, realization) must come out bit for bit as
    the one-at-a-time kernel with the same strip length (8) computes it, with a
    partial last group."""
    b, dy = _batch(n_curves=5, seed=61)
    n_real = 2 * R + 1
    P_off = np.zeros(b.n + 1, np.int64)
    P_off[1:] = np.cumsum(b.nf)
    outs = []
    for rhs in (1, R):
        ctx = lsp.Context(0, batch_rhs=rhs, freqs_per_thread=8)
        P = np.empty(n_real * int(P_off[-1]), np.float32)
        mx = np.empty(n_real * b.n, np.float32)
        am = np.empty(n_real * b.n, np.int32)
        ctx.batch_gls_noise(b.t_off, b.t, b.f0, b.df, b.nf, dy=dy, seed=8, n_real=n_real, P_out=P, P_off=P_off,
                            maxP=mx, argmax=am)
        outs.append((P, mx, am))
        ctx.close()
    assert np.array_equal(outs[0][0].view(np.uint32), outs[1][0].view(np.uint32))
    assert np.array_equal(outs[0][1].view(np.uint32), outs[1][1].view(np.uint32))
    assert np.array_equal(outs[0][2], outs[1][2])


def test_groups_of_eight_match_the_oracle(lsp):
    b, dy = _batch(n_curves=4, seed=71)
    n_real, seed = 11, 4242
    P_off = np.zeros(b.n + 1, np.int64)
    P_off[1:] = np.cumsum(b.nf)
    stride = int(P_off[-1])
    P = np.empty(n_real * stride, np.float32)
    ctx = lsp.Context(0, batch_rhs=8)
    ctx.batch_gls_noise(b.t_off, b.t, b.f0, b.df, b.nf, dy=dy, seed=seed, n_real=n_real, P_out=P, P_off=P_off,
                        maxP=np.empty(n_real * b.n, np.float32), argmax=np.empty(n_real * b.n, np.int32))
    ctx.close()
    for r in (0, 5, 7, 8, 10):
        for c in range(b.n):
            s = slice(b.t_off[c], b.t_off[c + 1])
            X = oracle.noise(seed, c, r, b.t_off[c + 1] - b.t_off[c]) * dy[s]
            ref = oracle.gls_at(b.t[s], X, _grid(b.f0[c], b.df[c], b.nf[c]), dy[s])
            base = r * stride + int(P_off[c])
            assert_parity(P[base:base + b.nf[c]].astype(np.float64), ref, what="curve %d realization %d" % (c, r))
