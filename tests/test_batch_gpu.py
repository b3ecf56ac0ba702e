"""GPU parity of the batched Monte-Carlo path (lsp_batch) and of its noise (lsp_noise).

Noise: the device's FP32 Philox-4x32-10 + Box-Muller values against the
oracle's FP64 evaluation of the same counter-based generator (same integers,
so the normals agree to FP32 rounding).  Periodograms: every batch result
against the FP64 oracle evaluated on the oracle's own noise, with the parity
tolerance of the single-curve tests (|dP| <= 1e-4 max P per periodogram);
argmax must hit a bin whose oracle value is within that tolerance of the
oracle's maximum.  A statistical pin checks the whole engine against the beta
law behind Eq. 3.
"""
import numpy as np
import pytest
from scipy import stats

import oracle
from tests.parity import TOL_ABS, assert_parity, assert_parity_with_degenerate_band

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


def _dev(a, dtype=None):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


@pytest.mark.parametrize("seed,curve,real,n", [(0, 0, 0, 1001), (2024, 3, 7, 4099), (2**40 + 5, 4095, 1, 17)])
def test_noise_matches_oracle_generator(ctx, seed, curve, real, n):
    got = ctx.noise(seed, curve, real, n).astype(np.float64)
    ref = oracle.noise(seed, curve, real, n)
    assert np.all(np.abs(got - ref) <= 4e-6 * np.maximum(1.0, np.abs(ref)))
    d = torch.empty(n, dtype=torch.float32, device="cuda")
    ctx.noise(seed, curve, real, n, out=d)
    ctx.sync(30.0)
    assert np.array_equal(d.cpu().numpy().astype(np.float64), got)


def _small_batch(n_curves=12, seed=5):
    from paper_1007_1658_gb300 import synth
    return synth.noise_batch(n_curves=n_curves, seed=seed, nt_min=40, nt_max=900, t_min=5.0, t_max=80.0)


def _oracle_noise_curve(b, seed, c, r):
    t = b.curve_t(c)
    X = oracle.noise(seed, c, r, t.size)
    return t, X


@pytest.mark.parametrize("mode,n_real,rhs", [(4, 3, 0), (3, 3, 0), (2, 3, 0), (1, 3, 0), (4, 19, 4), (3, 19, 4),
                                             (2, 19, 4), (1, 19, 4), (0, 13, 0), (0, 35, 0)])
def test_noise_batch_matches_oracle(ctx, lsp, mode, n_real, rhs):
    """Every (curve, realization) periodogram of a noise batch against the
    oracle on the same Philox noise.  n_real = 3 runs groups of 2 realizations
    that accumulate their own CC and CS; n_real = 19 at batch_rhs 4 runs five
    groups of 4 (the last one partial) that take CC and CS from the window
    pass; under the automatic mode (packed strips) n_real = 13 runs groups of
    8 with their own CC and CS and n_real = 35 groups of 8 that read the
    window pass, the last group partial in both."""
    b = _small_batch()
    seed = 99
    ctx.set_options(sincos_mode=mode, batch_rhs=rhs)
    P_off = np.zeros(b.n + 1, np.int64)
    P_off[1:] = np.cumsum(b.nf)
    P = torch.empty(n_real * int(P_off[-1]), dtype=torch.float32, device="cuda")
    maxP, argmax = ctx.batch(_dev(b.t_off), _dev(b.t), _dev(b.f0), _dev(b.df), _dev(b.nf), seed=seed,
                             n_real=n_real, P_out=P, P_off=_dev(P_off),
                             maxP=torch.empty(n_real * b.n, device="cuda"),
                             argmax=torch.empty(n_real * b.n, dtype=torch.int32, device="cuda"))
    ctx.sync(60.0)
    P = P.cpu().numpy().astype(np.float64)
    maxP = maxP.cpu().numpy()
    argmax = argmax.cpu().numpy()
    for r in range(n_real):
        for c in range(b.n):
            t, X = _oracle_noise_curve(b, seed, c, r)
            ref = oracle.periodogram(t, X, b.f0[c], b.df[c], b.nf[c])
            got = P[r * P_off[-1] + P_off[c]: r * P_off[-1] + P_off[c] + b.nf[c]]
            scale = ref.max()
            assert np.max(np.abs(got - ref)) <= TOL_ABS * scale, (r, c)
            i = r * b.n + c
            assert abs(maxP[i] - scale) <= TOL_ABS * scale
            assert 0 <= argmax[i] < b.nf[c] and ref[argmax[i]] >= scale * (1 - 2 * TOL_ABS)
            assert maxP[i] == np.float32(got[argmax[i]])


def test_measured_batch_host_and_device_paths(ctx, lsp):
    b = _small_batch(n_curves=7, seed=8)
    rng = np.random.default_rng(3)
    X = rng.normal(size=b.t.size) + 3.0
    for c in range(b.n):  # a line in every curve
        s = slice(b.t_off[c], b.t_off[c + 1])
        X[s] += 2.0 * np.sin(2 * np.pi * (0.3 + 0.05 * c) * b.t[s])
    ctx.set_options(sincos_mode=3)
    maxP_d, arg_d = ctx.batch(_dev(b.t_off), _dev(b.t), _dev(b.f0), _dev(b.df), _dev(b.nf), X=_dev(X))
    ctx.sync(60.0)
    maxP_h, arg_h = ctx.batch(b.t_off, b.t, b.f0, b.df, b.nf, X=X)  # numpy in and out
    assert np.array_equal(maxP_d.cpu().numpy(), maxP_h) and np.array_equal(arg_d.cpu().numpy(), arg_h)
    for c in range(b.n):
        s = slice(b.t_off[c], b.t_off[c + 1])
        ref = oracle.periodogram(b.t[s], X[s], b.f0[c], b.df[c], b.nf[c])
        assert abs(maxP_h[c] - ref.max()) <= TOL_ABS * ref.max()
        assert ref[arg_h[c]] >= ref.max() * (1 - 2 * TOL_ABS)


def test_graph_replay_is_deterministic_and_seeded(ctx):
    b = _small_batch(n_curves=20, seed=11)
    args = (_dev(b.t_off), _dev(b.t), _dev(b.f0), _dev(b.df), _dev(b.nf))
    ctx.set_options(sincos_mode=3)
    out = [torch.empty(2 * b.n, device="cuda") for _ in range(3)]
    arg = [torch.empty(2 * b.n, dtype=torch.int32, device="cuda") for _ in range(3)]
    for i, s in enumerate((1, 1, 2)):
        ctx.batch(*args, seed=s, n_real=2, maxP=out[i], argmax=arg[i])
    ctx.sync(60.0)
    assert torch.equal(out[0], out[1]) and torch.equal(arg[0], arg[1])
    assert not torch.equal(out[0], out[2])
    # realization 1 of seed 1 is its own stream, not a copy of realization 0
    assert not torch.equal(out[0][:b.n], out[0][b.n:])


def test_edge_curves(ctx, lsp):
    # a 2-sample curve, a curve with no frequencies, and a 3-sample curve
    t = np.array([0.0, 1.0, 0.0, 0.5, 2.0, 0.0, 0.3, 0.9], np.float64)
    off = np.array([0, 2, 5, 8], np.int64)
    X = np.array([1.0, -1.0, 0.2, 0.9, -1.3, 1.0, 2.0, 0.5])
    f0 = np.array([0.1, 0.1, 0.05])
    df = np.array([0.1, 0.1, 0.05])
    nf = np.array([5, 0, 9], np.int64)
    P_off = np.array([0, 5, 5, 14], np.int64)
    P = np.full(14, -1.0, np.float32)
    maxP, arg = ctx.batch(off, t, f0, df, nf, X=X, P_out=P, P_off=P_off,
                          maxP=np.empty(3, np.float32), argmax=np.empty(3, np.int32))
    assert maxP[1] == 0.0 and arg[1] == -1
    for c in (0, 2):
        s = slice(off[c], off[c + 1])
        fr = f0[c] + np.arange(nf[c]) * df[c]
        ref = oracle.periodogram(t[s], X[s], f0[c], df[c], nf[c])
        got = P[P_off[c]:P_off[c] + nf[c]].astype(np.float64)
        assert_parity_with_degenerate_band(got, ref, t[s], X[s], fr, what="curve %d" % c)
        assert maxP[c] == got.max() and got[arg[c]] == got.max()
    with pytest.raises(lsp.LspError) as e:
        ctx.batch(off, t, f0, df, nf, X=np.array([1.0, 1.0, 0.2, 0.9, -1.3, 1.0, 2.0, 0.5]))
        ctx.sync(10.0)
    assert e.value.status == lsp.ERR_DEGENERATE
    with pytest.raises(lsp.LspError) as e:
        ctx.batch(np.array([0, 1], np.int64), t[:1], f0[:1], df[:1], nf[:1], X=X[:1])
    assert e.value.status == lsp.ERR_INVALID_ARG
    with pytest.raises(lsp.LspError) as e:
        ctx.batch(off, t, f0, df, nf, X=X, n_real=2)
    assert e.value.status == lsp.ERR_INVALID_ARG


def test_noise_periodograms_follow_the_beta_law(ctx):
    """Whole-engine statistical pin: even sampling, one Fourier frequency, many
    noise realizations through lsp_batch -> 2P/N ~ Beta(1, (N-3)/2) (Eq. 3's law)."""
    N, m, R = 48, 5, 4000
    t = np.arange(N, dtype=np.float64)
    off = np.array([0, N], np.int64)
    P_off = np.array([0, 1], np.int64)
    P = np.empty(R, np.float32)
    ctx.set_options(sincos_mode=3)
    ctx.batch(off, t, np.array([m / N]), np.array([1.0 / N]), np.array([1], np.int64), seed=7, n_real=R,
              P_out=P, P_off=P_off)
    z = 2 * P.astype(np.float64) / N
    assert stats.kstest(z, stats.beta(1, (N - 3) / 2).cdf).pvalue > 1e-3


@pytest.mark.parametrize("packed", [False, True])
@pytest.mark.parametrize("groups", [1, 4])
@pytest.mark.parametrize("R,F", [(2, 8), (2, 16), (4, 8), (4, 12), (8, 4), (8, 8)])
def test_multi_rhs_equals_one_realization_at_a_time(lsp, R, F, groups, packed):
    """Groups of R realizations share the phase, the recurrence and CC/CS; each
    (frequency, realization) must come out bit for bit as the one-at-a-time
    kernel with the same strip length computes it (here with a partial last
    group).  With one full group per pattern the groups accumulate CC and CS
    themselves; with four or more they read them from the window pass, which
    runs strips of the same length, and in the packed mode run the packed
    strip (the (cos, sin) pair in the two FFMA2 lanes, signs folded into the
    sums).  With strips longer than 8 the one-at-a-time kernel runs the
    frequencies after a curve's last full block as 8-frequency tail strips, so
    there the comparison is to FP32 rounding instead."""
    if F <= 8:
        b = _small_batch(n_curves=9, seed=31)
    else:  # curves long enough for several full blocks of the longer strips
        from paper_1007_1658_gb300 import synth
        b = synth.noise_batch(n_curves=6, seed=31, nt_min=1500, nt_max=5000, t_min=5.0, t_max=80.0)
    n_real = groups * R + R // 2 + 1
    P_off = np.zeros(b.n + 1, np.int64)
    P_off[1:] = np.cumsum(b.nf)
    outs = []
    for rhs in (1, R):
        mode = 4 if packed and rhs > 1 else 3
        ctx = lsp.Context(0, sincos_mode=mode, freqs_per_thread=F, batch_rhs=rhs)
        P = np.empty(n_real * int(P_off[-1]), np.float32)
        mx = np.empty(n_real * b.n, np.float32)
        am = np.empty(n_real * b.n, np.int32)
        ctx.batch(b.t_off, b.t, b.f0, b.df, b.nf, seed=77, n_real=n_real, P_out=P, P_off=P_off, maxP=mx, argmax=am)
        outs.append((P, mx, am))
        ctx.close()
    if F <= 8:
        assert np.array_equal(outs[0][0], outs[1][0])
        assert np.array_equal(outs[0][1], outs[1][1]) and np.array_equal(outs[0][2], outs[1][2])
        return
    block = 32 * F  # frequencies per block of one-warp CTAs
    for r in range(n_real):
        for c in range(b.n):
            base = r * int(P_off[-1]) + int(P_off[c])
            full = (int(b.nf[c]) // block) * block
            a, m = outs[0][0][base:base + b.nf[c]], outs[1][0][base:base + b.nf[c]]
            assert np.array_equal(a[:full], m[:full]), (r, c)
            assert np.max(np.abs(a[full:] - m[full:]), initial=0.0) <= 1e-5 * max(1.0, float(m.max())), (r, c)


def test_full_noise_batch_sampled_curves(ctx):
    """The benchmark's Monte-Carlo batch at full size (4096 noise curves, N_t
    log-uniform in [200, 20000], N_f = 2 N_t, seed 1234, one graph launch):
    ten curves across the size range against the oracle's periodogram of
    the oracle's own noise."""
    from paper_1007_1658_gb300 import synth
    b = synth.noise_batch(n_curves=4096)
    seed = 1234
    ctx.set_options()
    P_off = np.zeros(b.n + 1, np.int64)
    P_off[1:] = np.cumsum(b.nf)
    P = torch.empty(int(P_off[-1]), dtype=torch.float32, device="cuda")
    maxP, argmax = ctx.batch(_dev(b.t_off), _dev(b.t), _dev(b.f0), _dev(b.df), _dev(b.nf), seed=seed,
                             P_out=P, P_off=_dev(P_off), maxP=torch.empty(b.n, dtype=torch.float32, device="cuda"),
                             argmax=torch.empty(b.n, dtype=torch.int32, device="cuda"))
    ctx.sync(300.0)
    maxP = maxP.cpu().numpy()
    argmax = argmax.cpu().numpy()
    P = P.cpu().numpy()
    n_t = np.diff(b.t_off)
    order = np.argsort(n_t, kind="stable")
    # the shortest, the middle and the longest curves: a batch item sums a whole
    # curve in FP32, so the longest carry the largest rounding error
    picks = np.concatenate([order[:4], order[2046:2050], order[-4:]])
    for c in picks:
        t, X = _oracle_noise_curve(b, seed, int(c), 0)
        ref = oracle.periodogram(t, X, b.f0[c], b.df[c], b.nf[c])
        got = P[P_off[c]:P_off[c + 1]].astype(np.float64)
        assert_parity(got, ref, what="curve %d (N_t = %d)" % (c, n_t[c]))
        assert maxP[c] == got.max() and got[argmax[c]] == got.max(), c
        assert abs(maxP[c] - ref.max()) <= TOL_ABS * ref.max(), c
        assert ref[argmax[c]] >= ref.max() * (1 - 2 * TOL_ABS), c
