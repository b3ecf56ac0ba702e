"""Pins of the surrogate's FP64 oracle (oracle/surrogate.py), CPU only.

Parity status: eq3_quantile, gelu, mlp_forward head, mlp_backward and
adam_step are pinned (Eq. 3 FAP round trip, scipy's normal CDF, finite
differences, Adam's closed-form first step); features are pinned by closed
forms on even and gapped grids and by exact invariances.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from oracle import surrogate as S


def test_eq3_quantile_inverts_eq3():
    for n, nf in [(200, 400), (1000, 2000), (20000, 40000), (50, 7)]:
        q = S.eq3_quantile(n, nf, S.LEVELS)
        assert np.all(np.diff(q) > 0)
        Q = np.array([oracle.fap(x, n, nf) for x in q])  # Eq. 3 as the C oracle evaluates it
        assert np.allclose(Q, 1.0 - S.LEVELS, rtol=1e-9, atol=1e-12)


def test_gelu_is_x_times_normal_cdf_and_its_derivative():
    x = np.linspace(-6, 6, 241)
    assert np.allclose(S.gelu(x), x * stats.norm.cdf(x), rtol=1e-12, atol=1e-15)
    h = 1e-6
    fd = (S.gelu(x + h) - S.gelu(x - h)) / (2 * h)
    assert np.allclose(S.gelu_grad(x), fd, rtol=1e-7, atol=1e-9)


def test_head_with_zero_output_is_eq3():
    # an untrained network (zero output layer) predicts Eq. 3's quantiles exactly
    rng = np.random.default_rng(0)
    ps = S.init_params(rng, hidden=4)
    counts = np.array([[300.0, 600.0], [5000.0, 10000.0]])
    q, _, _ = S.mlp_forward(ps, rng.normal(size=(2, S.N_FEATURES)), counts)
    expect = S.eq3_quantile(counts[:, :1], counts[:, 1:], S.LEVELS[None, :])
    assert np.allclose(q, expect, rtol=1e-12)
    # and any output keeps the quantiles ordered
    ps[6] = rng.normal(0, 3.0, ps[6].shape)
    q, _, _ = S.mlp_forward(ps, rng.normal(size=(50, S.N_FEATURES)), np.tile(counts, (25, 1)))
    assert np.all(np.diff(q, axis=1) > 0)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    ps = S.init_params(rng, hidden=5)
    ps = [p + 0.1 * rng.normal(size=p.shape) for p in ps]
    X = rng.normal(size=(7, S.N_FEATURES))
    counts = np.column_stack([rng.integers(200, 2000, 7), rng.integers(400, 4000, 7)]).astype(float)
    base = S.eq3_quantile(counts[:, :1], counts[:, 1:], S.LEVELS[None, :])
    y = base[:, 4] * np.exp(rng.normal(0, 0.3, 7))
    _, loss, cache = S.mlp_forward(ps, X, counts, y)
    g = S.mlp_backward(ps, cache, y)
    h = 1e-6
    for pi in range(8):
        flat = ps[pi].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = S.mlp_forward(ps, X, counts, y)[1]
            flat[idx] = old - h
            lm = S.mlp_forward(ps, X, counts, y)[1]
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[pi].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-5 * max(1.0, abs(fd)), (pi, idx, fd, an)


def test_pinball_minimum_is_the_sample_quantile():
    # the mean pinball loss of a constant prediction is minimized at the sample quantile
    rng = np.random.default_rng(2)
    y = rng.gamma(3.0, 2.0, 4001)
    for p in (0.05, 0.5, 0.95):
        qs = np.quantile(y, p, method="inverted_cdf")
        loss = lambda c: np.mean(np.maximum(p * (y - c), (p - 1) * (y - c)))
        assert loss(qs) <= loss(qs * 1.01) and loss(qs) <= loss(qs * 0.99)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(3)
    p = [rng.normal(size=(3, 4))]
    g = [rng.normal(size=(3, 4))]
    z = [np.zeros((3, 4))]
    out, m, v = S.adam_step(p, g, z, z, step=1, lr=0.01, eps=0.0)
    # bias-corrected first step: m_hat = g, v_hat = g^2 -> update = lr * sign(g)
    assert np.allclose(out[0], p[0] - 0.01 * np.sign(g[0]), rtol=0, atol=1e-15)
    assert np.allclose(m[0], 0.1 * g[0]) and np.allclose(v[0], 0.001 * g[0] ** 2)


def test_features_even_grid_closed_forms():
    N, dt = 400, 0.25
    t = np.arange(N) * dt
    T = (N - 1) * dt
    df = 1.0 / (4 * T)
    nf = 2 * N
    f = S.features(t, df, df, nf)
    assert f[0] == pytest.approx(math.log(N)) and f[1] == pytest.approx(math.log(T))
    assert f[2] == pytest.approx(math.log(nf)) and f[3] == pytest.approx(math.log(4.0))
    assert np.allclose(f[6:11], 0.0, atol=1e-12)          # every gap equals the mean gap
    assert np.all(f[11:14] == 0.0) and f[15] == 0.0
    assert f[14] == pytest.approx(1.0 / (N - 1))
    # window of an even grid: the Dirichlet kernel; its highest interior maxima
    fm = np.arange(1, int((df + (nf - 1) * df) / df) + 1) * df
    with np.errstate(invalid="ignore", divide="ignore"):
        W = (np.sin(np.pi * fm * N * dt) / (N * np.sin(np.pi * fm * dt))) ** 2
    W[~np.isfinite(W)] = 1.0
    loc = [i for i in range(1, W.size - 1) if W[i] > W[i - 1] and W[i] >= W[i + 1] and fm[i] * T >= 1]
    loc = sorted(loc, key=lambda i: (-W[i], i))[:8]
    assert np.allclose(f[16:24], W[loc], rtol=1e-9, atol=1e-12)
    assert np.allclose(f[24:32], fm[loc] / (df + (nf - 1) * df), rtol=1e-12)


def test_features_one_gap_closed_form():
    dt = 0.01
    t = np.concatenate([np.arange(0, 300) * dt, 10.0 + np.arange(0, 200) * dt])
    T = t[-1] - t[0]
    f = S.features(t, 0.05, 0.05, 500)
    gap = 10.0 - 299 * dt
    for k in (11, 12, 13):
        assert f[k] == pytest.approx(gap / T)
    assert f[14] == pytest.approx(gap / T) and f[15] == pytest.approx(1.0 / (t.size - 1))


def test_features_shift_and_scale():
    from paper_1007_1658_gb300 import synth
    b = synth.noise_batch(n_curves=2, seed=4, nt_min=300, nt_max=800)
    t, f0, df, nf = b.curve_t(1), b.f0[1], b.df[1], b.nf[1]
    a = S.features(t, f0, df, nf)
    sh = S.features(t + 12345.678, f0, df, nf)
    assert np.allclose(a, sh, rtol=1e-6, atol=1e-6)
    s = 3.0  # t -> s t with frequencies / s: only log T moves, by log s
    sc = S.features(t * s, f0 / s, df / s, nf)
    d = sc - a
    d[1] -= math.log(s)
    assert np.allclose(d, 0.0, atol=1e-6)
