"""FP64 numpy oracle of the learned false-alarm surrogate.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): the product never imports
this module and it imports nothing from the product.

The paper's false-alarm probability (Eq. 3) assumes N_f independent
frequencies; Sec. 6.2 notes that the exponent should be an empirical number of
independent frequencies and that Monte-Carlo periodograms of noise estimate
it.  The surrogate learns the quantiles of the largest noise peak directly
from features of the sampling pattern.  This module spells out, plainly:

* ``features``        -- the 32 sampling-pattern features (definitions below)
* ``eq3_quantile``    -- the level-p quantile of max P under Eq. 3
* ``mlp_forward`` / ``mlp_backward`` -- 32 -> H -> H -> H -> 9, exact-erf GELU,
  a monotone quantile head that equals Eq. 3's quantiles when the network's
  output is zero, pinball loss
* ``adam_step``       -- Kingma & Ba (2015), bias-corrected

Feature definitions (t sorted, N >= 2 samples, grid f_k = f0 + k df, k < N_f):
  T = t[-1] - t[0]; dt = diff(t) (M = N - 1 values); q(p) = sorted(dt)[floor(p (M-1))];
  med = q(1/2) (lower median); f_max = f0 + (N_f - 1) df.
   0 log N            1 log T             2 log N_f         3 log(1 / (df T))
   4 log(f_max T / N) 5 log(1 + f0 / df)
   6..10 log(max(q(p), 1e-12 T) / (T / M)) for p = 0.05, 0.25, 0.5, 0.75, 0.95
  11..13 sum of dt over gaps with dt / med > c (1 + 1e-6), divided by T, for
         c = 2, 10, 100 (the margin keeps exact multiples of the cadence, e.g. one
         dropped sample of an even grid, out of the gaps)
  14 max dt / T       15 fraction of the M gaps with dt / med > 2 (1 + 1e-6)
  16..23 heights of the 8 highest local maxima of the spectral window
         W(f) = |sum_j exp(2 pi i f t_j)|^2 / N^2 on f_m = m df, m = 1..floor(f_max/df),
         interior points m with W[m] > W[m-1] and W[m] >= W[m+1] and f_m T >= 1
         (outside the main lobe); ties to the lower m; missing ones are 0
  24..31 their frequencies as f_m / f_max (0 where missing)
"""
from __future__ import annotations

import math

import numpy as np

from . import window_at

N_FEATURES = 32
LEVELS = np.array([0.05, 0.10, 0.25, 0.50, 0.75, 0.90, 0.95, 0.98, 0.99])
N_LEVELS = LEVELS.size


def features(t, f0, df, nf):
    t = np.asarray(t, dtype=np.float64)
    n = t.size
    T = t[-1] - t[0]
    dt = np.diff(t)
    M = dt.size
    s = np.sort(dt)

    def q(p):
        return s[int(math.floor(p * (M - 1)))]

    med = q(0.5)
    f_max = f0 + (nf - 1) * df
    out = np.zeros(N_FEATURES)
    out[0] = math.log(n)
    out[1] = math.log(T)
    out[2] = math.log(nf)
    out[3] = math.log(1.0 / (df * T))
    out[4] = math.log(f_max * T / n)
    out[5] = math.log1p(f0 / df)
    for i, p in enumerate((0.05, 0.25, 0.5, 0.75, 0.95)):
        out[6 + i] = math.log(max(q(p), 1e-12 * T) / (T / M))
    r = dt / med
    for i, c in enumerate((2.0, 10.0, 100.0)):
        out[11 + i] = dt[r > c * (1.0 + 1e-6)].sum() / T
    out[14] = dt.max() / T
    out[15] = np.count_nonzero(r > 2.0 * (1.0 + 1e-6)) / M
    mw = int(math.floor(f_max / df))
    if mw >= 3:
        fm = np.arange(1, mw + 1) * df
        W = window_at(t, fm)
        cand = []
        for i in range(1, mw - 1):
            if W[i] > W[i - 1] and W[i] >= W[i + 1] and fm[i] * T >= 1.0:
                cand.append((-W[i], i))
        cand.sort()
        for r, (negw, i) in enumerate(cand[:8]):
            out[16 + r] = -negw
            out[24 + r] = fm[i] / f_max
    return out


def eq3_quantile(n, nf, p):
    """Level-p quantile of max P under Eq. 3: the CDF of the largest of N_f
    independent Beta-distributed peaks is [1 - (1 - 2P/N)^((N-3)/2)]^N_f."""
    n = np.asarray(n, dtype=np.float64)
    nf = np.asarray(nf, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    a = -np.expm1(np.log(p) / nf)                        # 1 - p^(1/N_f)
    return 0.5 * n * (-np.expm1(2.0 / (n - 3.0) * np.log(a)))


def gelu(x):
    from scipy.special import erf
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    from scipy.special import erf
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def softplus(x):
    return np.logaddexp(0.0, x)


def sigmoid(x):
    return 0.5 * (1.0 + np.tanh(0.5 * x))


def init_params(rng, hidden=256, n_in=N_FEATURES, n_out=N_LEVELS):
    """He-style normal init of the hidden layers, zero biases, zero output
    layer (so an untrained network predicts Eq. 3): [W1, b1, ..., W4, b4]."""
    sizes = [n_in, hidden, hidden, hidden, n_out]
    ps = []
    for i, (a, b) in enumerate(zip(sizes[:-1], sizes[1:])):
        ps.append(rng.normal(0.0, math.sqrt(2.0 / a), (a, b)) if i < 3 else np.zeros((a, b)))
        ps.append(np.zeros(b))
    return ps


def mlp_forward(params, X, counts, y=None):
    """Quantiles (B x 9) and, with targets y, the mean pinball loss.

    Head: with e_l = log q_l^Eq3 and d_l = e_l - e_{l-1} > 0 (Eq. 3's log-spacing),
    log q_1 = e_1 + z_1 and log q_l = log q_{l-1} + d_l softplus(z_l) / log 2.
    Monotone in l for any z, and z = 0 gives Eq. 3's quantiles exactly."""
    W1, b1, W2, b2, W3, b3, W4, b4 = params
    cache = {"X": X}
    h = X
    for li, (W, b) in enumerate(((W1, b1), (W2, b2), (W3, b3))):
        zz = h @ W + b
        cache["z%d" % li] = zz
        h = gelu(zz)
        cache["a%d" % li] = h
    z = h @ W4 + b4
    cache["z"] = z
    e = np.log(eq3_quantile(counts[:, 0][:, None], counts[:, 1][:, None], LEVELS[None, :]))
    d = np.diff(e, axis=1)
    cache["d"] = d
    lq = np.empty_like(z)
    lq[:, 0] = e[:, 0] + z[:, 0]
    for l in range(1, N_LEVELS):
        lq[:, l] = lq[:, l - 1] + d[:, l - 1] * softplus(z[:, l]) / math.log(2.0)
    q = np.exp(lq)
    cache["q"] = q
    if y is None:
        return q, None, cache
    u = y[:, None] - q
    loss = np.mean(np.sum(np.maximum(LEVELS * u, (LEVELS - 1.0) * u), axis=1))
    return q, loss, cache


def mlp_backward(params, cache, y):
    """Gradients of the mean pinball loss w.r.t. [W1, b1, ..., W4, b4]."""
    W1, b1, W2, b2, W3, b3, W4, b4 = params
    q, z, d = cache["q"], cache["z"], cache["d"]
    B = q.shape[0]
    u = y[:, None] - q
    dq = np.where(u > 0, -LEVELS, 1.0 - LEVELS) / B     # d loss / d q
    dlq = dq * q                                          # q = exp(log q)
    # log q_l = z_1 (+ e_1) + sum_{i=2..l} d_i softplus(z_i) / log 2
    tail = np.cumsum(dlq[:, ::-1], axis=1)[:, ::-1]
    dz = np.empty_like(z)
    dz[:, 0] = tail[:, 0]
    dz[:, 1:] = tail[:, 1:] * d * sigmoid(z[:, 1:]) / math.log(2.0)
    grads = [None] * 8
    a2 = cache["a2"]
    grads[6] = a2.T @ dz
    grads[7] = dz.sum(axis=0)
    dh = dz @ W4.T
    for li, (W, idx) in zip((2, 1, 0), ((W3, 4), (W2, 2), (W1, 0))):
        dzz = dh * gelu_grad(cache["z%d" % li])
        hin = cache["a%d" % (li - 1)] if li > 0 else cache["X"]
        grads[idx] = hin.T @ dzz
        grads[idx + 1] = dzz.sum(axis=0)
        dh = dzz @ W.T
    return grads


def adam_step(params, grads, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (in place on copies); step counts from 1."""
    out_p, out_m, out_v = [], [], []
    for p, g, mm, vv in zip(params, grads, m, v):
        mm = beta1 * mm + (1 - beta1) * g
        vv = beta2 * vv + (1 - beta2) * g * g
        mh = mm / (1 - beta1 ** step)
        vh = vv / (1 - beta2 ** step)
        out_p.append(p - lr * mh / (np.sqrt(vh) + eps))
        out_m.append(mm)
        out_v.append(vv)
    return out_p, out_m, out_v
