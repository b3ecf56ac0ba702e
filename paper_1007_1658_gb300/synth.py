"""Seeded synthetic light curves shaped like the workloads of the paper.

This module only draws inputs: sample times, measurements and the frequency
grid a workload asks for.  It holds none of the periodogram arithmetic, and
both the CUDA path and the CPU oracle take their inputs from it.  Every
generator is a pure function of its seed (numpy ``default_rng``).

Workloads (sizes as named by each function):

* ``plain_1k``        -- 1000 uniform times in [0, 100] d, one sinusoid at
  0.37 c/d plus N(0,1) noise, grid df = 1/(4T), f_k = (k+1) df, 2000 bins.
* ``gapped_100k``     -- 1000 nights x 100 samples over 1000 d (12-h nightly
  windows, +-0.4-slot jitter), three sinusoids (0.1-5 c/d, amplitudes
  0.05-1) + N(0, 0.5); oversampling 4, 200,000 bins.
* ``cadence_65k``     -- satellite-like cadence: 72,818 slots over 1300 d,
  7,282 dropped at random (first and last kept) -> 65,536 samples; two
  1e-3-amplitude sinusoids near 20 c/d + N(0, 1e-3); oversampling 10 up to
  24.5 c/d (318,500 bins).
* ``corot_382k``      -- the shape of the paper's benchmark light curve (a
  150-d space-photometry run, 382,003 samples at a nominal 32-s cadence, Sec.
  5.2): 32-s slots over 150 d with +-0.5-s timing jitter, runs of 8-16 slots
  dropped once per 103-min orbit in 80% of the orbits (trimmed to exactly
  382,003 samples), a beta-Cephei-like signal (dominant 5.49 c/d = 0.18-d mode,
  amplitude 1e-2, four weaker modes in 4-13 c/d) + N(0, 1e-3) noise + a slow
  drift; grid df = f_0 = 1/(4T), N_f = 1,528,064 (oversampling 4 to twice the
  mean Nyquist frequency, rounded up to a multiple of 256).  ``step`` > 1 keeps
  every step-th sample (uniform down-sampling) and scales N_f with N_t.
* ``with_errors``     -- per-sample errors for the floating-mean periodogram:
  dy log-uniform in [0.3, 3] x ``sigma``, 2% of the samples 10x noisier; the
  curve's values plus a constant ``offset`` plus dy_j N(0, 1).
* ``noise_batch``     -- sampling patterns for Monte-Carlo: N_t log-uniform
  in [200, 20000], span T log-uniform in [30, 1000] d, nightly windows and
  seasonal gaps, grid oversampling 4 up to the mean Nyquist frequency.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SEED_BASE = 10070


@dataclass
class Curve:
    t: np.ndarray        # float64 [N_t]
    X: np.ndarray        # float64 [N_t]
    f0: float
    df: float
    nf: int
    signal_freqs: tuple  # injected frequencies (c/d), empty for pure noise

    @property
    def terms(self) -> int:
        return int(self.t.size) * int(self.nf)


def _span(t):
    return float(t.max() - t.min())


def plain_1k(seed: int = SEED_BASE + 1, n: int = 1000, nf: int = 2000) -> Curve:
    rng = np.random.default_rng(seed)
    t = np.sort(rng.uniform(0.0, 100.0, n))
    X = np.sin(2 * np.pi * 0.37 * t) + rng.normal(0.0, 1.0, n)
    df = 1.0 / (4.0 * _span(t))
    return Curve(t, X, df, df, nf, (0.37,))


def _nightly(rng, nights, per_night, night_len=0.5, jitter=0.4):
    slot = night_len / per_night
    d = np.repeat(np.arange(nights, dtype=np.float64), per_night)
    i = np.tile(np.arange(per_night, dtype=np.float64), nights)
    t = d + (i + 0.5) * slot + rng.uniform(-jitter, jitter, d.size) * slot
    return np.sort(t)


def gapped_100k(seed: int = SEED_BASE + 2, nights: int = 1000, per_night: int = 100,
                nf: int = 200_000) -> Curve:
    rng = np.random.default_rng(seed)
    t = _nightly(rng, nights, per_night)
    freqs = np.exp(rng.uniform(np.log(0.1), np.log(5.0), 3))
    amps = np.exp(rng.uniform(np.log(0.05), np.log(1.0), 3))
    phases = rng.uniform(0, 2 * np.pi, 3)
    X = rng.normal(0.0, 0.5, t.size)
    for f, a, p in zip(freqs, amps, phases):
        X += a * np.sin(2 * np.pi * f * t + p)
    df = 1.0 / (4.0 * _span(t))
    return Curve(t, X, df, df, nf, tuple(float(f) for f in freqs))


def cadence_65k(seed: int = SEED_BASE + 3, slots: int = 72_818, keep: int = 65_536,
                span: float = 1300.0, f_over: float = 10.0, f_max: float = 24.5,
                offset: float = 0.0) -> Curve:
    rng = np.random.default_rng(seed)
    t_all = np.linspace(0.0, span, slots)
    inner = rng.choice(np.arange(1, slots - 1), size=keep - 2, replace=False)
    idx = np.sort(np.concatenate([[0, slots - 1], inner]))
    t = t_all[idx]
    sig = (19.97, 20.04)
    phases = rng.uniform(0, 2 * np.pi, 2)
    X = offset + rng.normal(0.0, 1e-3, t.size)
    for f, p in zip(sig, phases):
        X += 1e-3 * np.sin(2 * np.pi * f * t + p)
    df = 1.0 / (f_over * _span(t))
    nf = int(round(f_max / df))
    return Curve(t, X, df, df, nf, sig)


def corot_382k(seed: int = SEED_BASE + 6, step: int = 1) -> Curve:
    rng = np.random.default_rng(seed)
    cad = 32.0 / 86400.0                      # 32 s in days
    span = 150.0
    slots = int(span / cad)                   # 405,000
    keep_n = 382_003
    orbit = 103.0 / 1440.0
    per_orbit = orbit / cad
    drop = np.zeros(slots, dtype=bool)
    for o in range(int(span / orbit) + 1):
        if rng.random() < 0.8:
            start = int(o * per_orbit + rng.uniform(0, per_orbit))
            drop[start:start + int(rng.integers(8, 17))] = True
    kept = np.flatnonzero(~drop[:slots])
    if kept.size > keep_n:  # trim at random to the exact count (first and last kept)
        inner = rng.choice(kept[1:-1], size=keep_n - 2, replace=False)
        kept = np.sort(np.concatenate([[kept[0], kept[-1]], inner]))
    t = kept * cad + rng.uniform(-0.5, 0.5, kept.size) / 86400.0
    t = np.sort(t)
    freqs = (5.4869, 5.9173, 4.3716, 7.9342, 12.8127)
    amps = (1e-2, 2.1e-3, 1.2e-3, 6e-4, 3e-4)
    phases = rng.uniform(0, 2 * np.pi, len(freqs))
    X = 1.0 + 2e-3 * (t / span) ** 2 + rng.normal(0.0, 1e-3, t.size)
    for f, a, p in zip(freqs, amps, phases):
        X += a * np.sin(2 * np.pi * f * t + p)
    if step > 1:
        t, X = t[::step], X[::step]
    df = 1.0 / (4.0 * _span(t))
    nf = int(-(-(4 * t.size) // 256) * 256)  # F_over F_high N_t / 2 with F_over F_high = 8
    return Curve(t, X, df, df, nf, freqs)


@dataclass
class ErrCurve(Curve):
    dy: np.ndarray = None  # float64 [N_t], per-sample 1-sigma errors


def with_errors(make, seed: int = SEED_BASE + 5, sigma: float = 0.5, offset: float = 12.0, **kw) -> ErrCurve:
    """Curve `make(**kw)` with per-sample errors: dy_j log-uniform in
    [0.3, 3] sigma, 2% of the samples 10x noisier; X = the curve's own values
    + offset + dy_j N(0, 1)."""
    c = make(**kw)
    rng = np.random.default_rng(seed)
    n = c.t.size
    dy = sigma * np.exp(rng.uniform(np.log(0.3), np.log(3.0), n))
    dy[rng.random(n) < 0.02] *= 10.0
    X = c.X + offset + dy * rng.normal(0.0, 1.0, n)
    return ErrCurve(c.t, X, c.f0, c.df, c.nf, c.signal_freqs, dy)


def pattern_times(rng, n: int, T: float) -> np.ndarray:
    """One gapped sampling pattern: nightly windows of random width, Poisson(2)
    seasonal gaps of 5-20% of the span, times uniform inside what is left."""
    frac = rng.uniform(0.3, 0.7)
    night_off = rng.uniform(0.0, 1.0 - frac)
    n_gaps = rng.poisson(2.0)
    g_start = rng.uniform(0.0, T, n_gaps)
    g_len = rng.uniform(0.05, 0.2, n_gaps) * T
    out = np.empty(0)
    while out.size < n:
        m = 4 * (n - out.size) + 64
        c = rng.uniform(0.0, T, m)
        ph = c - np.floor(c)
        ok = (ph >= night_off) & (ph < night_off + frac)
        for s, L in zip(g_start, g_len):
            ok &= ~((c >= s) & (c < s + L))
        out = np.concatenate([out, c[ok]])
    return np.sort(out[:n])


@dataclass
class Batch:
    t_off: np.ndarray    # int64 [n+1] CSR offsets into t
    t: np.ndarray        # float64 [sum N_t]
    f0: np.ndarray       # float64 [n]
    df: np.ndarray       # float64 [n]
    nf: np.ndarray       # int64 [n]

    @property
    def n(self) -> int:
        return int(self.nf.size)

    def curve_t(self, i):
        return self.t[self.t_off[i]:self.t_off[i + 1]]

    @property
    def terms(self) -> int:
        return int(np.sum(np.diff(self.t_off) * self.nf))


def noise_batch(n_curves: int = 4096, seed: int = SEED_BASE + 4, nt_min: int = 200,
                nt_max: int = 20000, t_min: float = 30.0, t_max: float = 1000.0,
                f_over: float = 4.0) -> Batch:
    rng = np.random.default_rng(seed)
    nts = np.exp(rng.uniform(np.log(nt_min), np.log(nt_max), n_curves)).astype(np.int64)
    Ts = np.exp(rng.uniform(np.log(t_min), np.log(t_max), n_curves))
    ts, f0, df, nf = [], np.empty(n_curves), np.empty(n_curves), np.empty(n_curves, np.int64)
    for i in range(n_curves):
        t = pattern_times(rng, int(nts[i]), float(Ts[i]))
        ts.append(t)
        d = 1.0 / (f_over * _span(t))
        f0[i], df[i] = d, d
        nf[i] = int(f_over * nts[i] // 2)
    off = np.zeros(n_curves + 1, np.int64)
    off[1:] = np.cumsum(nts)
    return Batch(off, np.concatenate(ts), f0, df, nf)


WORKLOADS = {
    "plain_1k": plain_1k,
    "gapped_100k": gapped_100k,
    "cadence_65k": cadence_65k,
    "corot_382k": corot_382k,
}
