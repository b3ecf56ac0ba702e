"""Pins of the FP64 CPU oracle against facts the paper and the mathematics fix.

No test here compares the oracle with itself re-typed: each one checks a
closed form, an invariant, a brute-force computation by a different algorithm,
or a statistical law.  A dropped term, a wrong sign, a transposed operand or a
wrong index in ``oracle/oracle.c`` fails at least one of them (the
``test_planted_*`` cases show this for a few such mistakes).

Parity status per oracle routine:
  normalize ............ pinned (numpy mean/var; golden closed forms)
  periodogram[_at] ..... pinned (closed forms, LSQ brute force, invariances, beta law)
  periodogram_refac_at . pinned (equals the direct form; closed forms)
  lsq_power ............ pinned (closed forms; projection identity)
  fap .................. pinned (limits; scipy beta survival function at N_f = 1)
  grid ................. pinned (Eq. 10-11 arithmetic on the paper's configurations)
  periodogram_fp32phase_at pinned (equals exact form at small f*t; float rounding model)
  window_at ............ pinned (Dirichlet-kernel closed form)
  philox4x32_10 ........ pinned (the authors' published known-answer vectors,
                         tests/golden/philox4x32_10_kat.txt; bit balance, avalanche)
  noise ................ pinned (Box-Muller of pinned Philox words: normality, stream
                         separation, exact Dirichlet law of even-grid noise maxima)
"""
import os

import numpy as np
import pytest
from scipy import stats

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _even(N, m, phi, dt):
    j = np.arange(N)
    return j * dt, np.sqrt(2.0) * np.cos(2 * np.pi * m * j / N + phi)


def _golden_rows():
    rows = []
    with open(os.path.join(GOLDEN, "even_grid_sinusoid.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                N, m, phi, dt, p_m, p_o = line.split()
                rows.append((int(N), int(m), float(phi), float(dt), float(p_m), float(p_o)))
    return rows


@pytest.mark.parametrize("row", _golden_rows())
def test_even_grid_closed_form(row):
    N, m, phi, dt, p_m, p_other = row
    t, x = _even(N, m, phi, dt)
    others = [mm for mm in (1, 2, m - 1, m + 1, N // 2 - 1) if 0 < mm < N / 2 and mm != m]
    f = np.array([m] + others, dtype=np.float64) / (N * dt)
    for fn in (oracle.periodogram_at, oracle.periodogram_refac_at):
        P = fn(t, x, f)
        assert abs(P[0] - p_m) <= 1e-9 * p_m
        assert np.all(np.abs(P[1:] - p_other) <= 1e-9 * N)
    assert abs(oracle.lsq_power(t, x, f[0]) - p_m) <= 1e-9 * p_m


def test_normalize_population_variance():
    rng = np.random.default_rng(1)
    X = rng.normal(3.0, 7.0, 1001)
    x, mean, var = oracle.normalize(X)
    assert abs(mean - np.mean(X)) < 1e-12 * abs(np.mean(X))
    assert abs(var - np.var(X)) < 1e-12 * np.var(X)  # numpy's default is ddof=0
    assert abs(np.mean(x)) < 1e-14 and abs(np.mean(x * x) - 1.0) < 1e-13


def test_bounds_zero_to_half_n():
    # chi^2 reduction can never exceed sum x^2 = N (population normalization)
    rng = np.random.default_rng(2)
    for n in (3, 10, 257):
        t = np.sort(rng.uniform(0, 50, n))
        X = rng.normal(size=n) + 2 * np.sin(3.1 * t)
        f = rng.uniform(0, 5, 300)
        P = oracle.periodogram_at(t, X, f)
        assert np.all(P >= -1e-12) and np.all(P <= n / 2 * (1 + 1e-12))


@pytest.mark.parametrize("n", [3, 4, 7, 16, 64])
def test_equals_least_squares_brute_force(n):
    rng = np.random.default_rng(100 + n)
    t = np.sort(rng.uniform(0, 10, n))
    X = rng.normal(size=n) + np.cos(2 * np.pi * 1.3 * t)
    for f in rng.uniform(0.01, 4.0, 25):
        p_ls = oracle.periodogram_at(t, X, [f])[0]
        p_sq = oracle.lsq_power(t, X, f)
        assert abs(p_ls - p_sq) <= 1e-9 * max(1.0, abs(p_sq)), (n, f, p_ls, p_sq)


def test_direct_equals_refactored_form():
    rng = np.random.default_rng(3)
    t = np.sort(rng.uniform(0, 300, 2000))
    X = rng.normal(size=t.size) + 0.4 * np.sin(2 * np.pi * 0.77 * t)
    f = np.concatenate([rng.uniform(0, 20, 400), [0.77, 1e-6]])
    a = oracle.periodogram_at(t, X, f)
    b = oracle.periodogram_refac_at(t, X, f)
    assert np.max(np.abs(a - b) / np.maximum(1.0, a)) < 1e-10


def test_time_shift_and_affine_invariance():
    rng = np.random.default_rng(4)
    t = np.sort(rng.uniform(0, 100, 500))
    X = rng.normal(size=500) + np.sin(2 * np.pi * 2.2 * t)
    f = np.linspace(0.01, 10, 997)
    P = oracle.periodogram_at(t, X, f)
    Ps = oracle.periodogram_at(t + 2.4e6, X, f)  # a Julian-date-like origin
    assert np.max(np.abs(P - Ps)) < 1e-6 * P.max()
    Pa = oracle.periodogram_at(t, -3.5 * X + 1e3, f)
    assert np.max(np.abs(P - Pa)) < 1e-10 * P.max()
    # shuffling the samples is a relabelling of j
    perm = rng.permutation(500)
    Pp = oracle.periodogram_at(t[perm], X[perm], f)
    assert np.max(np.abs(P - Pp)) < 1e-10 * P.max()


def test_integer_times_alias_symmetry():
    # t_j integers: exp(2 pi i (f+1) t) = exp(2 pi i f t) and P(1-f) = P(f)
    rng = np.random.default_rng(5)
    t = np.sort(rng.choice(np.arange(0, 400), 150, replace=False)).astype(float)
    X = rng.normal(size=150)
    f = rng.uniform(0.001, 0.499, 50)
    P = oracle.periodogram_at(t, X, f)
    assert np.max(np.abs(P - oracle.periodogram_at(t, X, f + 1.0))) < 1e-9 * P.max()
    assert np.max(np.abs(P - oracle.periodogram_at(t, X, 1.0 - f))) < 1e-9 * P.max()


def test_degenerate_terms_and_zero_frequency():
    N = 32
    t, x = _even(N, 3, 0.0, 1.0)
    # Nyquist of an even grid: every sin w(t - tau) vanishes -> that term is zero
    P = oracle.periodogram_at(t, x, [0.5, 0.0])
    assert np.all(np.abs(P) < 1e-20 * N)
    with pytest.raises(oracle.OracleError):
        oracle.periodogram_at(t, np.ones(N), [0.1])  # zero variance
    with pytest.raises(oracle.OracleError):
        oracle.periodogram_at(t[:1], x[:1], [0.1])  # N_t < 2
    xx = x.copy()
    xx[3] = np.nan
    with pytest.raises(oracle.OracleError):
        oracle.periodogram_at(t, xx, [0.1])


def test_fap_eq3_limits_and_beta_survival():
    n, nf = 200, 1000
    assert oracle.fap(0.0, n, nf) == 1.0
    assert oracle.fap(n / 2, n, nf) == 0.0
    z = np.linspace(0.001, 0.2, 50)
    P = z * n / 2
    q1 = oracle.fap(P, n, 1)
    assert np.allclose(q1, stats.beta.sf(z, 1, (n - 3) / 2), rtol=1e-10, atol=1e-300)
    q = oracle.fap(P, n, nf)
    assert np.all(np.diff(q) <= 0)
    # N_f independent trials: Q = 1 - (1 - q1)^N_f
    assert np.allclose(q, -np.expm1(nf * np.log1p(-q1)), rtol=1e-9, atol=1e-15)


def test_grid_eq10_eq11():
    f0, df, nf = oracle.grid(0.0, 100.0, 1000, 4.0, 1.0)
    assert nf == 2000 and df == pytest.approx(1 / 400.0) and f0 == df
    # the highest frequency with F_high = 1 is the mean Nyquist N_t / (2 T)
    assert (nf * df) == pytest.approx(1000 / (2 * 100.0))
    f0, df, nf = oracle.grid(5.0, 1305.0, 65536, 10.0, 2.0)
    assert nf == 655360 and df == pytest.approx(1 / 13000.0)
    with pytest.raises(oracle.OracleError):
        oracle.grid(1.0, 1.0, 10, 4.0, 1.0)


def test_beta_law_for_gaussian_noise():
    # Even sampling at a Fourier frequency: 2P/N ~ Beta(1, (N-3)/2) exactly
    # (the law behind Eq. 3).
    N, m, R = 40, 7, 3000
    t = np.arange(N, dtype=float)
    rng = np.random.default_rng(6)
    z = np.empty(R)
    for r in range(R):
        z[r] = 2 * oracle.periodogram_at(t, rng.normal(size=N), [m / N])[0] / N
    ks = stats.kstest(z, stats.beta(1, (N - 3) / 2).cdf)
    assert ks.pvalue > 1e-3, ks
    # a wrong exponent would show up: Beta(1, (N-1)/2) must be rejected
    assert stats.kstest(z, stats.beta(1, (N - 1) / 2 + 4).cdf).pvalue < 1e-3


def test_window_dirichlet_closed_form():
    N = 50
    t = np.arange(N, dtype=float)
    f = np.array([0.0, 0.013, 0.1, 0.37, 1.0, 2.0 / N])
    W = oracle.window_at(t, f)
    with np.errstate(invalid="ignore", divide="ignore"):
        d = (np.sin(np.pi * f * N) / (N * np.sin(np.pi * f))) ** 2
    d[(f == 0) | (f == 1.0)] = 1.0
    assert np.allclose(W, d, rtol=1e-10, atol=1e-14)


def test_fp32_phase_model():
    rng = np.random.default_rng(7)
    # small f*t: single-precision phase is nearly exact
    t = np.sort(rng.uniform(0, 1.0, 300))
    X = rng.normal(size=300)
    ks = np.arange(0, 200)
    df = 0.01
    exact = oracle.periodogram(t, X, df, df, 200)
    approx = oracle.periodogram_fp32phase_at(t, X, df, df, ks)
    assert np.max(np.abs(exact - approx)) < 1e-4 * exact.max()
    # f*t ~ 3e4 turns: float rounding of f*t (ulp 2^-9 turn, random across samples)
    # costs ~(2 pi sigma)^2 ~ 1e-3 of the coherent peak, 10x the 1e-4 budget
    t = np.sort(rng.uniform(0, 1300, 3000))
    X = np.sin(2 * np.pi * 20.0 * t) + 0.1 * rng.normal(size=3000)
    df = 1 / 13000
    k0 = int(round(20.0 / df)) - 1  # grid index of 20 c/d (f_k = (k+1) df)
    ks = np.arange(k0 - 3, k0 + 4)
    exact = oracle.periodogram(t, X, df, df, k0 + 4)[ks]
    approx = oracle.periodogram_fp32phase_at(t, X, df, df, ks)
    assert np.max(np.abs(exact - approx)) > 3e-4 * exact.max()


def _philox_kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                w = [int(x, 16) for x in line.split()]
                assert len(w) == 10
                rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answer_vectors():
    # Salmon et al. 2011: the published Philox-4x32-10 known answers, word for word.
    rows = _philox_kat_rows()
    assert len(rows) == 3
    for ctr, key, want in rows:
        got = oracle.philox4x32_10(ctr, key)
        assert [int(x) for x in got] == want, (["%08x" % x for x in got], ["%08x" % x for x in want])


def test_philox_bits_and_avalanche():
    key = np.array([0x12345678, 0x9ABCDEF0], np.uint32)
    words = np.concatenate([oracle.philox4x32_10([i, 7, 0, 0], key) for i in range(4096)])
    bits = np.unpackbits(words.view(np.uint8))
    assert abs(bits.mean() - 0.5) < 0.005
    counts = np.bincount(words & 0xFF, minlength=256)
    assert stats.chisquare(counts).pvalue > 1e-4
    flips = []
    for i in range(200):
        a = oracle.philox4x32_10([i, 1, 2, 3], key)
        b = oracle.philox4x32_10([i ^ 1, 1, 2, 3], key)
        flips.append(np.unpackbits((a ^ b).view(np.uint8)).sum())
    assert 54 < np.mean(flips) < 74  # ~64 of 128 bits flip
    assert len({tuple(oracle.philox4x32_10([i, 0, 0, 0], [0, 0])) for i in range(1000)}) == 1000


def test_noise_is_standard_normal_and_stream_separated():
    x = oracle.noise(2024, 3, 0, 40001)
    assert stats.kstest(x, "norm").pvalue > 1e-3
    assert abs(x.mean()) < 0.02 and abs(x.var() - 1) < 0.03
    y = oracle.noise(2024, 3, 1, 40001)
    z = oracle.noise(2024, 4, 0, 40001)
    assert abs(np.corrcoef(x, y)[0, 1]) < 0.03 and abs(np.corrcoef(x, z)[0, 1]) < 0.03
    # a prefix is the same stream
    assert np.array_equal(oracle.noise(2024, 3, 0, 13), x[:13])


def test_even_grid_noise_maxima_follow_the_dirichlet_law():
    # N even, interior Fourier frequencies: the normalized peak heights 2P_k/N are
    # the first N/2 - 1 components of a Dirichlet(1, ..., 1, 1/2) vector (the
    # mean-removed noise splits into orthogonal cos/sin planes plus the Nyquist
    # cosine); the oracle's noise maxima must follow its maximum.
    N, R = 64, 2500
    t = np.arange(N, dtype=float)
    nf = N // 2 - 1
    fr = np.arange(1, nf + 1) / N
    rng = np.random.default_rng(12)
    m = np.array([oracle.periodogram_at(t, rng.normal(size=N), fr).max() for _ in range(R)])
    g = np.concatenate([rng.gamma(1.0, size=(R, nf)), rng.gamma(0.5, size=(R, 1))], axis=1)
    exact = N / 2 * (g[:, :nf].max(axis=1) / g.sum(axis=1))
    assert stats.ks_2samp(m, exact).pvalue > 1e-3
    # the single-peak marginal of the same law is Eq. 3's Beta(1, (N-3)/2)
    assert stats.kstest(g[:, 0] / g.sum(axis=1), stats.beta(1, (N - 3) / 2).cdf).pvalue > 1e-3
