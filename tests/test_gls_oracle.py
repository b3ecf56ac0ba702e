"""Pins of the oracle's floating-mean (generalized, weighted) periodogram.

The closed form (oracle.gls_at) is checked against things other than itself:
a brute-force weighted least-squares fit by Gram-Schmidt (oracle.gls_lsq),
the classic periodogram at frequencies where the two must coincide, exact
sinusoids (p = 1), invariances the definition implies (a floating mean, the
scale of the errors, the time origin, sample order), the equivalence of a
duplicated sample and a halved variance, and the exact Beta(1, (N-3)/2) law
of 2P/N for Gaussian noise with the stated errors, which holds for any
sampling once the mean is fitted.  Planted mistakes in the C source must each
fail one of these checks.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest
from scipy import stats

import oracle


def _uneven(n, seed, T=10.0):
    rng = np.random.default_rng(seed)
    t = np.sort(rng.uniform(0.0, T, n)) + 1234.5
    X = 5.0 + 1.5 * np.sin(2 * np.pi * 0.7 * t + 0.3) + rng.normal(size=n)
    dy = rng.uniform(0.3, 2.0, n)
    return t, X, dy


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("n,seed", [(7, 1), (40, 2), (133, 3)])
def test_equals_gram_schmidt_least_squares(weighted, n, seed):
    t, X, dy = _uneven(n, seed)
    d = dy if weighted else None
    freqs = np.array([0.13, 0.37, 0.7, 1.91, 4.4, 17.3])
    P = oracle.gls_at(t, X, freqs, d)
    ref = np.array([oracle.gls_lsq(t, X, f, d) for f in freqs])
    assert np.allclose(P, ref, rtol=1e-9, atol=1e-12 * n)


def test_classic_periodogram_at_even_grid_fourier_frequencies():
    # equal weights, t_j = j: at f = m/N (0 < m < N/2) sum cos = sum sin = 0,
    # so the fitted offset is the plain mean and the two periodograms agree;
    # at the Nyquist frequency only the cosine survives (rank-1 branch)
    rng = np.random.default_rng(9)
    for N in (16, 31):
        t = np.arange(N, dtype=np.float64) * 0.25 + 7.0
        X = rng.normal(size=N) + 2.0
        m = np.arange(1, (N - 1) // 2 + 1)
        f = m / (N * 0.25)
        assert np.allclose(oracle.gls_at(t, X, f), oracle.periodogram_at(t, X, f), rtol=1e-11, atol=1e-12)
    N = 16
    t = np.arange(N, dtype=np.float64)
    X = rng.normal(size=N)
    nyq = oracle.gls_at(t, X, [0.5])[0]
    assert nyq == pytest.approx(oracle.periodogram_at(t, X, [0.5])[0], rel=1e-11)
    assert nyq == pytest.approx(oracle.gls_lsq(t, X, 0.5), rel=1e-11)
    assert nyq == pytest.approx((np.sum((X - X.mean()) * (-1.0) ** t) ** 2 / N) / (2 * X.var()), rel=1e-11)
    assert oracle.gls_at(t, X, [0.0])[0] == 0.0


def _two_phase(seed):
    # samples at only two phases of f = 1 (integer times and integer + 0.3):
    # centred cos and sin are parallel, so the fit has one sinusoidal direction
    rng = np.random.default_rng(seed)
    t = np.sort(rng.integers(0, 50, 24) + 0.3 * rng.integers(0, 2, 24)).astype(np.float64)
    X = rng.normal(size=t.size) + 0.8 * (np.abs(t - np.round(t)) > 0.1)
    dy = rng.uniform(0.5, 1.5, t.size)
    return t, X, dy


@pytest.mark.parametrize("weighted", [False, True])
def test_rank_one_frequency_equals_least_squares(weighted):
    t, X, dy = _two_phase(21)
    d = dy if weighted else None
    P = oracle.gls_at(t, X, [1.0], d)[0]
    assert P > 0.1 and P == pytest.approx(oracle.gls_lsq(t, X, 1.0, d), rel=1e-9)


@pytest.mark.parametrize("weighted", [False, True])
def test_exact_sinusoid_with_offset_gives_full_power(weighted):
    t, _, dy = _uneven(50, 4)
    f = 0.83
    X = -3.0 + 2.0 * np.cos(2 * np.pi * f * t) + 0.5 * np.sin(2 * np.pi * f * t)
    P = oracle.gls_at(t, X, [f], dy if weighted else None)[0]
    assert P == pytest.approx(t.size / 2, rel=1e-10)


def test_bounds_and_invariances():
    t, X, dy = _uneven(60, 5)
    freqs = np.linspace(0.05, 6.0, 97)
    P = oracle.gls_at(t, X, freqs, dy)
    assert np.all(P >= -1e-12) and np.all(P <= t.size / 2 * (1 + 1e-12))
    perm = np.random.default_rng(1).permutation(t.size)
    for t2, X2, dy2 in [(t, X + 100.0, dy),          # floating mean
                        (t, -3.0 * X, dy),           # scale of the data
                        (t, X, 7.0 * dy),            # common scale of the errors
                        (t + 1e4, X, dy),            # time origin
                        (t[perm], X[perm], dy[perm])]:  # sample order
        assert np.allclose(oracle.gls_at(t2, X2, freqs, dy2), P, rtol=1e-8, atol=1e-10)
    # with unequal errors the weights matter
    assert not np.allclose(oracle.gls_at(t, X, freqs, None), P, rtol=1e-3)


def test_duplicated_sample_equals_halved_variance():
    t, X, dy = _uneven(30, 6)
    freqs = np.array([0.21, 0.7, 2.3])
    j = 11
    t2, X2, dy2 = np.insert(t, j, t[j]), np.insert(X, j, X[j]), np.insert(dy, j, dy[j])
    p_dup = 2 * oracle.gls_at(t2, X2, freqs, dy2) / t2.size
    dyh = dy.copy()
    dyh[j] /= np.sqrt(2.0)
    p_half = 2 * oracle.gls_at(t, X, freqs, dyh) / t.size
    assert np.allclose(p_dup, p_half, rtol=1e-11)


def test_noise_power_follows_the_exact_beta_law():
    """y_j = mu + dy_j e_j, e_j ~ N(0,1), uneven t: with the mean fitted and
    weights 1/dy^2, 2P/N at a fixed frequency is Beta(1, (N-3)/2) exactly."""
    n, R = 25, 3000
    rng = np.random.default_rng(12)
    t = np.sort(rng.uniform(0, 3.0, n))
    dy = rng.uniform(0.2, 3.0, n)
    dy[::6] = 20.0  # a few very noisy samples
    z = np.empty(R)
    for r in range(R):
        X = 4.0 + dy * rng.normal(size=n)
        z[r] = 2 * oracle.gls_at(t, X, [1.37], dy)[0] / n
    assert stats.kstest(z, stats.beta(1, (n - 3) / 2).cdf).pvalue > 1e-3
    # the same data read with equal weights is not Beta(1, (N-3)/2)
    zu = np.empty(R)
    for r in range(R):
        X = 4.0 + dy * rng.normal(size=n)
        zu[r] = 2 * oracle.gls_at(t, X, [1.37], None)[0] / n
    assert stats.kstest(zu, stats.beta(1, (n - 3) / 2).cdf).pvalue < 1e-3


def test_errors():
    t, X, dy = _uneven(10, 7)
    with pytest.raises(oracle.OracleError):
        oracle.gls_at(t, np.ones_like(X), [0.5])
    bad = dy.copy()
    bad[3] = 0.0
    with pytest.raises(oracle.OracleError):
        oracle.gls_at(t, X, [0.5], bad)
    with pytest.raises(oracle.OracleError):
        oracle.gls_at(t[:2], X[:2], [0.5])


# ---- planted mistakes ---------------------------------------------------------

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTANTS = {
    "dropped_C2": ("double CC = nsum_value(&cc) - C * C,", "double CC = nsum_value(&cc),"),
    "cross_sign": ("- 2.0 * CS * YC * YS) / (YY * D);", "+ 2.0 * CS * YC * YS) / (YY * D);"),
    "weights_1_over_dy": ("w[j] = 1.0 / (dy[j] * dy[j]);", "w[j] = 1.0 / dy[j];"),
    "transposed_ys": ("nsum_add(&ysn, w[j] * X[j] * si);", "nsum_add(&ysn, w[j] * X[j] * co);"),
    "mean_not_removed": ("double YC = nsum_value(&yc) - Y * C,", "double YC = nsum_value(&yc),"),
    "rank1_cos_only": ("p = (YC * YC + YS * YS) / (YY * (CC + SS));", "p = (YC * YC) / (YY * (CC + SS));"),
    "unweighted_yy": ("nsum_add(&yv, w[j] * d * d);", "nsum_add(&yv, d * d / (double)n);"),
}


def _build(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    c = tmp_path / (name + ".c")
    so = tmp_path / (name + ".so")
    c.write_text(src.replace(old, new))
    subprocess.run(["gcc", "-O1", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC", str(c), "-o", str(so), "-lm"],
                   check=True)
    lib = ctypes.CDLL(str(so))
    p = ctypes.c_void_p
    lib.oracle_gls_at.argtypes = [p, p, p, ctypes.c_int64, p, ctypes.c_int64, p]
    lib.oracle_gls_at.restype = ctypes.c_int
    return lib


def _gls(lib, t, X, freqs, dy=None):
    t, X, freqs = (np.ascontiguousarray(a, np.float64) for a in (t, X, freqs))
    dyp = None if dy is None else np.ascontiguousarray(dy, np.float64)
    P = np.empty(freqs.size)
    st = lib.oracle_gls_at(t.ctypes.data, X.ctypes.data, None if dyp is None else dyp.ctypes.data, t.size,
                           freqs.ctypes.data, freqs.size, P.ctypes.data)
    assert st == 0
    return P


def _pins_pass(lib):
    # brute-force least squares, weighted and not
    t, X, dy = _uneven(40, 2)
    freqs = np.array([0.13, 0.7, 1.91, 4.4])
    for d in (None, dy):
        ref = np.array([oracle.gls_lsq(t, X, f, d) for f in freqs])
        if not np.allclose(_gls(lib, t, X, freqs, d), ref, rtol=1e-9, atol=1e-10):
            return False
    # even-grid Nyquist (rank 1)
    rng = np.random.default_rng(9)
    tn = np.arange(16, dtype=np.float64)
    Xn = rng.normal(size=16)
    if not np.isclose(_gls(lib, tn, Xn, [0.5])[0], oracle.periodogram_at(tn, Xn, [0.5])[0], rtol=1e-11):
        return False
    # two-phase sampling (rank 1 with both cos and sin)
    tp, Xp, dyp = _two_phase(21)
    if not np.isclose(_gls(lib, tp, Xp, [1.0], dyp)[0], oracle.gls_lsq(tp, Xp, 1.0, dyp), rtol=1e-9):
        return False
    # duplicated sample vs halved variance
    j = 11
    t2, X2, dy2 = np.insert(t, j, t[j]), np.insert(X, j, X[j]), np.insert(dy, j, dy[j])
    dyh = dy.copy()
    dyh[j] /= np.sqrt(2.0)
    if not np.allclose(2 * _gls(lib, t2, X2, freqs, dy2) / t2.size, 2 * _gls(lib, t, X, freqs, dyh) / t.size,
                       rtol=1e-11):
        return False
    return True


def test_pins_pass_on_the_real_source(tmp_path):
    old, _ = MUTANTS["dropped_C2"]
    src = open(SRC).read()
    c = tmp_path / "real.c"
    so = tmp_path / "real.so"
    c.write_text(src)
    subprocess.run(["gcc", "-O1", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC", str(c), "-o", str(so), "-lm"],
                   check=True)
    lib = ctypes.CDLL(str(so))
    p = ctypes.c_void_p
    lib.oracle_gls_at.argtypes = [p, p, p, ctypes.c_int64, p, ctypes.c_int64, p]
    lib.oracle_gls_at.restype = ctypes.c_int
    assert _pins_pass(lib)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    assert not _pins_pass(_build(tmp_path, name)), name
