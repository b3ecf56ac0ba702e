"""Shared parity helpers for the GPU tests (tolerances of the periodogram)."""
import numpy as np

# |dP| <= TOL_ABS * max P over the compared bins, and relative error <= TOL_PEAK
# at the ten largest well-separated peaks.
TOL_ABS = 1e-4
TOL_PEAK = 1e-4


def top_peaks(P, n=10, sep=4):
    """Indices of the n largest strict local maxima, greedily >= sep bins apart
    (ties go to the lower index)."""
    P = np.asarray(P, dtype=np.float64)
    if P.size < 3:
        return np.argsort(-P, kind="stable")[:n]
    loc = np.where((P[1:-1] > P[:-2]) & (P[1:-1] >= P[2:]))[0] + 1
    order = loc[np.argsort(-P[loc], kind="stable")]
    chosen = []
    for i in order:
        if all(abs(int(i) - c) >= sep for c in chosen):
            chosen.append(int(i))
        if len(chosen) == n:
            break
    return np.array(chosen, dtype=np.int64)


def assert_parity(got, ref, tol_abs=TOL_ABS, tol_peak=TOL_PEAK, peaks=None, what=""):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape, (got.shape, ref.shape)
    assert np.all(np.isfinite(got)), what + ": non-finite output"
    scale = ref.max()
    err = np.abs(got - ref)
    worst = int(np.argmax(err))
    assert err[worst] <= tol_abs * scale, "%s: max|dP| = %.3g at %d (ref %.6g got %.6g), bound %.3g" % (
        what, err[worst], worst, ref[worst], got[worst], tol_abs * scale)
    if peaks is None:
        peaks = top_peaks(ref)
    if len(peaks):
        rel = err[peaks] / ref[peaks]
        assert rel.max() <= tol_peak, "%s: peak rel err %.3g at %d" % (what, rel.max(), peaks[np.argmax(rel)])
    return float(err.max() / scale)


def degenerate_band(t, freqs, rel=2.0 ** -15):
    """Mask of the frequencies where the smaller denominator of Eq. 1,
    (N - R)/2 with R = |sum_j exp(4 pi i f t_j)| (the tau sums of Eq. 2), is
    at most N rel.  The GPU leaves out a term whose FP32 denominator is below
    N 2^-16 and the FP64 oracle one below N 2^-40, so only inside this band
    may the two take different branches of the degenerate-term rule.  R is
    formed here in FP64 from its definition (tiny inputs only)."""
    t = np.asarray(t, np.float64)
    f = np.asarray(freqs, np.float64)
    ph = 2.0 * np.outer(f, t - t.min())
    ph -= np.round(ph)
    R = np.abs(np.exp(2j * np.pi * ph).sum(axis=1))
    return (t.size - R) / 2.0 <= t.size * rel


def kept_term(t, X, freqs):
    """P_n with the (N - R)/2 term of Eq. 5 left out: what the degenerate-term
    rule leaves when that denominator vanishes.  With x the data at zero mean
    and unit population variance, Z = sum x_j e^{i w t_j}, W = sum e^{2 i w t_j},
    R = |W| and e^{2 i w tau} = W / R (Eq. 6):
    (|Z|^2 + Re(conj(W) Z^2) / R) / (2 (N + R)).  Tiny inputs only."""
    t = np.asarray(t, np.float64)
    X = np.asarray(X, np.float64)
    x = (X - X.mean()) / X.std()
    f = np.asarray(freqs, np.float64)
    ph = np.outer(f, t - t.min())
    ph -= np.round(ph)
    e1 = np.exp(2j * np.pi * ph)
    Z = e1 @ x
    W = (e1 * e1).sum(axis=1)
    R = np.abs(W)
    return (np.abs(Z) ** 2 + np.real(np.conj(W) * Z * Z) / R) / (2.0 * (t.size + R))


def assert_parity_with_degenerate_band(got, ref, t, X, freqs, rel=2.0 ** -15, kept_tol=TOL_ABS, what=""):
    """assert_parity (|dP| <= 1e-4 max P) on every bin outside the degenerate
    band; inside it, the GPU value is the kept term of the degenerate-term
    rule (to the same 1e-4) and never above the oracle's (which may still
    count the vanishing term)."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    band = degenerate_band(t, freqs, rel)
    scale = max(ref.max(), 1e-300)
    out = ~band
    if out.any():
        err = np.abs(got[out] - ref[out])
        assert err.max() <= TOL_ABS * scale, "%s: max|dP| = %.3g outside the band, bound %.3g" % (
            what, err.max(), TOL_ABS * scale)
    if band.any():
        kept = kept_term(t, X, np.asarray(freqs, np.float64)[band])
        assert np.all(np.abs(got[band] - kept) <= kept_tol * max(scale, kept.max())), (what, got[band], kept)
        assert np.all(got[band] <= ref[band] + TOL_ABS * scale), (what, got[band], ref[band])
    return int(band.sum())
