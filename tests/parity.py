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
