"""FP64 CPU oracle for the normalized Lomb-Scargle periodogram.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package; the
product library (``paper_1007_1658_gb300``) never does, and this package never
imports the product.  The heavy lifting lives in ``oracle.c`` (plain C, FP64,
OpenMP over frequencies); this module only compiles it and marshals numpy
arrays.  Every routine cites the passage of the paper it follows:

* ``normalize``            -- Sec. 3 (zero mean, unit *population* variance)
* ``periodogram[_at]``     -- Eq. 1 with tau from Eq. 2 (direct two-pass form)
* ``periodogram_refac_at`` -- Eq. 5-8 (single-pass sums), pinned against Eq. 1-2
* ``lsq_power``            -- chi^2-reduction reading of Eq. 1 (brute force)
* ``fap``                  -- Eq. 3
* ``grid``                 -- Eq. 9-11
* ``periodogram_fp32phase_at`` -- the paper's single-precision phase (Sec. 4.3)
* ``window_at``            -- spectral window (|sum exp(2 pi i f t)|^2 / N^2)
* ``gls_at`` / ``gls_lsq`` -- floating-mean weighted periodogram (Sec. 6.3) and its
  brute-force least-squares reading
* ``philox4x32_10`` / ``noise`` -- counter-based Gaussian noise for Sec. 6.2's
  Monte-Carlo use (Salmon et al. 2011; Box & Muller 1958); the generator is
  pinned against the authors' published known-answer vectors

Parity status of each routine is listed in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_STATUS = {0: "ok", 1: "bad argument", 2: "degenerate (zero variance)",
           3: "non-finite input", 4: "out of memory"}


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, FP64, OpenMP)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB)
        d, i64, p = ctypes.c_double, ctypes.c_int64, ctypes.c_void_p
        u32, u64 = ctypes.c_uint32, ctypes.c_uint64
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_normalize.argtypes = [p, i64, p, p, p]
        lib.oracle_periodogram_at.argtypes = [p, p, i64, p, i64, p]
        lib.oracle_periodogram.argtypes = [p, p, i64, d, d, i64, p]
        lib.oracle_periodogram_refac_at.argtypes = [p, p, i64, p, i64, p]
        lib.oracle_lsq_power.argtypes = [p, p, i64, d, p]
        lib.oracle_fap.argtypes = [d, i64, d]
        lib.oracle_fap.restype = d
        lib.oracle_grid.argtypes = [d, d, i64, d, d, p, p, p]
        lib.oracle_periodogram_fp32phase_at.argtypes = [p, p, i64, d, d, p, i64, p]
        lib.oracle_window_at.argtypes = [p, i64, p, i64, p]
        lib.oracle_philox4x32_10.argtypes = [p, p, p]
        lib.oracle_philox4x32_10.restype = None
        lib.oracle_gls_at.argtypes = [p, p, p, i64, p, i64, p]
        lib.oracle_gls_lsq.argtypes = [p, p, p, i64, d, p]
        lib.oracle_noise.argtypes = [u64, u32, u32, i64, p]
        lib.oracle_noise.restype = None
        for name in ("oracle_normalize", "oracle_periodogram_at", "oracle_periodogram",
                     "oracle_periodogram_refac_at", "oracle_lsq_power", "oracle_grid",
                     "oracle_periodogram_fp32phase_at", "oracle_window_at", "oracle_gls_at", "oracle_gls_lsq"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(st):
    if st != 0:
        raise OracleError(_STATUS.get(st, "status %d" % st))


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def normalize(X):
    """Sec. 3: zero mean, unit population variance.  Returns (x, mean, var)."""
    X = _f64(X)
    out = np.empty_like(X)
    m, v = ctypes.c_double(), ctypes.c_double()
    _check(_load().oracle_normalize(_ptr(X), X.size, _ptr(out), ctypes.byref(m), ctypes.byref(v)))
    return out, m.value, v.value


def periodogram_at(t, X, freqs):
    """Eq. 1-2 (direct two-pass form) at arbitrary frequencies."""
    t, X, freqs = _f64(t), _f64(X), _f64(freqs)
    if t.size != X.size:
        raise ValueError("t and X differ in length")
    P = np.empty(freqs.size, dtype=np.float64)
    _check(_load().oracle_periodogram_at(_ptr(t), _ptr(X), t.size, _ptr(freqs), freqs.size, _ptr(P)))
    return P


def periodogram(t, X, f0, df, nf):
    """Eq. 1-2 on the grid f_k = f0 + k df, k = 0..nf-1."""
    t, X = _f64(t), _f64(X)
    if t.size != X.size:
        raise ValueError("t and X differ in length")
    P = np.empty(int(nf), dtype=np.float64)
    _check(_load().oracle_periodogram(_ptr(t), _ptr(X), t.size, float(f0), float(df), int(nf), _ptr(P)))
    return P


def periodogram_refac_at(t, X, freqs):
    """Eq. 5-8 (refactored single-pass sums) at arbitrary frequencies."""
    t, X, freqs = _f64(t), _f64(X), _f64(freqs)
    P = np.empty(freqs.size, dtype=np.float64)
    _check(_load().oracle_periodogram_refac_at(_ptr(t), _ptr(X), t.size, _ptr(freqs), freqs.size, _ptr(P)))
    return P


def lsq_power(t, X, f):
    """Half the chi^2 drop of a least-squares sinusoid fit (tiny inputs only)."""
    t, X = _f64(t), _f64(X)
    P = ctypes.c_double()
    _check(_load().oracle_lsq_power(_ptr(t), _ptr(X), t.size, float(f), ctypes.byref(P)))
    return P.value


def fap(P, n, nf):
    """Eq. 3 false-alarm probability for peak height P, N_t = n, N_f = nf."""
    lib = _load()
    P = np.asarray(P, dtype=np.float64)
    out = np.vectorize(lambda p: lib.oracle_fap(float(p), int(n), float(nf)))(P)
    return float(out) if out.ndim == 0 else out


def grid(t_min, t_max, n, f_over, f_high):
    """Eq. 9-11: returns (f0, df, nf) with f0 = df."""
    f0, df, nf = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    _check(_load().oracle_grid(float(t_min), float(t_max), int(n), float(f_over), float(f_high),
                               ctypes.byref(f0), ctypes.byref(df), ctypes.byref(nf)))
    return f0.value, df.value, nf.value


def periodogram_fp32phase_at(t, X, f0, df, ks):
    """Eq. 1-2 with the paper's single-precision phase (Sec. 4.3) at grid indices ks."""
    t, X = _f64(t), _f64(X)
    ks = np.ascontiguousarray(ks, dtype=np.int64)
    P = np.empty(ks.size, dtype=np.float64)
    _check(_load().oracle_periodogram_fp32phase_at(_ptr(t), _ptr(X), t.size, float(f0), float(df),
                                                   _ptr(ks), ks.size, _ptr(P)))
    return P


def window_at(t, freqs):
    """Spectral window |sum_j exp(2 pi i f t_j)|^2 / N^2."""
    t, freqs = _f64(t), _f64(freqs)
    W = np.empty(freqs.size, dtype=np.float64)
    _check(_load().oracle_window_at(_ptr(t), t.size, _ptr(freqs), freqs.size, _ptr(W)))
    return W


def gls_at(t, X, freqs, dy=None):
    """Floating-mean (generalized) periodogram, (N/2) p, at arbitrary frequencies (Sec. 6.3)."""
    t, X, freqs = _f64(t), _f64(X), _f64(freqs)
    dyp = None if dy is None else _f64(dy)
    P = np.empty(freqs.size, dtype=np.float64)
    _check(_load().oracle_gls_at(_ptr(t), _ptr(X), None if dyp is None else _ptr(dyp), t.size, _ptr(freqs),
                                 freqs.size, _ptr(P)))
    return P


def gls_lsq(t, X, f, dy=None):
    """Brute-force 3-parameter weighted least-squares reading of gls_at (tiny inputs)."""
    t, X = _f64(t), _f64(X)
    dyp = None if dy is None else _f64(dy)
    P = ctypes.c_double()
    _check(_load().oracle_gls_lsq(_ptr(t), _ptr(X), None if dyp is None else _ptr(dyp), t.size, float(f),
                                  ctypes.byref(P)))
    return P.value


def philox4x32_10(ctr, key):
    """One Philox-4x32-10 block: 4 counter words, 2 key words -> 4 words."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.empty(4, dtype=np.uint32)
    _load().oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def noise(seed, curve, real, n):
    """N(0,1) samples of (seed, curve, realization) via Philox + Box-Muller."""
    x = np.empty(int(n), dtype=np.float64)
    _load().oracle_noise(ctypes.c_uint64(int(seed)), int(curve), int(real), int(n), _ptr(x))
    return x
