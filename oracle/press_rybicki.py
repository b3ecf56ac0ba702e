"""Press & Rybicki (1989) fast approximate Lomb-Scargle periodogram, FP64 numpy.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): only ``tests/`` and
the benchmark's CPU legs use it; the product library never does.

The paper's introduction cites this method as the O(N log N) alternative to
the direct O(N_t N_f) evaluation: the unevenly sampled data are replaced by a
uniformly sampled approximation ("extirpolation") whose FFT gives the sums of
Eq. 5-8 at every grid frequency at once.  The steps, in the order of Press &
Rybicki (1989, ApJ 338, 277):

1. normalize X as for Eq. 1 (zero mean, unit population variance);
2. take a periodic grid of ``n_fft`` (a power of two) nodes spanning one
   period 1/df of the grid spacing, so that FFT bin K is the frequency K df;
   n_fft >= 2 macc (K_hi + 1) keeps at least macc nodes per period of the
   highest doubled frequency 2 K_hi df that the tau sums need;
3. spread ("extirpolate") every sample onto the ``macc`` nodes around its
   position g = frac((t - t0) df) n_fft with the Lagrange weights that would
   interpolate a function from those nodes to g -- the data values x_j for the
   sums over x, unit values at the positions of 2(t - t0) for the sums over
   the doubled angle;
4. one FFT of each grid: sum_j x_j exp(i w t_j) and sum_j exp(2 i w t_j) at
   every w = 2 pi K df;
5. Eq. 5-6 from those sums, tau by the half-angle formulas.

The result is exact when every sample sits on a node (the weights reduce to
a single 1) and approaches the direct periodogram as macc grows; both are
pinned in ``tests/test_press_rybicki_oracle.py``.  The FFT is numpy's.
"""
from __future__ import annotations

import numpy as np


def fft_size(k_hi: int, macc: int) -> int:
    """Smallest power of two >= 2 macc (k_hi + 1)."""
    need = 2 * macc * (int(k_hi) + 1)
    n = 1
    while n < need:
        n *= 2
    return n


def lagrange_nodes_weights(g: np.ndarray, macc: int, n_fft: int):
    """Nodes (mod n_fft) and Lagrange weights of the macc-point interpolation
    from integer nodes to the real positions g: nodes floor(g) - (macc/2 - 1)
    ... for even macc (centred), weight_i = prod_{l != i} (g - m_l)/(m_i - m_l)."""
    g = np.asarray(g, dtype=np.float64)
    lo = np.floor(g).astype(np.int64) - (macc // 2 - 1)
    m = lo[:, None] + np.arange(macc)[None, :]
    w = np.ones((g.size, macc))
    for i in range(macc):
        for l in range(macc):
            if l != i:
                w[:, i] *= (g - m[:, l]) / float(i - l)
    return np.mod(m, n_fft), w


def extirpolate(g: np.ndarray, y: np.ndarray, macc: int, n_fft: int) -> np.ndarray:
    """Grid of n_fft nodes that carries the values y at the positions g."""
    nodes, w = lagrange_nodes_weights(g, macc, n_fft)
    grid = np.zeros(n_fft)
    np.add.at(grid, nodes.ravel(), (w * np.asarray(y, dtype=np.float64)[:, None]).ravel())
    return grid


def sums(t, X, j0: int, nf: int, df: float, macc: int = 4, n_fft: int | None = None):
    """(Z, W2, n, n_fft): approximations of sum x_j e^{i w t'_j} and
    sum e^{2 i w t'_j} at w = 2 pi (j0 + k) df, k < nf, t' = t - min t, x the
    normalized data."""
    t = np.asarray(t, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    x = (X - X.mean()) / X.std()
    tt = t - t.min()
    k_hi = j0 + nf - 1
    if n_fft is None:
        n_fft = fft_size(k_hi, macc)
    g1 = np.mod(tt * df, 1.0) * n_fft
    g2 = np.mod(2.0 * tt * df, 1.0) * n_fft
    grid1 = extirpolate(g1, x, macc, n_fft)
    grid2 = extirpolate(g2, np.ones_like(x), macc, n_fft)
    # sum_m grid[m] exp(+2 pi i K m / n_fft)
    F1 = np.fft.ifft(grid1) * n_fft
    F2 = np.fft.ifft(grid2) * n_fft
    K = j0 + np.arange(nf)
    return F1[K], F2[K], t.size, n_fft


def periodogram(t, X, j0: int, nf: int, df: float, macc: int = 4, n_fft: int | None = None):
    """P_n at f = (j0 + k) df, k < nf, by the Press-Rybicki approximation."""
    Z, W2, n, _ = sums(t, X, j0, nf, df, macc, n_fft)
    R = np.abs(W2)
    with np.errstate(invalid="ignore", divide="ignore"):
        c2 = np.where(R > 0, W2.real / np.where(R > 0, R, 1.0), 1.0)
    s2sign = np.where(W2.imag >= 0, 1.0, -1.0)
    # half angle: cos wtau >= 0, sin wtau with the sign of sin 2 wtau
    c = np.sqrt(np.maximum(0.5 * (1.0 + c2), 0.0))
    s = s2sign * np.sqrt(np.maximum(0.5 * (1.0 - c2), 0.0))
    Ct = Z.real * c + Z.imag * s
    St = Z.imag * c - Z.real * s
    den1 = 0.5 * (n + R)
    den2 = 0.5 * (n - R)
    eps = n * 2.0 ** -40
    P = np.where(den1 > eps, Ct * Ct / np.where(den1 > eps, den1, 1.0), 0.0)
    P += np.where(den2 > eps, St * St / np.where(den2 > eps, den2, 1.0), 0.0)
    return 0.5 * P
