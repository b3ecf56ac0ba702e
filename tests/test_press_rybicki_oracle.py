"""Pins of the oracle's Press-Rybicki approximation (oracle/press_rybicki.py).

Pinned against things other than itself: the direct Eq. 1-2 oracle (C) when
every sample sits on a grid node (extirpolation is then exact), convergence
to the direct periodogram as the number of extirpolation nodes grows, the
accuracy of the default (4 nodes) on uneven sampling, the textbook centred
cubic weights at a midpoint, the Lagrange weights' reproduction of
polynomials, and invariances.  Planted mistakes in the module
(copied to a temporary file) must each fail one of these checks.
"""
import importlib.util

import numpy as np
import pytest

import oracle
from oracle import press_rybicki as pr


def _uneven(n=300, seed=0, T=50.0):
    rng = np.random.default_rng(seed)
    t = np.sort(rng.uniform(0, T, n)) + 17.0
    X = np.sin(2 * np.pi * 1.3 * t) + 0.5 * np.cos(2 * np.pi * 0.21 * t) + rng.normal(size=n)
    return t, X


def _grid(t, n):
    df = 1.0 / (4 * (t.max() - t.min()))
    return df, 4 * n


def _on_grid(mod, n=257, seed=1):
    rng = np.random.default_rng(seed)
    df, nf = 1.0 / 4000.0, 4 * n
    n_fft = mod.fft_size(nf, 4)
    idx = np.sort(rng.choice(np.arange(0, n_fft // 4), n, replace=False))
    t = 3.0 + idx / (df * n_fft)
    X = rng.normal(size=n) + np.sin(2 * np.pi * 0.01 * t)
    return t, X, df, nf


def test_exact_when_samples_sit_on_grid_nodes():
    t, X, df, nf = _on_grid(pr)
    ref = oracle.periodogram(t, X, df, df, nf)
    got = pr.periodogram(t, X, 1, nf, df, 4)
    assert np.max(np.abs(got - ref)) <= 1e-11 * ref.max()


def test_converges_to_the_direct_periodogram():
    t, X = _uneven()
    df, nf = _grid(t, t.size)
    ref = oracle.periodogram(t, X, df, df, nf)
    errs = [np.max(np.abs(pr.periodogram(t, X, 1, nf, df, m) - ref)) / ref.max() for m in (4, 6, 8, 10)]
    assert errs[0] <= 1e-3
    assert all(b < a / 5 for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] <= 1e-9


def test_grid_offset_and_larger_fft():
    # a grid starting at j0 = 37 and an FFT twice the default size
    t, X = _uneven(200, 3)
    df, _ = _grid(t, t.size)
    nf = 500
    ref = oracle.periodogram(t, X, 37 * df, df, nf)
    got = pr.periodogram(t, X, 37, nf, df, 6, n_fft=2 * pr.fft_size(36 + nf, 6))
    assert np.max(np.abs(got - ref)) <= 1e-7 * ref.max()


def test_centred_four_point_weights_at_the_midpoint():
    # textbook centred cubic interpolation halfway between nodes k and k+1:
    # nodes k-1 .. k+2 with weights (-1, 9, 9, -1)/16
    nodes, w = pr.lagrange_nodes_weights(np.array([10.5, 0.5]), 4, 64)
    assert np.array_equal(nodes, np.array([[9, 10, 11, 12], [63, 0, 1, 2]]))
    assert np.allclose(w, np.array([[-1, 9, 9, -1], [-1, 9, 9, -1]]) / 16.0, rtol=0, atol=1e-15)


def test_lagrange_weights_reproduce_polynomials():
    rng = np.random.default_rng(4)
    g = rng.uniform(5, 100, 50)
    for macc in (2, 4, 6):
        nodes, w = pr.lagrange_nodes_weights(g, macc, 1 << 20)
        for p in range(macc):
            assert np.allclose((w * nodes.astype(float) ** p).sum(axis=1), g ** p, rtol=1e-9)


def test_invariances():
    t, X = _uneven(150, 5)
    df, nf = _grid(t, t.size)
    P = pr.periodogram(t, X, 1, nf, df, 6)
    assert np.allclose(pr.periodogram(t, 3.0 * X - 7.0, 1, nf, df, 6), P, rtol=1e-9, atol=1e-12)
    perm = np.random.default_rng(2).permutation(t.size)
    assert np.allclose(pr.periodogram(t[perm], X[perm], 1, nf, df, 6), P, rtol=1e-9, atol=1e-12)


# ---- planted mistakes ---------------------------------------------------------

SRC = pr.__file__

MUTANTS = {
    "weights_drop_factor": ("                w[:, i] *= (g - m[:, l]) / float(i - l)",
                            "                w[:, i] *= (g - m[:, l]) / float(i - l) if l != i - 1 else 1.0"),
    "single_angle_for_tau": ("g2 = np.mod(2.0 * tt * df, 1.0) * n_fft", "g2 = np.mod(tt * df, 1.0) * n_fft"),
    "forward_fft_for_x": ("F1 = np.fft.ifft(grid1) * n_fft", "F1 = np.fft.fft(grid1)"),
    "half_angle_sign": ("s2sign = np.where(W2.imag >= 0, 1.0, -1.0)", "s2sign = 1.0"),
    "off_centre_nodes": ("lo = np.floor(g).astype(np.int64) - (macc // 2 - 1)", "lo = np.floor(g).astype(np.int64)"),
    "sample_variance": ("x = (X - X.mean()) / X.std()", "x = (X - X.mean()) / X.std(ddof=1)"),
}


def _load_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    p = tmp_path / ("pr_%s.py" % name)
    p.write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location("pr_%s" % name, str(p))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _pins_pass(mod):
    nodes, w = mod.lagrange_nodes_weights(np.array([10.5]), 4, 64)
    if not (np.array_equal(nodes, [[9, 10, 11, 12]]) and np.allclose(w, np.array([[-1, 9, 9, -1]]) / 16.0)):
        return False
    t, X, df, nf = _on_grid(mod)
    ref = oracle.periodogram(t, X, df, df, nf)
    if not np.max(np.abs(mod.periodogram(t, X, 1, nf, df, 4) - ref)) <= 1e-11 * ref.max():
        return False
    t, X = _uneven()
    df, nf = _grid(t, t.size)
    ref = oracle.periodogram(t, X, df, df, nf)
    if not np.max(np.abs(mod.periodogram(t, X, 1, nf, df, 8) - ref)) <= 1e-8 * ref.max():
        return False
    rng = np.random.default_rng(4)
    g = rng.uniform(5, 100, 50)
    nodes, w = mod.lagrange_nodes_weights(g, 4, 1 << 20)
    for p in range(4):
        if not np.allclose((w * nodes.astype(float) ** p).sum(axis=1), g ** p, rtol=1e-9):
            return False
    return True


def test_pins_pass_on_the_real_module():
    assert _pins_pass(pr)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    assert not _pins_pass(_load_mutant(tmp_path, name)), name
