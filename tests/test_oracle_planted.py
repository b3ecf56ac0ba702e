"""Planted mistakes: each mutant of oracle.c must fail at least one pin.

The mutants are compiled on the CPU into a temporary library; nothing here
touches a GPU or the product library.  This shows that the pins in
test_oracle_pins.py would catch a dropped term, a wrong sign, a transposed
operand, a wrong argument or the other variance convention.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTANTS = {
    "tau_sign": ("double arg = TWO_PI * r - wtau;", "double arg = TWO_PI * r + wtau;"),
    "dropped_sine_term": ("    if (Ds > eps) P += B * B / Ds;\n    return 0.5 * P;\n}\n\n/* Shared",
                          "    return 0.5 * P;\n}\n\n/* Shared"),
    "single_angle_in_tau": ("nsum_add(&s2, sin(2.0 * TWO_PI * r));", "nsum_add(&s2, sin(TWO_PI * r));"),
    "transposed_xs": ("nsum_add(&b, x[j] * s);", "nsum_add(&b, x[j] * c);"),
    "sample_variance": ("double var = nsum_value(&v) / (double)n;",
                        "double var = nsum_value(&v) / (double)(n - 1);"),
    "missing_half": ("    return 0.5 * P;\n}\n\n/* Shared", "    return P;\n}\n\n/* Shared"),
}


def _build_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, name
    src = src.replace(old, new, 1)
    c = tmp_path / (name + ".c")
    so = tmp_path / (name + ".so")
    c.write_text(src)
    subprocess.run(["gcc", "-O1", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
                    str(c), "-o", str(so), "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    p = ctypes.c_void_p
    lib.oracle_periodogram_at.argtypes = [p, p, ctypes.c_int64, p, ctypes.c_int64, p]
    lib.oracle_periodogram_at.restype = ctypes.c_int
    return lib


def _call(lib, t, X, f):
    t, X, f = (np.ascontiguousarray(a, np.float64) for a in (t, X, f))
    P = np.empty(f.size)
    st = lib.oracle_periodogram_at(t.ctypes.data, X.ctypes.data, t.size, f.ctypes.data, f.size, P.ctypes.data)
    assert st == 0
    return P


def _pins_pass(lib):
    """The same checks as the pin suite, run on a candidate library."""
    # closed form: even grid, on-grid sinusoid -> N/2
    N, m = 64, 5
    j = np.arange(N)
    t, x = j * 1.0, np.sqrt(2) * np.cos(2 * np.pi * m * j / N + 0.3)
    if abs(_call(lib, t, x, [m / N])[0] - N / 2) > 1e-9 * N:
        return False
    # brute-force least squares on an uneven grid
    rng = np.random.default_rng(11)
    t = np.sort(rng.uniform(0, 10, 16))
    X = rng.normal(size=16) + np.cos(2 * np.pi * 1.3 * t)
    for f in rng.uniform(0.01, 4.0, 10):
        if abs(_call(lib, t, X, [f])[0] - oracle.lsq_power(t, X, f)) > 1e-9 * max(1, abs(oracle.lsq_power(t, X, f))):
            return False
    return True


def test_unmutated_source_passes(tmp_path):
    src = tmp_path / "orig.c"
    src.write_text(open(SRC).read())
    so = tmp_path / "orig.so"
    subprocess.run(["gcc", "-O1", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
                    str(src), "-o", str(so), "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    p = ctypes.c_void_p
    lib.oracle_periodogram_at.argtypes = [p, p, ctypes.c_int64, p, ctypes.c_int64, p]
    assert _pins_pass(lib)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    assert not _pins_pass(_build_mutant(tmp_path, name)), name


# Plausible slips in the Philox-4x32-10 round function or key schedule
# (Salmon et al. 2011); each must miss the published known-answer vectors.
PHILOX_MUTANTS = {
    "swapped_multipliers": ("const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;",
                            "const uint32_t M0 = 0xCD9E8D57u, M1 = 0xD2511F53u;"),
    "swapped_weyl_constants": ("const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;",
                               "const uint32_t W0 = 0xBB67AE85u, W1 = 0x9E3779B9u;"),
    "key_bumped_before_first_round": ("if (round > 0) { k0 += W0; k1 += W1; }", "{ k0 += W0; k1 += W1; }"),
    "nine_rounds": ("for (int round = 0; round < 10; ++round)", "for (int round = 0; round < 9; ++round)"),
    "output_word_order": ("out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;",
                          "out[0] = c1; out[1] = c0; out[2] = c3; out[3] = c2;"),
    "hi_lo_swapped": ("c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;", "c0 = n0; c1 = lo0; c2 = n2; c3 = lo1;"),
}


def _philox_kat_rows():
    rows = []
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    with open(path) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                w = [int(x, 16) for x in line.split()]
                rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def _philox_lib(tmp_path, name, old=None, new=None):
    src = open(SRC).read()
    if old is not None:
        assert src.count(old) == 1, name
        src = src.replace(old, new, 1)
    c = tmp_path / (name + ".c")
    so = tmp_path / (name + ".so")
    c.write_text(src)
    subprocess.run(["gcc", "-O1", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
                    str(c), "-o", str(so), "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    lib.oracle_philox4x32_10.argtypes = [ctypes.c_void_p] * 3
    lib.oracle_philox4x32_10.restype = None
    return lib


def _kat_pass(lib):
    for ctr, key, want in _philox_kat_rows():
        c = np.array(ctr, np.uint32)
        k = np.array(key, np.uint32)
        out = np.empty(4, np.uint32)
        lib.oracle_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
        if [int(x) for x in out] != want:
            return False
    return True


def test_unmutated_philox_passes_known_answers(tmp_path):
    assert _kat_pass(_philox_lib(tmp_path, "philox_orig"))


@pytest.mark.parametrize("name", sorted(PHILOX_MUTANTS))
def test_philox_mutant_is_caught(tmp_path, name):
    old, new = PHILOX_MUTANTS[name]
    assert not _kat_pass(_philox_lib(tmp_path, name, old, new)), name
