"""Host-side pieces of bench.py: the roof accounting of the multi-realization
leg, the number compaction of the JSON line and the lookup of recorded DRAM
traffic (no GPU)."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_mrhs_ops_per_term_counts_each_sum_once():
    # one at a time: 4 accumulate + 2 three-term FMA per term
    assert bench.mrhs_ops_per_term(1, 64) == 6.0
    # fewer than four groups: every group keeps CC and CS (2 + (2 + 2) / R)
    assert bench.mrhs_ops_per_term(4, 8) == 3.0
    assert bench.mrhs_ops_per_term(4, 12) == 3.0
    assert bench.mrhs_ops_per_term(2, 4) == 4.0
    # four groups or more: CC and CS once per pattern (4 / n_real)
    assert bench.mrhs_ops_per_term(4, 16) == pytest.approx(2.0 + 0.5 + 4.0 / 16)
    assert bench.mrhs_ops_per_term(4, 64) == pytest.approx(2.5625)
    assert bench.mrhs_ops_per_term(8, 64) == pytest.approx(2.3125)
    # sharing never costs more than one at a time
    for R in (2, 4, 8):
        for n_real in range(R, 200):
            assert bench.mrhs_ops_per_term(R, n_real) < 6.0


def test_compact_rounds_floats_only():
    v = {"a": 1.23456789, "b": [2.000049, 7], "c": "x", "d": float("nan"), "e": {"f": 123456.789}}
    out = bench._compact(v)
    assert out["a"] == 1.235 and out["b"] == [2.0, 7] and out["c"] == "x"
    assert out["d"] != out["d"] and out["e"]["f"] == 123500.0
    json.dumps(out)


def test_recorded_traffic_matches_current_sources():
    # the profiles record DRAM bytes per launch against a hash of the kernel
    # sources; a record taken on other sources must read as unknown (None)
    for kernel, profile, files in (("ls_main_kernel<24,4>", "ls_main_gapped_100k.md", bench.MAIN_SOURCES),
                                   ("gls_main_kernel<16,5>", "gls_main_gapped_100k_errors.md", bench.GLS_SOURCES)):
        got = bench._recorded_traffic(kernel, profile, files)
        assert got is None or got > 0
        assert bench._recorded_traffic(kernel + "x", profile, files) is None
